"""The C-ABI library builds, loads and exports every entry point declared in
include/adafac.h; host-side argument checks work without a GPU."""
import ctypes
import os
import re

import pytest

from paper_1903_10367_gb300 import adafac

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "adafac.h")).read()
    return sorted(set(re.findall(r"\b(adafac_[a-z_]+)\s*\(", text)))


def test_library_builds_and_exports_every_declared_symbol():
    lib = adafac.load()
    names = _declared()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name
    # the binding declares exactly the header's entry points
    assert sorted(n for n, _, _ in adafac._SIGNATURES) == names


def test_library_is_in_tree():
    lib = adafac.load()
    assert os.path.commonpath([lib._name, ROOT]) == ROOT


def test_default_options():
    o = adafac.default_options()
    assert (o.variant, o.transfer, o.precision, o.rtilde, o.form) == (1, 0, 0, 0, 0)
    assert o.omega == 0.6 and o.omega_tilde == 0.6 and o.inner_cycles >= 1


def test_workspace_size_grows_with_depth_and_mixed_needs_fp32_copies():
    o = adafac.default_options()
    s3 = adafac.workspace_size(2, 3, o)
    s4 = adafac.workspace_size(2, 4, o)
    assert 0 < s3 < s4
    m = adafac.default_options(precision="mixed")
    assert adafac.workspace_size(2, 4, m) > 0


@pytest.mark.parametrize("dim,depth", [(4, 3), (2, 0), (3, 20)])
def test_invalid_tree_is_rejected(dim, depth):
    with pytest.raises(adafac.AdafacError) as ei:
        adafac.workspace_size(dim, depth, adafac.default_options())
    assert ei.value.status == 1


def test_invalid_options_are_rejected():
    bad = adafac.default_options(form="fas", precision="mixed")
    with pytest.raises(adafac.AdafacError) as ei:
        adafac.workspace_size(2, 3, bad)
    assert "FAS" in str(ei.value)
    bad = adafac.default_options()
    bad.inner_cycles = 0
    with pytest.raises(adafac.AdafacError):
        adafac.workspace_size(2, 3, bad)


def test_setup_rejects_bad_eps_before_touching_the_device():
    lib = adafac.load()
    h = ctypes.c_void_p()
    eps = (ctypes.c_double * 1)(-1.0)
    o = adafac.default_options()
    st = lib.adafac_setup(ctypes.byref(adafac.Tree(2, 2)), ctypes.cast(eps, ctypes.c_void_p), 1,
                          None, 0, ctypes.byref(o), None, 0, None, ctypes.byref(h))
    assert st == 1 and not h.value
    assert b"eps" in lib.adafac_last_error(None)


@pytest.mark.parametrize("dim", [2, 3])
def test_workspace_layout_is_consistent_for_every_option_combination(dim):
    # adafac_workspace_size lays the arrays out twice (measuring and against a
    # fake base) and fails on any difference
    for variant in adafac.VARIANT:
        for transfer in adafac.TRANSFER:
            for precision in adafac.PRECISION:
                for rtilde in adafac.RTILDE:
                    for form in adafac.FORM:
                        if form == "fas" and precision == "mixed":
                            continue
                        o = adafac.default_options(variant=variant, transfer=transfer,
                                                   precision=precision, rtilde=rtilde, form=form)
                        assert adafac.workspace_size(dim, 3, o) > 0


def test_server_arguments_are_checked_before_any_device_call():
    lib = adafac.load()
    out = ctypes.c_void_p()
    assert lib.adafac_server_create(1 << 20, 0, 4, ctypes.byref(out)) == 1
    assert lib.adafac_server_create(1 << 20, 4, 0, ctypes.byref(out)) == 1
    assert lib.adafac_server_create(16, 4, 4, ctypes.byref(out)) == 1
    assert lib.adafac_server_create(1 << 20, 4, 4, None) == 1
    assert not out.value
    info = adafac.RequestInfo()
    assert lib.adafac_poll(None, 1, ctypes.byref(info)) == 1
    assert lib.adafac_fetch(None, 1, None) == 1
    assert lib.adafac_server_destroy(None) == 1


def _c_layout(struct, fields):
    """sizeof and offsetof of a header struct, from a C program compiled
    against include/adafac.h with the host compiler."""
    import shutil
    import subprocess
    import tempfile
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no host C compiler")
    body = "\n".join(f'  printf("%zu\\n", offsetof({struct}, {f}));' for f in fields)
    src = f"""#include <stddef.h>
#include <stdio.h>
#include "adafac.h"
int main(void) {{
  printf("%zu\\n", sizeof({struct}));
{body}
  return 0;
}}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        open(c, "w").write(src)
        subprocess.run([cc, "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    return [int(v) for v in out]


@pytest.mark.parametrize("struct,cls", [("adafac_tree", adafac.Tree),
                                        ("adafac_options", adafac.Options),
                                        ("adafac_tuning", adafac.Tuning),
                                        ("adafac_request_info", adafac.RequestInfo)])
def test_binding_structs_match_the_header_layout(struct, cls):
    names = [n for n, _ in cls._fields_]
    got = _c_layout(struct, names)
    assert got[0] == ctypes.sizeof(cls)
    assert got[1:] == [getattr(cls, n).offset for n in names]


def test_autotune_and_path_arguments_are_checked_on_the_host():
    lib = adafac.load()
    t = adafac.Tuning()
    assert lib.adafac_autotune(None, 5, ctypes.byref(t)) == 1
    assert adafac.workspace_size(3, 3, adafac.default_options(precision="mixed", path="generic")) > 0
    bad = adafac.default_options()
    bad.path = 3
    with pytest.raises(adafac.AdafacError):
        adafac.workspace_size(2, 3, bad)

"""The library serves plain C callers: a C program compiled against
include/adafac.h and linked with libadafac.so (no Python, no torch) calls the
host-side entry points.  None of the calls below touches a GPU."""
import os
import shutil
import subprocess

import pytest

from paper_1903_10367_gb300 import adafac

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "adafac.h"

int main(void) {
  adafac_options o;
  if (adafac_default_options(&o) != ADAFAC_OK) return 10;
  if (o.variant != ADAFAC_VARIANT_JAC || o.omega != 0.6) return 11;
  o.precision = ADAFAC_PRECISION_MIXED;
  o.transfer = ADAFAC_TRANSFER_BOXMG;
  adafac_tree t = {3, 4};
  size_t bytes = 0;
  if (adafac_workspace_size(&t, &o, &bytes) != ADAFAC_OK || bytes == 0) return 12;
  printf("%zu\n", bytes);
  /* invalid input is refused before any device work */
  double eps = -1.0;
  adafac_handle h = 0;
  if (adafac_setup(&t, &eps, 1, NULL, 0, &o, NULL, 0, NULL, &h) != ADAFAC_ERR_INVALID_ARG) return 13;
  if (h != 0 || strstr(adafac_last_error(NULL), "eps") == NULL) return 14;
  adafac_tuning tune;
  if (adafac_autotune(NULL, 5, &tune) != ADAFAC_ERR_INVALID_ARG) return 15;
  adafac_tree bad = {4, 2};
  if (adafac_workspace_size(&bad, &o, &bytes) != ADAFAC_ERR_INVALID_ARG) return 16;
  if (adafac_destroy(NULL) != ADAFAC_OK) return 17;
  return 0;
}
"""


def test_a_c_program_links_and_calls_the_host_entry_points(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no host C compiler")
    lib = adafac.load()
    libdir = os.path.dirname(lib._name)
    src = tmp_path / "host.c"
    exe = tmp_path / "host"
    src.write_text(PROGRAM)
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-L", libdir, "-ladafac", f"-Wl,-rpath,{libdir}", "-o", str(exe)],
                   check=True)
    res = subprocess.run([str(exe)], capture_output=True, text=True)
    assert res.returncode == 0, (res.returncode, res.stderr)
    opts = adafac.default_options(precision="mixed", transfer="boxmg")
    assert int(res.stdout.split()[0]) == adafac.workspace_size(3, 4, opts)

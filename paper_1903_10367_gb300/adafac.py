"""Thin Python binding of the adAFAC C ABI (include/adafac.h).

Argument marshalling only: every numerical step runs in the CUDA kernels of
``libadafac.so``.  PyTorch provides the device workspace (a uint8 tensor) and
the CUDA stream.  The binding raises ``AdafacError`` on every non-zero status
and refuses to run without the compiled library: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

__all__ = [
    "AdafacError", "Tree", "Options", "Tuning", "load", "default_options", "workspace_size",
    "Solver", "AdaptiveSolver", "FIELD", "VARIANT", "TRANSFER", "PRECISION", "RTILDE", "FORM",
]

VARIANT = {"additive": 0, "jac": 1, "pi": 2, "exp": 3}
TRANSFER = {"dlinear": 0, "boxmg": 1}
PRECISION = {"fp64": 0, "mixed": 1}
RTILDE = {"truncated": 0, "exact": 1}
FORM = {"cs": 0, "fas": 1}
PATH = {"auto": 0, "levelwise": 1, "generic": 2, "batched": 3}
FIELD = {"u": 0, "b": 1, "r": 2, "bt": 3, "g": 4, "t": 5, "P": 6, "stencil": 7, "invdiag": 8,
         "active": 9}
COARSE = {"galerkin": 0, "rediscretised": 1}
KERNEL = {"fine_residual": 0, "fine_update": 1, "fine_restrict": 2, "refine": 3,
          "fine_down": 4, "fine_up": 5, "fine_down_u": 6, "batch_step": 7}
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "DIVERGED", 4: "TIMEOUT", 5: "CUDA",
          6: "NOT_CONVERGED"}


class AdafacError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"adafac {STATUS.get(status, status)}: {message}")
        self.status = status


class Tree(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("depth", ctypes.c_int)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int), ("status", ctypes.c_int), ("cycles", ctypes.c_int),
                ("rel", ctypes.c_double), ("queue_ms", ctypes.c_double),
                ("latency_ms", ctypes.c_double)]


REQUEST_STATE = {0: "pending", 1: "running", 2: "done", 3: "failed"}


class Tuning(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int), ("cached", ctypes.c_int), ("sweep_nz", ctypes.c_int),
                ("sweep_nz_down", ctypes.c_int), ("res_bx", ctypes.c_int),
                ("res_by", ctypes.c_int), ("res_zr", ctypes.c_int), ("upd_bx", ctypes.c_int),
                ("upd_by", ctypes.c_int), ("candidates", ctypes.c_int),
                ("us_default", ctypes.c_double), ("us_tuned", ctypes.c_double)]


class Options(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("transfer", ctypes.c_int),
                ("precision", ctypes.c_int), ("rtilde", ctypes.c_int),
                ("form", ctypes.c_int), ("inner_cycles", ctypes.c_int),
                ("omega", ctypes.c_double), ("omega_tilde", ctypes.c_double),
                ("omega_exp", ctypes.c_double), ("path", ctypes.c_int),
                ("coarse_op", ctypes.c_int), ("lmin", ctypes.c_int)]


_LIB = None

# (name, restype, argtypes) of every entry point declared in include/adafac.h
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_SIGNATURES = [
    ("adafac_default_options", _I, [ctypes.POINTER(Options)]),
    ("adafac_workspace_size", _I, [ctypes.POINTER(Tree), ctypes.POINTER(Options),
                                   ctypes.POINTER(ctypes.c_size_t)]),
    ("adafac_setup", _I, [ctypes.POINTER(Tree), _P, _I, _P, _I, ctypes.POINTER(Options),
                          _P, ctypes.c_size_t, _P, ctypes.POINTER(_P)]),
    ("adafac_cycle", _I, [_P, _I]),
    ("adafac_solve", _I, [_P, _D, _I, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    ("adafac_residual_norm", _I, [_P, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    ("adafac_solution", _I, [_P, _P, _I]),
    ("adafac_set_solution", _I, [_P, _P, _I]),
    ("adafac_set_boundary", _I, [_P, _P, _I]),
    ("adafac_reset", _I, [_P]),
    ("adafac_set_wait_limit", _I, [_P, ctypes.c_longlong]),
    ("adafac_set_batch_cluster", _I, [_P, _I]),
    ("adafac_batch_cluster", _I, [_P, ctypes.POINTER(_I)]),
    ("adafac_get_field", _I, [_P, _I, _I, _P, _I, ctypes.POINTER(ctypes.c_size_t)]),
    ("adafac_history", _I, [_P, _P, _I, ctypes.POINTER(_I)]),
    ("adafac_launch_count", _I, [_P, ctypes.POINTER(ctypes.c_uint64)]),
    ("adafac_timing", _I, [_P, _I]),
    ("adafac_timing_read", _I, [_P, _I, ctypes.POINTER(_D), ctypes.POINTER(_I)]),
    ("adafac_autotune", _I, [_P, _I, ctypes.POINTER(Tuning)]),
    ("adafac_residual_norm_static", _I, [_I, _I, _D, _P, _P, _P, _P]),
    ("adafac_server_create", _I, [ctypes.c_size_t, _I, _I, ctypes.POINTER(_P)]),
    ("adafac_submit", _I, [_P, ctypes.POINTER(Tree), _P, _I, _P, ctypes.POINTER(Options), _D,
                           _I, ctypes.POINTER(ctypes.c_int64)]),
    ("adafac_poll", _I, [_P, ctypes.c_int64, ctypes.POINTER(RequestInfo)]),
    ("adafac_fetch", _I, [_P, ctypes.c_int64, _P]),
    ("adafac_server_stats", _I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I),
                                 ctypes.POINTER(ctypes.c_size_t)]),
    ("adafac_server_destroy", _I, [_P]),
    ("adafac_adaptive_setup", _I, [_I, _I, ctypes.POINTER(_P), _P, _I, _P, ctypes.POINTER(Options),
                                   _P, ctypes.POINTER(_P)]),
    ("adafac_adaptive_cycle", _I, [_P, _I]),
    ("adafac_adaptive_residual_norm", _I, [_P, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    ("adafac_adaptive_solve", _I, [_P, _D, _I, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    ("adafac_adaptive_nodes", _I, [_P, _P, ctypes.POINTER(ctypes.c_int64)]),
    ("adafac_adaptive_solution", _I, [_P, _P]),
    ("adafac_adaptive_set_solution", _I, [_P, _P]),
    ("adafac_adaptive_level", _I, [_P, _I, _I, _P, ctypes.POINTER(ctypes.c_int64)]),
    ("adafac_adaptive_transfer", _I, [_P, _P]),
    ("adafac_adaptive_last_error", ctypes.c_char_p, [_P]),
    ("adafac_adaptive_destroy", _I, [_P]),
    ("adafac_last_error", ctypes.c_char_p, [_P]),
    ("adafac_destroy", _I, [_P]),
]


def load(build_if_missing: bool = True):
    """Loads (building if needed) the shared library and declares its symbols."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if not os.path.exists(path) or not _build.up_to_date():
        if not build_if_missing:
            raise AdafacError(5, f"library not built: {path}")
        path = _build.build()
    lib = ctypes.CDLL(path)
    for name, res, args in _SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _check(status: int, handle=None):
    if status != 0:
        msg = _LIB.adafac_last_error(handle).decode(errors="replace")
        raise AdafacError(status, msg)


def default_options(**kw) -> Options:
    lib = load()
    o = Options()
    _check(lib.adafac_default_options(ctypes.byref(o)))
    for k, v in kw.items():
        table = {"variant": VARIANT, "transfer": TRANSFER, "precision": PRECISION,
                 "rtilde": RTILDE, "form": FORM, "path": PATH, "coarse_op": COARSE}.get(k)
        setattr(o, k, table[v] if table and isinstance(v, str) else v)
    return o


def workspace_size(dim: int, depth: int, opts: Options) -> int:
    lib = load()
    n = ctypes.c_size_t()
    _check(lib.adafac_workspace_size(ctypes.byref(Tree(dim, depth)), ctypes.byref(opts),
                                     ctypes.byref(n)))
    return n.value


def residual_norm_static(dim: int, depth: int, eps: float, u, b, norm, stream=None):
    """sqrt(h^dim * sum over interior vertices of r^2), r = b - A u with the
    uniform d-linear stencil of -div(eps grad u), on device tensors u, b
    ((3^depth+1)^dim float64 each; u's boundary ring holds the Dirichlet
    values, b's is ignored), written into the 1-element float64 device tensor
    ``norm`` on ``stream`` (default: torch's current stream).  The library
    allocates nothing for this call (adafac_residual_norm_static), for callers
    that cannot allocate device memory."""
    import torch
    lib = load()
    for t in (u, b, norm):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
                and t.is_contiguous()):
            raise TypeError("u, b and norm must be contiguous float64 CUDA tensors")
    V = (3 ** depth + 1) ** dim
    if u.numel() != V or b.numel() != V or norm.numel() < 1:
        raise ValueError("u and b must hold (3^depth + 1)^dim values, norm at least one")
    s = torch.cuda.current_stream() if stream is None else stream
    st = lib.adafac_residual_norm_static(dim, depth, float(eps), ctypes.c_void_p(u.data_ptr()),
                                         ctypes.c_void_p(b.data_ptr()),
                                         ctypes.c_void_p(norm.data_ptr()),
                                         ctypes.c_void_p(s.cuda_stream))
    if st != 0:
        raise AdafacError(st, "adafac_residual_norm_static failed")


def _host_ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Solver:
    """One adAFAC problem on the current CUDA device.

    ``eps``: per-fine-cell array (shape (3^L,)*dim) or a scalar; ``f``: values
    at every fine vertex (shape (3^L+1,)*dim) or None.  Host numpy arrays or
    torch CUDA tensors (float64, contiguous) are accepted.
    """

    def __init__(self, dim: int, depth: int, eps, f=None, opts: Options | None = None,
                 workspace=None, stream=None):
        import torch
        self._torch = torch
        self.lib = load()
        self.dim, self.depth = dim, depth
        self.n = 3 ** depth
        self.shape = (self.n + 1,) * dim
        self.opts = opts if opts is not None else default_options()
        eps_is_scalar = np.isscalar(eps) or (hasattr(eps, "numel") and eps.numel() == 1) or \
            (isinstance(eps, np.ndarray) and eps.size == 1)
        on_device = hasattr(eps, "is_cuda") and eps.is_cuda
        keep = []
        if on_device:
            eps_t = eps.to(torch.float64).contiguous().reshape(-1)
            f_t = None if f is None else f.to(torch.float64).contiguous()
            keep += [eps_t, f_t]
            eps_p = ctypes.c_void_p(eps_t.data_ptr())
            f_p = None if f_t is None else ctypes.c_void_p(f_t.data_ptr())
        else:
            eps_a = np.ascontiguousarray(np.asarray(eps, dtype=np.float64).reshape(-1))
            f_a = None if f is None else np.ascontiguousarray(np.asarray(f, dtype=np.float64))
            if f_a is not None and f_a.shape != self.shape:
                raise ValueError(f"f must have shape {self.shape}")
            if not eps_is_scalar and eps_a.size != self.n ** dim:
                raise ValueError(f"eps must have {self.n ** dim} entries")
            keep += [eps_a, f_a]
            eps_p = _host_ptr(eps_a)
            f_p = None if f_a is None else _host_ptr(f_a)
        nbytes = workspace_size(dim, depth, self.opts)
        if workspace is None:
            workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        self._ws = workspace
        base = workspace.data_ptr()
        aligned = (base + 255) & ~255
        avail = workspace.numel() - (aligned - base)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.h = ctypes.c_void_p()
        _check(self.lib.adafac_setup(ctypes.byref(Tree(dim, depth)), eps_p, int(eps_is_scalar),
                                     f_p, int(on_device), ctypes.byref(self.opts),
                                     ctypes.c_void_p(aligned), avail,
                                     ctypes.c_void_p(self.stream.cuda_stream),
                                     ctypes.byref(self.h)))
        del keep

    # -- the C ABI, one method per entry point -----------------------------
    def cycle(self, n: int = 1):
        _check(self.lib.adafac_cycle(self.h, int(n)), self.h)

    def solve(self, rel_tol: float = 1e-8, max_cycles: int = 1000, check: bool = True):
        cycles = ctypes.c_int()
        rel = ctypes.c_double()
        st = self.lib.adafac_solve(self.h, rel_tol, int(max_cycles), ctypes.byref(cycles),
                                   ctypes.byref(rel))
        if check:
            _check(st, self.h)
        return cycles.value, rel.value

    def residual_norm(self):
        rel = ctypes.c_double()
        ab = ctypes.c_double()
        _check(self.lib.adafac_residual_norm(self.h, ctypes.byref(rel), ctypes.byref(ab)), self.h)
        return rel.value, ab.value

    def solution(self, out=None):
        if out is None:
            out = np.empty(self.shape)
        if isinstance(out, np.ndarray):
            _check(self.lib.adafac_solution(self.h, _host_ptr(out), 0), self.h)
        else:
            _check(self.lib.adafac_solution(self.h, ctypes.c_void_p(out.data_ptr()), 1), self.h)
        return out

    def set_wait_limit(self, polls: int):
        """Poll limit of the sweeps' bounded waits (0: every wait gives up at
        once, which exercises the timeout path)."""
        _check(self.lib.adafac_set_wait_limit(self.h, int(polls)), self.h)

    def set_batch_cluster(self, ctas: int):
        """CTAs per instance of the batched path (a power of two)."""
        _check(self.lib.adafac_set_batch_cluster(self.h, int(ctas)), self.h)

    def batch_cluster(self) -> int:
        c = _I(0)
        _check(self.lib.adafac_batch_cluster(self.h, ctypes.byref(c)), self.h)
        return c.value

    def set_solution(self, u):
        if isinstance(u, np.ndarray):
            a = np.ascontiguousarray(u, dtype=np.float64)
            _check(self.lib.adafac_set_solution(self.h, _host_ptr(a), 0), self.h)
        else:
            _check(self.lib.adafac_set_solution(self.h, ctypes.c_void_p(u.data_ptr()), 1), self.h)

    def set_boundary(self, g):
        """Dirichlet values: the boundary entries of g (a (3^L+1)^dim array)."""
        g = np.ascontiguousarray(np.asarray(g, dtype=np.float64))
        _check(self.lib.adafac_set_boundary(self.h, _host_ptr(g), 0), self.h)

    def reset(self):
        _check(self.lib.adafac_reset(self.h), self.h)

    def field(self, name: str, level: int) -> np.ndarray:
        count = ctypes.c_size_t()
        _check(self.lib.adafac_get_field(self.h, FIELD[name], level, None, 0,
                                         ctypes.byref(count)), self.h)
        out = np.empty(count.value)
        _check(self.lib.adafac_get_field(self.h, FIELD[name], level, _host_ptr(out), 0,
                                         ctypes.byref(count)), self.h)
        nl = 3 ** level
        V = (nl + 1) ** self.dim
        if out.size == V:
            return out.reshape((nl + 1,) * self.dim)
        return out.reshape((-1,) + (nl + 1,) * self.dim)

    def history(self) -> np.ndarray:
        count = ctypes.c_int()
        _check(self.lib.adafac_history(self.h, None, 0, ctypes.byref(count)), self.h)
        out = np.empty(max(count.value, 1))
        _check(self.lib.adafac_history(self.h, _host_ptr(out), count.value,
                                       ctypes.byref(count)), self.h)
        return out[:count.value]

    def launch_count(self) -> int:
        c = ctypes.c_uint64()
        _check(self.lib.adafac_launch_count(self.h, ctypes.byref(c)), self.h)
        return c.value

    def timing(self, enable: bool):
        _check(self.lib.adafac_timing(self.h, int(enable)), self.h)

    def timing_read(self, kind: str):
        ms = ctypes.c_double()
        n = ctypes.c_int()
        _check(self.lib.adafac_timing_read(self.h, KERNEL[kind], ctypes.byref(ms),
                                           ctypes.byref(n)), self.h)
        return ms.value, n.value

    def autotune(self, repeats: int = 5) -> dict:
        """Times candidate launch shapes of the fine-level kernels and keeps
        the fastest (adafac_autotune); returns the tuning record."""
        t = Tuning()
        _check(self.lib.adafac_autotune(self.h, int(repeats), ctypes.byref(t)), self.h)
        return {name: getattr(t, name) for name, _ in Tuning._fields_}

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.lib.adafac_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Server:
    """Continuous-batching request server (adafac_server_*): solves submitted
    from the host are admitted by device-memory footprint, run concurrently on
    the server's streams and return their solutions to host memory.  Requests
    on the batched path share launches.  Start the process with
    CUDA_DEVICE_MAX_CONNECTIONS=32 (before anything creates the CUDA
    context) so that the streams get hardware work queues of their own."""

    def __init__(self, device_bytes: int, n_streams: int = 16, max_running: int = 64):
        self.lib = load()
        self.s = ctypes.c_void_p()
        st = self.lib.adafac_server_create(int(device_bytes), int(n_streams), int(max_running),
                                           ctypes.byref(self.s))
        if st != 0:
            raise AdafacError(st, "adafac_server_create failed")

    def submit(self, dim: int, depth: int, eps, f=None, opts: Options | None = None,
               rel_tol: float = 1e-8, max_cycles: int = 2000) -> int:
        opts = opts or default_options()
        eps_is_scalar = np.isscalar(eps)
        e = np.ascontiguousarray(np.atleast_1d(np.asarray(eps, dtype=np.float64)))
        fa = None if f is None else np.ascontiguousarray(np.asarray(f, dtype=np.float64))
        t = ctypes.c_int64()
        st = self.lib.adafac_submit(self.s, ctypes.byref(Tree(dim, depth)), _host_ptr(e),
                                    int(eps_is_scalar), None if fa is None else _host_ptr(fa),
                                    ctypes.byref(opts), float(rel_tol), int(max_cycles),
                                    ctypes.byref(t))
        if st != 0:
            raise AdafacError(st, "adafac_submit failed")
        self._shapes = getattr(self, "_shapes", {})
        self._shapes[t.value] = (3 ** depth + 1,) * dim
        return t.value

    def poll(self, ticket: int) -> dict:
        info = RequestInfo()
        st = self.lib.adafac_poll(self.s, ctypes.c_int64(ticket), ctypes.byref(info))
        if st != 0:
            raise AdafacError(st, "adafac_poll: unknown ticket")
        return {"state": REQUEST_STATE[info.state], "status": info.status, "cycles": info.cycles,
                "rel": info.rel, "queue_ms": info.queue_ms, "latency_ms": info.latency_ms}

    def fetch(self, ticket: int) -> np.ndarray:
        out = np.empty(self._shapes[ticket])
        st = self.lib.adafac_fetch(self.s, ctypes.c_int64(ticket), _host_ptr(out))
        del self._shapes[ticket]
        if st != 0:
            raise AdafacError(st, f"request {ticket} ended with status {st}")
        return out

    def stats(self):
        p, r, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
        _check(self.lib.adafac_server_stats(self.s, ctypes.byref(p), ctypes.byref(r),
                                            ctypes.byref(b)))
        return p.value, r.value, b.value

    def close(self):
        if self.s:
            self.lib.adafac_server_destroy(self.s)
            self.s = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class AdaptiveSolver:
    """adAFAC on a static adaptive spacetree (adafac_adaptive_*; FP64, or
    MIXED refinement steps on the per-level grid engine).

    ``refine``: for l = 1 .. depth-1 an array of shape (3^l,)*dim (array axis
    order, the last axis is x) whose non-zero entries cut existing level-l
    cells; ``eps`` a scalar or one value per finest cell (shape (3^depth,)*dim);
    ``f`` the load density at the finest-level positions (shape
    (3^depth + 1,)*dim) or None.  The iterate lives at the leaf nodes, in the
    order of ``nodes()`` (ascending finest-level grid index)."""

    def __init__(self, dim: int, depth: int, refine, eps, f=None, opts: Options | None = None,
                 stream=None):
        import torch
        self.lib = load()
        self.dim, self.depth = dim, depth
        n = 3 ** depth
        self.opts = opts if opts is not None else default_options()
        flags = [np.ascontiguousarray(np.asarray(refine[l - 1]).astype(np.uint8).reshape(-1))
                 for l in range(1, depth)]
        for l, a in enumerate(flags, start=1):
            if a.size != 3 ** (l * dim):
                raise ValueError(f"refine flags of level {l} must have {3 ** (l * dim)} entries")
        ptrs = (ctypes.c_void_p * max(len(flags), 1))(*[a.ctypes.data for a in flags])
        eps_a = np.ascontiguousarray(np.asarray(eps, dtype=np.float64).reshape(-1))
        scalar = eps_a.size == 1
        if not scalar and eps_a.size != n ** dim:
            raise ValueError(f"eps must be a scalar or have {n ** dim} entries")
        f_a = None if f is None else np.ascontiguousarray(np.asarray(f, dtype=np.float64))
        if f_a is not None and f_a.shape != (n + 1,) * dim:
            raise ValueError(f"f must have shape {(n + 1,) * dim}")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.h = ctypes.c_void_p()
        st = self.lib.adafac_adaptive_setup(dim, depth, ptrs, _host_ptr(eps_a), int(scalar),
                                            None if f_a is None else _host_ptr(f_a),
                                            ctypes.byref(self.opts),
                                            ctypes.c_void_p(self.stream.cuda_stream),
                                            ctypes.byref(self.h))
        if st != 0:
            raise AdafacError(st, "adafac_adaptive_setup failed")
        count = ctypes.c_int64()
        self._check(self.lib.adafac_adaptive_nodes(self.h, None, ctypes.byref(count)))
        self.count = count.value

    def _check(self, st):
        if st != 0:
            msg = self.lib.adafac_adaptive_last_error(self.h)
            raise AdafacError(st, msg.decode() if msg else "")

    def cycle(self, n: int = 1):
        self._check(self.lib.adafac_adaptive_cycle(self.h, int(n)))

    def residual_norm(self):
        rel, ab = ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.adafac_adaptive_residual_norm(self.h, ctypes.byref(rel),
                                                           ctypes.byref(ab)))
        return rel.value, ab.value

    def solve(self, rel_tol: float = 1e-8, max_cycles: int = 2000, check: bool = True):
        cycles, rel = ctypes.c_int(), ctypes.c_double()
        st = self.lib.adafac_adaptive_solve(self.h, rel_tol, int(max_cycles), ctypes.byref(cycles),
                                            ctypes.byref(rel))
        if check:
            self._check(st)
        return cycles.value, rel.value

    def nodes(self) -> np.ndarray:
        out = np.empty(self.count, dtype=np.int64)
        count = ctypes.c_int64()
        self._check(self.lib.adafac_adaptive_nodes(self.h, _host_ptr(out), ctypes.byref(count)))
        return out

    def solution(self) -> np.ndarray:
        out = np.empty(self.count)
        self._check(self.lib.adafac_adaptive_solution(self.h, _host_ptr(out)))
        return out

    def set_solution(self, u):
        a = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(-1))
        if a.size != self.count:
            raise ValueError(f"the iterate has {self.count} leaf-node values")
        self._check(self.lib.adafac_adaptive_set_solution(self.h, _host_ptr(a)))

    def transfer_from(self, other: "AdaptiveSolver"):
        """Takes the iterate of a solver on another tree of the same depth:
        the old function at this tree's vertices, rebuilt in this tree's
        space (new and hanging vertices d-linearly interpolated), with the
        other solver's r_0 as the normalisation."""
        self._check(self.lib.adafac_adaptive_transfer(self.h, other.h))

    def level(self, name: str, level: int) -> np.ndarray:
        count = ctypes.c_int64()
        self._check(self.lib.adafac_adaptive_level(self.h, FIELD[name], level, None,
                                                   ctypes.byref(count)))
        out = np.empty(count.value)
        self._check(self.lib.adafac_adaptive_level(self.h, FIELD[name], level, _host_ptr(out),
                                                   ctypes.byref(count)))
        return out

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.lib.adafac_adaptive_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

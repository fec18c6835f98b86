"""Thin ctypes binding of libshl (include/shl.h).

Argument marshalling only: every step of the path runs in the CUDA library.
Device buffers are torch CUDA tensors (their data_ptr() is passed); host
outputs are numpy arrays.  The library must have been built
(``paper_2511_04025_b300.build``); loading fails loudly otherwise, and there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libshl.so")

SHL_OK, SHL_EINVAL, SHL_ENOMEM, SHL_ENOCONV, SHL_ENUMERIC, SHL_ECUDA, SHL_EAGAIN, SHL_ENOTFOUND = range(8)
SHL_FP64, SHL_FP32_REFINE = 0, 1
SHL_MASK, SHL_SMOOTH = 0, 1
SHL_PRECOND_JACOBI, SHL_PRECOND_MG = 0, 1
STATUS_NAMES = ["SHL_OK", "SHL_EINVAL", "SHL_ENOMEM", "SHL_ENOCONV", "SHL_ENUMERIC", "SHL_ECUDA", "SHL_EAGAIN",
                "SHL_ENOTFOUND"]

_dp = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p
_i64p = ctypes.POINTER(ctypes.c_int64)


class shl_opts(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("hbm_budget_bytes", ctypes.c_uint64)]


class shl_design(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("K", ctypes.c_int32), ("pos", _dp), ("q", _dp), ("alpha", _dp),
                ("iso", ctypes.c_double), ("t", ctypes.c_double), ("vf", ctypes.c_double)]


class shl_solve_opts(ctypes.Structure):
    _fields_ = [("E", ctypes.c_double), ("nu", ctypes.c_double), ("E_void", ctypes.c_double),
                ("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("density", ctypes.c_int32), ("warm_start", ctypes.c_int32), ("kappa", ctypes.c_double),
                ("inner_tol", ctypes.c_double), ("precond", ctypes.c_int32), ("mg_nu", ctypes.c_int32),
                ("mg_omega", ctypes.c_double), ("active", ctypes.c_int32), ("cull", ctypes.c_double),
                ("mg_nu_coarse", ctypes.c_int32), ("mg_gamma", ctypes.c_int32)]


class shl_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32 * 6), ("relres", ctypes.c_double * 6), ("n_refine", ctypes.c_int32),
                ("status", ctypes.c_int32), ("t", ctypes.c_double), ("margin", ctypes.c_double),
                ("n_solid", ctypes.c_int64), ("n_ambiguous", ctypes.c_int64), ("ms_field", ctypes.c_float),
                ("ms_rhs", ctypes.c_float), ("ms_solve", ctypes.c_float), ("ms_chom", ctypes.c_float),
                ("precond", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return dict(iters=list(self.iters), relres=list(self.relres), n_refine=self.n_refine, status=self.status,
                    t=self.t, margin=self.margin, n_solid=self.n_solid, n_ambiguous=self.n_ambiguous,
                    ms_field=self.ms_field, ms_solve=self.ms_solve, ms_chom=self.ms_chom, precond=self.precond)


class shl_request(ctypes.Structure):
    _fields_ = [("design", shl_design), ("r", ctypes.c_int32), ("opts", shl_solve_opts), ("session", ctypes.c_int64)]


class shl_result(ctypes.Structure):
    _fields_ = [("C", ctypes.c_double * 36), ("stats", shl_stats), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double), ("warm", ctypes.c_int32),
                ("slot", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return dict(C=np.array(self.C).reshape(6, 6), stats=self.stats.as_dict(), t_submit=self.t_submit,
                    t_admit=self.t_admit, t_done=self.t_done, warm=bool(self.warm), slot=self.slot)


class shl_serve_info(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("queued", ctypes.c_int32), ("running", ctypes.c_int32),
                ("completed", ctypes.c_uint64), ("held_bytes", ctypes.c_uint64), ("budget_bytes", ctypes.c_uint64)]


# Every symbol include/shl.h declares, with its ctypes signature.
SIGNATURES = {
    "shl_create": (ctypes.c_int, [ctypes.POINTER(shl_opts), ctypes.POINTER(_vp)]),
    "shl_destroy": (ctypes.c_int, [_vp]),
    "shl_last_error": (ctypes.c_char_p, [_vp]),
    "shl_default_solve_opts": (None, [ctypes.POINTER(shl_solve_opts)]),
    "shl_field": (ctypes.c_int, [_vp, ctypes.POINTER(shl_design), ctypes.c_int32, _vp, _vp, _vp]),
    "shl_voxelize": (ctypes.c_int, [_vp, ctypes.POINTER(shl_design), ctypes.c_int32, ctypes.c_double, _vp, _vp, _vp,
                                    _dp, _dp, _i64p, _i64p, _vp]),
    "shl_apply": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_int32, ctypes.c_int32, _vp, _vp, _vp]),
    "shl_rhs": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                               _vp, _vp]),
    "shl_chom": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                _vp, _dp, _vp]),
    "shl_solve": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp, ctypes.POINTER(shl_solve_opts), _vp, _dp,
                                 ctypes.POINTER(shl_stats), _vp]),
    "shl_homogenize": (ctypes.c_int, [_vp, ctypes.POINTER(shl_design), ctypes.c_int32,
                                      ctypes.POINTER(shl_solve_opts), _dp, ctypes.POINTER(shl_stats), _vp]),
    "shl_homogenize_batch": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.POINTER(shl_design),
                                            ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(shl_solve_opts), _dp,
                                            ctypes.POINTER(shl_stats), _vp]),
    "shl_get_counters": (ctypes.c_int, [_vp, ctypes.c_void_p]),
    "shl_probe_peaks": (ctypes.c_int, [_vp, ctypes.c_void_p]),
    "shl_probe_wait_timeout": (ctypes.c_int, [_vp, ctypes.c_uint32, ctypes.POINTER(ctypes.c_int32)]),
    "shl_chom_noalloc": (ctypes.c_int, [ctypes.c_int32, _vp, _vp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        _vp, _vp, _vp]),
    "shl_grad": (ctypes.c_int, [_vp, ctypes.POINTER(shl_design), ctypes.c_int32, ctypes.POINTER(shl_solve_opts), _dp,
                                ctypes.c_double, _vp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, ctypes.POINTER(shl_stats),
                                _vp]),
    "shl_serve_submit": (ctypes.c_int, [_vp, ctypes.POINTER(shl_request), ctypes.POINTER(ctypes.c_uint64)]),
    "shl_serve_poll": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.POINTER(shl_result)]),
    "shl_serve_wait": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.POINTER(shl_result)]),
    "shl_serve_cancel": (ctypes.c_int, [_vp, ctypes.c_uint64]),
    "shl_serve_drain": (ctypes.c_int, [_vp]),
    "shl_serve_info_get": (ctypes.c_int, [_vp, ctypes.POINTER(shl_serve_info)]),
}

_lib = None


def lib():
    """Load libshl.so (no GPU needed to load).  Raises if it was not built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libshl.so not built at {LIB_PATH}: run paper_2511_04025_b300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class ShlError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


def _check(ctx, st: int, ok=(SHL_OK,)):
    if st not in ok:
        raise ShlError(st, lib().shl_last_error(ctx).decode())
    return st


def _ptr(t) -> Optional[int]:
    """Device pointer of a torch tensor (or None)."""
    if t is None:
        return None
    return int(t.data_ptr())


def _stream(stream) -> Optional[int]:
    if stream is None:
        return None
    return int(getattr(stream, "cuda_stream", stream))


class DesignArg:
    """Keeps the numpy arrays of a design alive while the C struct points at them."""

    def __init__(self, d, t: Optional[float] = None):
        self.pos = np.ascontiguousarray(d.pos, dtype=np.float64)
        self.q = np.ascontiguousarray(d.q, dtype=np.float64)
        self.alpha = None if d.alpha is None else np.ascontiguousarray(d.alpha, dtype=np.float64)
        tt = t if t is not None else (d.t if d.t is not None else 0.0)
        self.s = shl_design(
            n=self.pos.shape[0], K=d.K, pos=self.pos.ctypes.data_as(_dp), q=self.q.ctypes.data_as(_dp),
            alpha=self.alpha.ctypes.data_as(_dp) if self.alpha is not None else None, iso=float(d.iso),
            t=float(tt), vf=float(d.vf if d.vf is not None else 0.0))


def default_solve_opts(**kw) -> shl_solve_opts:
    o = shl_solve_opts()
    lib().shl_default_solve_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


# ---------------------------------------------------------------------------
# Same-name wrappers of the C entry points
# ---------------------------------------------------------------------------

_ctx_device = {}  # handle -> CUDA device ordinal it was created on


def shl_create(device: int = 0, max_batch: int = 0, hbm_budget_bytes: int = 0) -> int:
    o = shl_opts(device=device, max_batch=max_batch, hbm_budget_bytes=hbm_budget_bytes)
    out = _vp()
    st = lib().shl_create(ctypes.byref(o), ctypes.byref(out))
    if st != SHL_OK:
        raise ShlError(st, lib().shl_last_error(None).decode())
    _ctx_device[out.value] = device
    return out.value


def shl_destroy(ctx: int) -> None:
    _ctx_device.pop(ctx, None)
    lib().shl_destroy(ctx)


def ctx_device(ctx: int):
    """torch.device of the GPU a context (made by shl_create) runs on: buffers
    that the context's kernels read or write must be allocated there."""
    import torch
    if ctx not in _ctx_device:
        raise ValueError("ctx_device: handle was not created by shl_create in this process")
    return torch.device("cuda", _ctx_device[ctx])


def shl_field(ctx, design, r: int, F, gradF=None, stream=None):
    d = DesignArg(design)
    _check(ctx, lib().shl_field(ctx, ctypes.byref(d.s), r, _ptr(F), _ptr(gradF), _stream(stream)))


def shl_voxelize(ctx, design, r: int, kappa: float = 0.0, mask=None, rho=None, d=None, t: Optional[float] = None,
                 stream=None) -> dict:
    da = DesignArg(design, t)
    tt, mg = ctypes.c_double(), ctypes.c_double()
    ns, na = ctypes.c_int64(), ctypes.c_int64()
    _check(ctx, lib().shl_voxelize(ctx, ctypes.byref(da.s), r, kappa, _ptr(mask), _ptr(rho), _ptr(d),
                                   ctypes.byref(tt), ctypes.byref(mg), ctypes.byref(ns), ctypes.byref(na),
                                   _stream(stream)))
    return dict(t=tt.value, margin=mg.value, n_solid=ns.value, n_ambiguous=na.value)


def shl_apply(ctx, r: int, p, q, mask=None, rho=None, E=1.0, nu=0.3, E_void=1e-6, precision=None, nvec=None,
              stream=None):
    import torch
    if precision is None:
        precision = SHL_FP64 if p.dtype == torch.float64 else SHL_FP32_REFINE
    if nvec is None:
        nvec = p.shape[0] // 3
    _check(ctx, lib().shl_apply(ctx, r, _ptr(mask), _ptr(rho), E, nu, E_void, precision, nvec, _ptr(p), _ptr(q),
                                _stream(stream)))


def shl_rhs(ctx, r: int, f, mask=None, rho=None, E=1.0, nu=0.3, E_void=1e-6, stream=None):
    _check(ctx, lib().shl_rhs(ctx, r, _ptr(mask), _ptr(rho), E, nu, E_void, _ptr(f), _stream(stream)))


def shl_chom(ctx, r: int, u, mask=None, rho=None, E=1.0, nu=0.3, E_void=1e-6, stream=None) -> np.ndarray:
    C = np.zeros(36)
    _check(ctx, lib().shl_chom(ctx, r, _ptr(mask), _ptr(rho), E, nu, E_void, _ptr(u), C.ctypes.data_as(_dp),
                               _stream(stream)))
    return C.reshape(6, 6)


def shl_solve(ctx, r: int, opts: shl_solve_opts, mask=None, rho=None, u=None, stream=None):
    C = np.zeros(36)
    st = shl_stats()
    rc = lib().shl_solve(ctx, r, _ptr(mask), _ptr(rho), ctypes.byref(opts), _ptr(u), C.ctypes.data_as(_dp),
                         ctypes.byref(st), _stream(stream))
    _check(ctx, rc, ok=(SHL_OK, SHL_ENOCONV))
    return C.reshape(6, 6), st.as_dict()


def shl_homogenize(ctx, design, r: int, opts: shl_solve_opts, t: Optional[float] = None, stream=None):
    d = DesignArg(design, t)
    C = np.zeros(36)
    st = shl_stats()
    rc = lib().shl_homogenize(ctx, ctypes.byref(d.s), r, ctypes.byref(opts), C.ctypes.data_as(_dp),
                              ctypes.byref(st), _stream(stream))
    _check(ctx, rc, ok=(SHL_OK, SHL_ENOCONV))
    return C.reshape(6, 6), st.as_dict()


def shl_homogenize_batch(ctx, designs: Sequence, rs: Sequence[int], opts: shl_solve_opts, stream=None):
    args = [DesignArg(d) for d in designs]
    arr = (shl_design * len(args))(*[a.s for a in args])
    r_arr = (ctypes.c_int32 * len(args))(*rs)
    C = np.zeros(36 * len(args))
    st = (shl_stats * len(args))()
    rc = lib().shl_homogenize_batch(ctx, len(args), arr, r_arr, ctypes.byref(opts), C.ctypes.data_as(_dp), st,
                                    _stream(stream))
    _check(ctx, rc, ok=(SHL_OK, SHL_ENOCONV))
    return C.reshape(-1, 6, 6), [s.as_dict() for s in st]


NOALLOC_MAX_R = 512  # largest grid of shl_chom_noalloc (its fixed scratch)


def shl_chom_noalloc(r: int, u, C_dev, mask=None, rho=None, E=1.0, nu=0.3, E_void=1e-6, stream=None):
    """C^H into the 36-double device tensor C_dev without any device allocation
    by the library (for callers that cannot allocate); see include/shl.h.
    Every tensor must sit on C_dev's device, contiguous, with its dtype and at
    least its size (u: 18 r^3 float64; mask: r^3 uint8 or rho: r^3 float64;
    C_dev: 36 float64); the call runs with that device current."""
    import torch
    # a grid size the library rejects is passed through so that it reports it
    n = r ** 3 if 1 <= r <= NOALLOC_MAX_R else 0
    need = [("u", u, torch.float64, 18 * n), ("C_dev", C_dev, torch.float64, 36),
            ("mask", mask, torch.uint8, n), ("rho", rho, torch.float64, n)]
    for name, t, dt, size in need:
        if t is None:
            continue
        if not (t.is_cuda and t.device == C_dev.device):
            raise ValueError(f"shl_chom_noalloc: {name} must be on {C_dev.device}, got {t.device}")
        if t.dtype != dt or not t.is_contiguous() or t.numel() < size:
            raise ValueError(f"shl_chom_noalloc: {name} must be a contiguous {dt} tensor of >= {size} elements")
    with torch.cuda.device(C_dev.device):
        _check(None, lib().shl_chom_noalloc(r, _ptr(mask), _ptr(rho), E, nu, E_void, _ptr(u), _ptr(C_dev),
                                            _stream(stream)))


def shl_grad(ctx, design, r: int, opts: shl_solve_opts, dEdC, u=None, t: Optional[float] = None,
             want_alpha: bool = False, dEdV: float = 0.0, stream=None) -> dict:
    """C^H, the smoothed volume fraction V and dE/d(positions, magnitudes,
    iso-level, thickness[, alpha]) for an objective with dE/dC^H = dEdC (6x6)
    and dE/dV = dEdV, through the smoothed density."""
    d = DesignArg(design, t)
    n = d.pos.shape[0]
    G = np.ascontiguousarray(np.asarray(dEdC, dtype=np.float64).reshape(36))
    C = np.zeros(36)
    g_pos = np.zeros((n, 3))
    g_q = np.zeros(n)
    g_iso, g_t, V = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    g_alpha = np.zeros((design.K + 1) ** 3) if want_alpha else None
    st = shl_stats()
    rc = lib().shl_grad(ctx, ctypes.byref(d.s), r, ctypes.byref(opts), G.ctypes.data_as(_dp), float(dEdV), _ptr(u),
                        C.ctypes.data_as(_dp), g_pos.ctypes.data_as(_dp), g_q.ctypes.data_as(_dp), ctypes.byref(g_iso),
                        ctypes.byref(g_t), g_alpha.ctypes.data_as(_dp) if want_alpha else None, ctypes.byref(V),
                        ctypes.byref(st), _stream(stream))
    _check(ctx, rc, ok=(SHL_OK, SHL_ENOCONV))
    return dict(C=C.reshape(6, 6), V=V.value, g_pos=g_pos, g_q=g_q, g_iso=g_iso.value, g_t=g_t.value,
                g_alpha=g_alpha, stats=st.as_dict())


def shl_serve_submit(ctx, design, r: int, opts: shl_solve_opts, session: int = -1) -> int:
    """Queue one design (copied at submit); returns its ticket."""
    d = DesignArg(design)
    req = shl_request(design=d.s, r=r, opts=opts, session=session)
    t = ctypes.c_uint64()
    _check(ctx, lib().shl_serve_submit(ctx, ctypes.byref(req), ctypes.byref(t)))
    return t.value


def shl_serve_poll(ctx, ticket: int) -> Optional[dict]:
    """Result dict when the request has completed, None while it is pending."""
    res = shl_result()
    st = lib().shl_serve_poll(ctx, ticket, ctypes.byref(res))
    if st == SHL_EAGAIN:
        return None
    _check(ctx, st)
    return res.as_dict()


def shl_serve_wait(ctx, ticket: int) -> dict:
    res = shl_result()
    _check(ctx, lib().shl_serve_wait(ctx, ticket, ctypes.byref(res)))
    return res.as_dict()


def shl_serve_cancel(ctx, ticket: int) -> bool:
    """True if the request was removed from the queue, False if it was already running."""
    st = lib().shl_serve_cancel(ctx, ticket)
    if st == SHL_EAGAIN:
        return False
    _check(ctx, st)
    return True


def shl_serve_drain(ctx) -> None:
    _check(ctx, lib().shl_serve_drain(ctx))


def shl_serve_info_get(ctx) -> dict:
    i = shl_serve_info()
    _check(ctx, lib().shl_serve_info_get(ctx, ctypes.byref(i)))
    return dict(slots=i.slots, queued=i.queued, running=i.running, completed=i.completed,
                held_bytes=i.held_bytes, budget_bytes=i.budget_bytes)


class shl_counters(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_uint64), ("workspace_bytes", ctypes.c_uint64)]


def shl_get_counters(ctx) -> dict:
    c = shl_counters()
    _check(ctx, lib().shl_get_counters(ctx, ctypes.byref(c)))
    return dict(kernel_launches=c.kernel_launches, workspace_bytes=c.workspace_bytes)


class Context:
    """Owns one shl_ctx (closed on exit or garbage collection)."""

    def __init__(self, device: int = 0, **kw):
        self.handle = shl_create(device, **kw)

    def close(self):
        if self.handle:
            shl_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class shl_peaks(ctypes.Structure):
    _fields_ = [("fp32_fma_gflops", ctypes.c_double), ("fp32x2_fma_gflops", ctypes.c_double),
                ("fp64_fma_gflops", ctypes.c_double)]


def shl_probe_peaks(ctx) -> dict:
    """Measured FP32, packed-FP32 and FP64 FMA throughput of the context's device (GFLOP/s)."""
    p = shl_peaks()
    _check(ctx, lib().shl_probe_peaks(ctx, ctypes.byref(p)))
    return dict(fp32_fma_gflops=p.fp32_fma_gflops, fp32x2_fma_gflops=p.fp32x2_fma_gflops,
                fp64_fma_gflops=p.fp64_fma_gflops)


def shl_probe_wait_timeout(ctx, polls: int = 4096) -> bool:
    """True when the probe's bounded device wait ended by its bound (the
    expected outcome: nothing completes the barrier it waits on)."""
    out = ctypes.c_int32(-1)
    _check(ctx, lib().shl_probe_wait_timeout(ctx, polls, ctypes.byref(out)))
    return out.value == 1

"""FP64 CPU oracle for the charge-shell homogenisation path (arXiv 2511.04025).

TEST INFRASTRUCTURE ONLY: the slow, plain reference that the CUDA library is
checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it.  It shares no code with the
CUDA path (``paper_2511_04025_b300``); the only module both use is the seeded
input generator ``paper_2511_04025_b300.inputs``, which holds none of the
method's arithmetic.

The heavy loops (field direct sum, assembled block-CSR stiffness, Jacobi-PCG,
energy sums) are plain C in ``shl_oracle.c`` (built by ``oracle.build``); the
rest is numpy written step by step from the paper:

  field        Sec. 3.1, Eq. charge-field, w_hkl from Eq. inf-series
  distance     Sec. 4.1, Eq. beta: d_e = |F(p_e)| / |grad F(p_e)|
  mask/beta    Sec. 4.1: logistic h(v) = 1/(1+exp(-kappa (t - v))); binary mask
  select_t     Sec. 4.3 (volume constraint through t); margin rule, see below
  assembly     Sec. 4.1, K_e = beta_e K_0 with ersatz floor E_void
  solve        Eq. inv-design constraint K u^(k) = f^(k), six load cases
  chom         Eq. inv-design: C^H_ij = sum_e (chi^i+u^i_e)^T K_e (chi^j+u^j_e)
  gradient     Eq. chain

Readings where the paper is silent:
  * iso-level c generalises the zero level set: solid iff |F-c| <= t |grad F|;
  * t from a volume fraction: the margin rule in ``select_t``;
  * kappa = ln(9) * r: h rises from 10 % to 90 % over two voxels.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "shl_oracle.c")
_SO = os.path.join(_HERE, "libshl_oracle.so")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the C oracle (plain -O2, no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        # built beside the target and renamed into place: a process that has the
        # old library loaded keeps its (unlinked) copy
        tmp = f"{_SO}.{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
                               "-shared", "-Wall", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        L.shlo_field.argtypes = [ctypes.c_int, _dp, _dp, _dp, ctypes.c_int, ctypes.c_long, _dp, _dp, _dp]
        L.shlo_field_param_derivs.argtypes = [ctypes.c_int, _dp, _dp, _dp, ctypes.c_int, _dp, _dp]
        L.shlo_element_stiffness.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp]
        L.shlo_test_displacement.argtypes = [ctypes.c_int, ctypes.c_double, _dp]
        L.shlo_apply.argtypes = [ctypes.c_int, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_int, _dp, _dp]
        L.shlo_rhs.argtypes = [ctypes.c_int, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp]
        L.shlo_solve.argtypes = [ctypes.c_int, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_int, _dp, _ip, _dp]
        L.shlo_solve_ex.argtypes = [ctypes.c_int, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_long, ctypes.c_double, ctypes.c_int, _dp, _ip, _dp]
        L.shlo_chom.argtypes = [ctypes.c_int, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                _dp, _dp, _dp]
        L.shlo_element_sensitivity.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                               _dp, _dp, _dp]
        L.shlo_field_vjp.argtypes = [ctypes.c_int, _dp, _dp, _dp, ctypes.c_int, ctypes.c_long, _dp, _dp, _dp, _dp,
                                     _dp, _dp]
        _lib = L
    return _lib


def _p(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def num_threads() -> int:
    return int(lib().shlo_num_threads())


# --------------------------------------------------------------------------- #
# Field and voxelisation (Sec. 3.1, Sec. 4.1)
# --------------------------------------------------------------------------- #

def voxel_centres(r: int) -> np.ndarray:
    """p_e = ((ix+1/2)/r, (iy+1/2)/r, (iz+1/2)/r), e = (iz*r + iy)*r + ix."""
    i = (np.arange(r) + 0.5) / r
    z, y, x = np.meshgrid(i, i, i, indexing="ij")
    return np.ascontiguousarray(np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1))


def field(design, pts: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """F and grad F of Eq. charge-field at arbitrary points (npts x 3)."""
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    pos = np.ascontiguousarray(design.pos, dtype=np.float64)
    q = np.ascontiguousarray(design.q, dtype=np.float64)
    alpha = None if design.alpha is None else np.ascontiguousarray(design.alpha, dtype=np.float64)
    if alpha is not None:
        assert alpha.size == (design.K + 1) ** 3
    F = np.empty(pts.shape[0])
    gF = np.empty((pts.shape[0], 3))
    st = lib().shlo_field(design.n, _p(pos), _p(q), _p(alpha), design.K, pts.shape[0], _p(pts), _p(F), _p(gF))
    assert st == 0, st
    return F, gF


def field_grid(design, r: int) -> Tuple[np.ndarray, np.ndarray]:
    return field(design, voxel_centres(r))


def field_param_derivs(design, pt: np.ndarray) -> np.ndarray:
    """Per charge j (rows): dF/dq_j, dF/dx_j (3), dgradF/dq_j (3), dgradF_i/dx_j,m (9)."""
    out = np.empty((design.n, 16))
    pt = np.ascontiguousarray(pt, dtype=np.float64)
    alpha = None if design.alpha is None else np.ascontiguousarray(design.alpha, dtype=np.float64)
    st = lib().shlo_field_param_derivs(design.n, _p(np.ascontiguousarray(design.pos, dtype=np.float64)),
                                       _p(np.ascontiguousarray(design.q, dtype=np.float64)), _p(alpha),
                                       design.K, _p(pt), _p(out))
    assert st == 0
    return out


def distance(F: np.ndarray, gF: np.ndarray, iso: float = 0.0) -> np.ndarray:
    """d_e = |F - c| / |grad F| (Eq. beta, iso-level c); +inf where grad F = 0."""
    g = np.sqrt(np.sum(gF * gF, axis=1))
    with np.errstate(divide="ignore", invalid="ignore"):
        d = np.abs(F - iso) / g
    d[g == 0.0] = np.inf
    return d


def mask(F: np.ndarray, gF: np.ndarray, iso: float, t: float) -> np.ndarray:
    """Binary shell: solid iff |F - c| <= t |grad F| (d <= t; ties solid)."""
    g = np.sqrt(np.sum(gF * gF, axis=1))
    return (np.abs(F - iso) <= t * g).astype(np.uint8)


def beta(d: np.ndarray, t: float, kappa: float) -> np.ndarray:
    """Smoothed Heaviside h(v) = 1 / (1 + exp(-kappa (t - v))) (Sec. 4.1)."""
    with np.errstate(over="ignore"):
        return 1.0 / (1.0 + np.exp(-kappa * (t - d)))


def default_kappa(r: int) -> float:
    """Transition of about two voxels: h goes 10 % -> 90 % over 2h => kappa = ln 9 / h."""
    return math.log(9.0) * r


GAP_REL = 1e-9


def select_t(d: np.ndarray, vf: float) -> Tuple[float, int, float]:
    """Half-thickness t for a target solid fraction (volume constraint of Sec. 4.3).

    Sort d ascending (d_(1) <= ... <= d_(n)); k0 = round(vf * n) clamped to
    [1, n-1].  Take the k nearest k0 (k0, k0-1, k0+1, k0-2, ...) whose gap is
    resolvable, d_(k+1) - d_(k) > 1e-9 d_(k+1), and return
    t = (d_(k) + d_(k+1)) / 2, the solid count k and the margin (d_(k+1)-d_(k))/2.
    Placing t mid-gap keeps every voxel at least the margin away from the
    threshold, so two independent FP64 evaluations give the same mask; the gap
    test steps over runs of equal distances (symmetric designs).
    """
    s = np.sort(np.asarray(d, dtype=np.float64))
    n = s.size
    assert n >= 2
    k0 = int(min(max(int(round(vf * n)), 1), n - 1))
    for j in range(0, n):
        for k in ((k0 - j, k0 + j) if j else (k0,)):
            if 1 <= k <= n - 1:
                lo, hi = s[k - 1], s[k]
                if np.isfinite(hi) and hi - lo > GAP_REL * hi:
                    return 0.5 * (lo + hi), k, 0.5 * (hi - lo)
    raise ValueError("no resolvable gap in the distance distribution")


def ambiguous_count(d: np.ndarray, t: float) -> int:
    """Voxels whose distance is within 1e-9 t of the threshold."""
    return int(np.sum(np.abs(d - t) <= 1e-9 * t))


# --------------------------------------------------------------------------- #
# FEM (Sec. 4.1, Eq. inv-design)
# --------------------------------------------------------------------------- #

def element_stiffness(E: float, nu: float, h: float) -> np.ndarray:
    K = np.empty((24, 24))
    assert lib().shlo_element_stiffness(E, nu, h, _p(K)) == 0
    return K


def test_displacement(k: int, h: float) -> np.ndarray:
    chi = np.empty(24)
    assert lib().shlo_test_displacement(k, h, _p(chi)) == 0
    return chi


def _rho(rho: np.ndarray, r: int) -> np.ndarray:
    rho = np.ascontiguousarray(rho, dtype=np.float64).ravel()
    assert rho.size == r ** 3
    return rho


def apply(r: int, rho: np.ndarray, x: np.ndarray, E=1.0, nu=0.3, Evoid=1e-6) -> np.ndarray:
    """y = K x with the assembled periodic stiffness; x is (nvec, r^3, 3)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    nvec = x.shape[0]
    y = np.empty_like(x)
    assert lib().shlo_apply(r, _p(_rho(rho, r)), E, nu, Evoid, nvec, _p(x), _p(y)) == 0
    return y


def rhs(r: int, rho: np.ndarray, E=1.0, nu=0.3, Evoid=1e-6) -> np.ndarray:
    """f^(k) = -sum_e K_e chi^k, shape (6, r^3, 3)."""
    f = np.empty((6, r ** 3, 3))
    assert lib().shlo_rhs(r, _p(_rho(rho, r)), E, nu, Evoid, _p(f)) == 0
    return f


def solve(r: int, rho: np.ndarray, E=1.0, nu=0.3, Evoid=1e-6, tol=1e-12, maxit=200000):
    """Six periodic cell problems, node 0 pinned, Jacobi-PCG in FP64.

    Returns (u (6, r^3, 3), iters (6,), relres (6,), status)."""
    u = np.empty((6, r ** 3, 3))
    iters = np.zeros(6, dtype=np.int32)
    relres = np.zeros(6)
    st = lib().shlo_solve(r, _p(_rho(rho, r)), E, nu, Evoid, tol, maxit, _p(u),
                          iters.ctypes.data_as(_ip), _p(relres))
    return u, iters, relres, st


# --------------------------------------------------------------------------- #
# Active set (Sec. 4.2.1): culled void, no ersatz floor
# --------------------------------------------------------------------------- #

CULL_THRESHOLD = 1e-3  # an element is active when beta_e (or the mask) exceeds it


def cull(rho: np.ndarray, theta: float = CULL_THRESHOLD) -> np.ndarray:
    """Element densities of the active set: rho_e where rho_e > theta, else 0
    (a culled element contributes no stiffness)."""
    rho = np.asarray(rho, dtype=np.float64)
    return np.where(rho > theta, rho, 0.0)


def active_nodes(r: int, rho_culled: np.ndarray) -> np.ndarray:
    """Nodes with at least one active incident element (the DOFs the culled
    problem keeps)."""
    act = (np.asarray(rho_culled).reshape(r, r, r) > 0.0)  # [iz, iy, ix]
    out = np.zeros_like(act)
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                out |= np.roll(act, shift=(dz, dy, dx), axis=(0, 1, 2))
    return out.ravel()


def solve_active(r: int, rho: np.ndarray, E=1.0, nu=0.3, theta=CULL_THRESHOLD, tol=1e-12, maxit=200000):
    """The cell problems on the active set of Sec. 4.2.1: elements with
    rho_e <= theta are culled (zero stiffness, no ersatz floor), active ones
    have E_e = rho_e E; nodes without an active element are removed (u = 0
    there) and the first active node is pinned.  Jacobi-PCG in FP64.
    Returns (u, iters, relres, status, rho_culled, pin)."""
    rc = cull(_rho(rho, r), theta)
    nodes = np.flatnonzero(active_nodes(r, rc))
    if nodes.size == 0:
        raise ValueError("no active element")
    pin = int(nodes[0])
    u = np.empty((6, r ** 3, 3))
    iters = np.zeros(6, dtype=np.int32)
    relres = np.zeros(6)
    st = lib().shlo_solve_ex(r, _p(np.ascontiguousarray(rc)), E, nu, 0.0, pin, tol, maxit, _p(u),
                             iters.ctypes.data_as(_ip), _p(relres))
    return u, iters, relres, st, rc, pin


def homogenize_active(design, r: int, t: Optional[float] = None, E=1.0, nu=0.3, theta=CULL_THRESHOLD, tol=1e-12,
                      maxit=200000):
    """Field -> mask -> C^H on the active set (the solid voxels; no ersatz void)."""
    vox = voxelize(design, r, t)
    u, iters, relres, st, rc, pin = solve_active(r, vox["mask"].astype(np.float64), E, nu, theta, tol, maxit)
    C, Calt = chom(r, rc, u, E, nu, 0.0)
    vox.update(C=C, Calt=Calt, u=u, iters=iters, relres=relres, status=st, rho=rc, pin=pin)
    return vox


def chom(r: int, rho: np.ndarray, u: np.ndarray, E=1.0, nu=0.3, Evoid=1e-6):
    """C^H (energy form) and the equivalent chi^T K (chi + u) form."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    C = np.empty(36)
    Calt = np.empty(36)
    assert lib().shlo_chom(r, _p(_rho(rho, r)), E, nu, Evoid, _p(u), _p(C), _p(Calt)) == 0
    return C.reshape(6, 6), Calt.reshape(6, 6)


def element_sensitivity(r: int, u: np.ndarray, G: np.ndarray, E=1.0, nu=0.3, Evoid=1e-6) -> np.ndarray:
    """g_e = dE/drho_e = sum_ij G_ij (E-E_void) (chi^i+u^i_e)^T Khat (chi^j+u^j_e)."""
    g = np.empty(r ** 3)
    G = np.ascontiguousarray(G, dtype=np.float64).ravel()
    assert lib().shlo_element_sensitivity(r, E, nu, Evoid, _p(np.ascontiguousarray(u)), _p(G), _p(g)) == 0
    return g


def field_vjp(design, pts: np.ndarray, Fbar: np.ndarray, gFbar: np.ndarray, want_alpha: bool = False):
    """sum_p Fbar dF/dtheta + gFbar . d(grad F)/dtheta for theta = charge positions
    (n x 3), magnitudes (n) and, with want_alpha, the mode weights alpha_hkl
    ((K+1)^3, indexed [h][k][l]; Sec. 4.3) (chain rule through Eq. charge-field)."""
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    g_pos = np.zeros((design.n, 3))
    g_q = np.zeros(design.n)
    g_alpha = np.zeros((design.K + 1) ** 3) if want_alpha else None
    alpha = None if design.alpha is None else np.ascontiguousarray(design.alpha, dtype=np.float64)
    st = lib().shlo_field_vjp(design.n, _p(np.ascontiguousarray(design.pos, dtype=np.float64)),
                              _p(np.ascontiguousarray(design.q, dtype=np.float64)), _p(alpha), design.K,
                              pts.shape[0], _p(pts), _p(np.ascontiguousarray(Fbar, dtype=np.float64)),
                              _p(np.ascontiguousarray(gFbar, dtype=np.float64)), _p(g_pos), _p(g_q), _p(g_alpha))
    assert st == 0
    if want_alpha:
        return g_pos, g_q, g_alpha
    return g_pos, g_q


def gradient(design, r: int, dEdC: np.ndarray, t: float, kappa: Optional[float] = None, E=1.0, nu=0.3,
             Evoid=1e-6, tol=1e-12, maxit=200000):
    """dE/dtheta through the smoothed density (Eq. chain), theta = charge
    positions, magnitudes, mode weights alpha_hkl (Sec. 4.3), iso-level c and
    half-thickness t, for an objective
    with dE/dC^H = dEdC (6x6):
      g_e        = dE/drho_e = sum_ij dEdC_ij (E - E_void) w_i^T Khat w_j  (self-adjoint cell problems)
      dbeta/dd   = -kappa beta (1 - beta),   dbeta/dt = +kappa beta (1 - beta)
      d          = |F - c| / |grad F|:  dd/dF = sgn(F - c)/|grad F|, dd/dc = -dd/dF,
                   dd/d(grad F) = -|F - c| grad F / |grad F|^3
    then back through F and grad F to the charges."""
    F, gF = field_grid(design, r)
    kap = default_kappa(r) if kappa is None else kappa
    d = distance(F, gF, design.iso)
    rho = beta(d, t, kap)
    u, iters, relres, st = solve(r, rho, E, nu, Evoid, tol, maxit)
    C, _ = chom(r, rho, u, E, nu, Evoid)
    out = gradient_backward(design, r, dEdC, t, kap, F, gF, rho, u, E, nu, Evoid)
    out.update(C=C, u=u, rho=rho, iters=iters, relres=relres, status=st)
    return out


def gradient_backward(design, r: int, dEdC: np.ndarray, t: float, kap: float, F: np.ndarray, gF: np.ndarray,
                      rho: np.ndarray, u: np.ndarray, E=1.0, nu=0.3, Evoid=1e-6):
    """The backward half of ``gradient`` for given cell-problem solutions u of
    the smoothed density rho = beta(d, t, kap) (Eq. chain, steps as listed there)."""
    g_e = element_sensitivity(r, u, dEdC, E, nu, Evoid)
    db = kap * rho * (1.0 - rho)            # dbeta/dt = -dbeta/dd
    dE_dd = -g_e * db
    gn = np.sqrt(np.sum(gF * gF, axis=1))
    ok = gn > 0
    Fbar = np.zeros_like(F)
    gFbar = np.zeros_like(gF)
    Fbar[ok] = dE_dd[ok] * np.sign(F[ok] - design.iso) / gn[ok]
    gFbar[ok] = (dE_dd[ok] * (-np.abs(F[ok] - design.iso) / gn[ok] ** 3))[:, None] * gF[ok]
    g_pos, g_q, g_alpha = field_vjp(design, voxel_centres(r), Fbar, gFbar, want_alpha=True)
    return dict(g_pos=g_pos, g_q=g_q, g_alpha=g_alpha, g_iso=float(-Fbar.sum()), g_t=float(np.sum(g_e * db)),
                g_e=g_e)


def isotropic_C(E=1.0, nu=0.3) -> np.ndarray:
    """Base material tensor C_0 (Voigt, engineering shear)."""
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    for i in range(3):
        C[i, i] = lam + 2 * mu
        C[3 + i, 3 + i] = mu
    return C


# --------------------------------------------------------------------------- #
# Whole pipeline
# --------------------------------------------------------------------------- #

def voxelize(design, r: int, t: Optional[float] = None):
    """Field -> distance -> t (explicit or from design.vf) -> binary mask."""
    F, gF = field_grid(design, r)
    d = distance(F, gF, design.iso)
    margin = None
    if t is None:
        t = design.t
    if t is None:
        t, _, margin = select_t(d, design.vf)
    m = mask(F, gF, design.iso, t)
    return dict(F=F, gF=gF, d=d, t=t, margin=margin, mask=m, ambiguous=ambiguous_count(d, t))


def homogenize(design, r: int, t: Optional[float] = None, E=1.0, nu=0.3, Evoid=1e-6, tol=1e-12, maxit=200000):
    vox = voxelize(design, r, t)
    rho = vox["mask"].astype(np.float64)
    u, iters, relres, st = solve(r, rho, E, nu, Evoid, tol, maxit)
    C, Calt = chom(r, rho, u, E, nu, Evoid)
    vox.update(C=C, Calt=Calt, u=u, iters=iters, relres=relres, status=st, rho=rho)
    return vox


def aos_to_soa(v: np.ndarray) -> np.ndarray:
    """(6, N, 3) -> (18, N) with plane k*3+i, the CUDA library's node-vector layout."""
    return np.ascontiguousarray(np.transpose(v, (0, 2, 1)).reshape(v.shape[0] * 3, v.shape[1]))


def soa_to_aos(v: np.ndarray) -> np.ndarray:
    nv = v.shape[0] // 3
    return np.ascontiguousarray(np.transpose(v.reshape(nv, 3, -1), (0, 2, 1)))

"""The active-set solve (Sec. 4.2.1: void culled, no ersatz floor; solve
option active = 1) against the oracle's active-set problem, through the C-ABI.

Tolerances as for the ersatz problem: C^H entry error (relative to
max(|C_ij|, 1e-2 max|C|)) <= 1e-9 at tol 1e-10 in both precision modes.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2511_04025_b300 import inputs, shl  # noqa: E402

GOLD = os.path.join(os.path.dirname(__file__), "golden")
DEV = "cuda:0"


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device: GPU tests need a B300")
    c = shl.Context(0)
    yield c.handle
    c.close()


def entry_err(C, Cref):
    s = np.abs(Cref).max()
    return np.max(np.abs(C - Cref) / np.maximum(np.abs(Cref), 1e-2 * s))


def gold(name):
    with open(os.path.join(GOLD, name + ".json")) as f:
        g = json.load(f)
    g["C"] = np.array(g["C"])
    return g


@pytest.mark.parametrize("prec", [shl.SHL_FP64, shl.SHL_FP32_REFINE])
def test_active_set_matches_oracle_32(ctx, prec):
    g = gold("plain32_s0_active")
    C, st = shl.shl_homogenize(ctx, inputs.plain_32(0), 32, shl.default_solve_opts(tol=1e-10, precision=prec,
                                                                                      active=1))
    assert st["status"] == 0 and st["n_solid"] == g["n_solid"]
    assert max(st["relres"]) <= 1e-10
    assert entry_err(C, g["C"]) <= 1e-9


@pytest.mark.parametrize("tol,bound", [(1e-10, 1e-9), (1e-7, 1e-5)])
def test_active_set_matches_oracle_64(ctx, tol, bound):
    g = gold("gaussian64_s0_active")
    C, st = shl.shl_homogenize(ctx, inputs.gaussian_64(0), 64,
                               shl.default_solve_opts(tol=tol, precision=shl.SHL_FP32_REFINE, active=1))
    assert st["status"] == 0 and max(st["relres"]) <= tol
    assert entry_err(C, g["C"]) <= bound


def test_active_set_smoothed_density_matches_oracle(ctx):
    """Smoothed densities with a share below the threshold, through shl_solve:
    culled elements carry no stiffness, active ones rho_e E."""
    r = 12
    rng = np.random.default_rng(4)
    rho = rng.uniform(0.0, 1.0, r ** 3) ** 3
    rho[rng.uniform(size=r ** 3) < 0.4] = 5e-4
    u, it, rr, st_o, rc, pin = oracle.solve_active(r, rho, tol=1e-13)
    Cref, _ = oracle.chom(r, rc, u, Evoid=0.0)
    o = shl.default_solve_opts(tol=1e-11, precision=shl.SHL_FP64, density=shl.SHL_SMOOTH, active=1)
    C, st = shl.shl_solve(ctx, r, o, rho=torch.tensor(rho, device=DEV))
    assert st["status"] == 0
    assert entry_err(C, Cref) <= 1e-9


def test_active_set_needs_fewer_iterations(ctx):
    """On the 64^3 throughput design the active set converges in fewer
    iterations than the ersatz problem at the same tolerance (the void's
    O(E_void) residual no longer has to be resolved)."""
    d = inputs.gaussian_64(0)
    o = dict(tol=1e-7, precision=shl.SHL_FP32_REFINE)
    _, se = shl.shl_homogenize(ctx, d, 64, shl.default_solve_opts(**o))
    _, sa = shl.shl_homogenize(ctx, d, 64, shl.default_solve_opts(active=1, **o))
    assert se["status"] == 0 and sa["status"] == 0
    assert max(sa["iters"]) < max(se["iters"])


def test_active_set_not_in_the_adjoint(ctx):
    d = inputs.random_design(5, 8, 0.12)
    o = shl.default_solve_opts(density=shl.SHL_SMOOTH, active=1)
    with pytest.raises(shl.ShlError) as e:
        shl.shl_grad(ctx, d, 16, o, np.zeros((6, 6)), t=0.02)
    assert e.value.status == shl.SHL_EINVAL


def _slab_mask(r, seed):
    """Solid in a slab of three z planes (half of its voxels) plus 1 % scattered
    voxels: some warps of elements are wholly culled, some mixed, some solid."""
    rng = np.random.default_rng(seed)
    m = np.zeros((r, r, r), np.uint8)  # [z][y][x]
    m[r // 3:r // 3 + 3] = rng.uniform(size=(3, r, r)) < 0.5
    m |= (rng.uniform(size=(r, r, r)) < 0.01).astype(np.uint8)
    return m.reshape(-1)


@pytest.mark.parametrize("r,dtype", [(20, "f64"), (20, "f32"), (32, "f32"), (48, "f32"), (64, "f32")])
def test_apply_culled_void_matches_oracle(ctx, r, dtype):
    """The stiffness apply with the void culled (E_void = 0, Sec. 4.2.1) -- tile
    kernel at r = 20, row kernel at 32, 48, 64 -- against the oracle's
    assembled operator of the culled problem."""
    m = _slab_mask(r, 60 + r)
    x = np.random.default_rng(70 + r).standard_normal((6, r ** 3, 3))
    y = oracle.apply(r, m.astype(np.float64), x, Evoid=0.0)
    td = torch.float64 if dtype == "f64" else torch.float32
    p = torch.tensor(oracle.aos_to_soa(x), dtype=td, device=DEV)
    q = torch.full_like(p, float("nan"))
    shl.shl_apply(ctx, r, p, q, mask=torch.tensor(m, device=DEV), E_void=0.0)
    torch.cuda.synchronize()
    yq = oracle.soa_to_aos(q.double().cpu().numpy())
    tol = 1e-12 if dtype == "f64" else 2e-6
    assert np.isfinite(yq).all()
    assert np.abs(yq - y).max() <= tol * np.abs(y).max()


def test_chom_culled_void_matches_oracle(ctx):
    """C^H with the void culled (culled elements add nothing) against the
    oracle's energy sum on the same displacements."""
    r = 16
    m = _slab_mask(r, 81)
    u = np.random.default_rng(82).standard_normal((6, r ** 3, 3)) * 0.02
    ref, _ = oracle.chom(r, m.astype(np.float64), u, Evoid=0.0)
    C = shl.shl_chom(ctx, r, torch.tensor(oracle.aos_to_soa(u), device=DEV),
                     mask=torch.tensor(m, device=DEV), E_void=0.0)
    assert np.abs(C - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("r", [64, 128])
def test_thin_shell_active_set_multigrid_matches_fp64(ctx, r):
    """The timing table's thin shell (t = 0.02) with the active set: the FP32 +
    refinement solve, whose multigrid skips inactive nodes on every level,
    against the FP64 point-Jacobi solve of the same culled problem (no
    multigrid), both to a relative residual of 1e-10."""
    d = inputs.shell_256(0)
    o32 = shl.default_solve_opts(tol=1e-10, precision=shl.SHL_FP32_REFINE, active=1)
    o64 = shl.default_solve_opts(tol=1e-10, precision=shl.SHL_FP64, active=1, max_iter=100000,
                                 precond=shl.SHL_PRECOND_JACOBI)
    C32, s32 = shl.shl_homogenize(ctx, d, r, o32)
    C64, s64 = shl.shl_homogenize(ctx, d, r, o64)
    assert s32["status"] == 0 and s64["status"] == 0 and s32["precond"] == shl.SHL_PRECOND_MG
    assert s64["precond"] == shl.SHL_PRECOND_JACOBI
    assert entry_err(C32, C64) <= 1e-9

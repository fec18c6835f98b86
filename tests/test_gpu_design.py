"""Inverse-design driver on the GPU: the volume term of the adjoint against
central differences of the oracle's smoothed volume fraction, and the
alternating driver (thickness, Adam on alpha, CMA-ES on positions through the
serving path) on a small grid."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2511_04025_b300 import inputs, objectives, shl  # noqa: E402
from paper_2511_04025_b300.design import InverseDesign  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device: GPU tests need a B300")
    c = shl.Context(0, max_batch=8)
    yield c.handle
    c.close()


def _smooth(prec=shl.SHL_FP64, tol=1e-12, **kw):
    return shl.default_solve_opts(precision=prec, tol=tol, density=shl.SHL_SMOOTH, **kw)


def _design16():
    d = inputs.random_design(21, 6, 0.12)
    d.alpha = 1.0 + 0.3 * np.random.default_rng(2).standard_normal((d.K + 1) ** 3)
    d.iso = 0.002
    return d


def _oracle_volume(d, r, t):
    F, gF = oracle.field_grid(d, r)
    return float(np.mean(oracle.beta(oracle.distance(F, gF, d.iso), t, oracle.default_kappa(r))))


def test_volume_term_matches_oracle_differences(ctx):
    """With dE/dC = 0 and dE/dV = 1 the adjoint returns dV/dtheta, V the mean
    smoothed occupancy; compare with central differences (h = 1e-6) of the
    oracle's V for the thickness, iso-level, positions, magnitudes and alpha."""
    r = 16
    d = _design16()
    t = oracle.voxelize(d, r)["t"]
    out = shl.shl_grad(ctx, d, r, _smooth(), np.zeros((6, 6)), t=t, want_alpha=True, dEdV=1.0)
    V0 = _oracle_volume(d, r, t)
    assert abs(out["V"] - V0) <= 1e-12
    h = 1e-6
    fd = {}
    fd["t"] = (_oracle_volume(d, r, t + h) - _oracle_volume(d, r, t - h)) / (2 * h)
    dp, dm = d.copy(iso=d.iso + h), d.copy(iso=d.iso - h)
    fd["iso"] = (_oracle_volume(dp, r, t) - _oracle_volume(dm, r, t)) / (2 * h)
    for j, m in ((0, 0), (3, 2), (5, 1)):
        dp, dm = d.copy(), d.copy()
        dp.pos[j, m] += h
        dm.pos[j, m] -= h
        fd[("pos", j, m)] = (_oracle_volume(dp, r, t) - _oracle_volume(dm, r, t)) / (2 * h)
    for j in (1, 4):
        dp, dm = d.copy(), d.copy()
        dp.q[j] += h
        dm.q[j] -= h
        fd[("q", j)] = (_oracle_volume(dp, r, t) - _oracle_volume(dm, r, t)) / (2 * h)
    for a in (0, 7, 26):
        dp, dm = d.copy(), d.copy()
        dp.alpha[a] += h
        dm.alpha[a] -= h
        fd[("alpha", a)] = (_oracle_volume(dp, r, t) - _oracle_volume(dm, r, t)) / (2 * h)
    got = {"t": out["g_t"], "iso": out["g_iso"]}
    for k in fd:
        if isinstance(k, tuple) and k[0] == "pos":
            got[k] = out["g_pos"][k[1], k[2]]
        elif isinstance(k, tuple) and k[0] == "q":
            got[k] = out["g_q"][k[1]]
        elif isinstance(k, tuple):
            got[k] = out["g_alpha"][k[1]]
    scale = max(abs(v) for v in fd.values())
    for k in fd:
        assert abs(got[k] - fd[k]) <= 2e-6 * scale, (k, got[k], fd[k])


def test_volume_term_is_additive(ctx):
    """grad(G, c) = grad(G, 0) + c grad(0, 1): the volume term adds a constant
    to every element sensitivity and nothing else."""
    r = 16
    d = _design16()
    t = oracle.voxelize(d, r)["t"]
    G = np.arange(36, dtype=np.float64).reshape(6, 6) / 36.0
    o = _smooth()
    a = shl.shl_grad(ctx, d, r, o, G, t=t, want_alpha=True)
    b = shl.shl_grad(ctx, d, r, o, np.zeros((6, 6)), t=t, want_alpha=True, dEdV=1.0)
    c = shl.shl_grad(ctx, d, r, o, G, t=t, want_alpha=True, dEdV=-2.5)
    for k in ("g_pos", "g_q", "g_alpha"):
        ref = a[k] - 2.5 * b[k]
        assert np.abs(c[k] - ref).max() <= 1e-9 * np.abs(ref).max(), k
    for k in ("g_t", "g_iso"):
        ref = a[k] - 2.5 * b[k]
        assert abs(c[k] - ref) <= 1e-9 * abs(ref), k
    assert a["V"] == b["V"] == c["V"]


def test_alpha_gradient_is_a_descent_direction_for_specific_modulus(ctx):
    """E = -K_eff / V at fixed t, V the smoothed volume: a step of length eps
    along -dE/dalpha lowers E by eps |g|^2 to first order."""
    r = 24
    d = inputs.random_design(5, 8, 0.12)
    d.alpha = np.ones((d.K + 1) ** 3)
    t = oracle.voxelize(d, r)["t"]
    fn = objectives.objective("Keff")
    o = _smooth()
    f0 = shl.shl_grad(ctx, d, r, o, np.zeros((6, 6)), t=t)
    e0, G, gV = objectives.value_and_grad(fn, f0["C"], f0["V"])
    g = shl.shl_grad(ctx, d, r, o, G, t=t, want_alpha=True, dEdV=gV)["g_alpha"]
    eps = 1e-3 * abs(e0) / float(g @ g)
    f1 = shl.shl_grad(ctx, d.copy(alpha=d.alpha - eps * g), r, o, np.zeros((6, 6)), t=t)
    e1 = objectives.value_and_grad(fn, f1["C"], f1["V"])[0]
    pred = eps * float(g @ g)
    assert e1 < e0
    assert abs((e0 - e1) - pred) <= 0.05 * pred, (e0 - e1, pred)


def test_inverse_design_driver_small(ctx):
    r, vf = 24, 0.12
    d = inputs.random_design(5, 8, vf)
    drv = InverseDesign(ctx, d, r, "Keff", vf, popsize=8, seed=0, lr_alpha=0.05)
    # the serving evaluation agrees with a direct homogenisation at the target volume
    o = shl.default_solve_opts(precision=shl.SHL_FP32_REFINE, tol=1e-7, density=shl.SHL_SMOOTH)
    C, st = shl.shl_homogenize(ctx, drv.design, r, o)
    direct = -objectives.bulk_hill(torch.tensor(C)) / vf
    assert abs(drv.value - float(direct)) <= 1e-5 * abs(float(direct))
    # stage (i): the thickness meets the volume fraction on the voxel count
    vox = shl.shl_voxelize(ctx, drv.design.copy(t=drv.thickness()), r)
    assert abs(vox["n_solid"] - vf * r ** 3) <= 1.0
    hist = drv.run(outer=1, n_alpha=2, n_gen=2)
    assert hist.stage == ["alpha", "positions"]
    assert np.all(np.isfinite(hist.objective))
    assert hist.objective[1] <= hist.objective[0]  # the incumbent never worsens in stage (iii)
    assert hist.evaluations == 1 + 1 + 2 * 8
    assert np.all((drv.design.pos >= 0.0) & (drv.design.pos < 1.0))
    assert np.all(drv.design.alpha >= 0.0)
    # the incumbent's value is reproducible through the direct path
    C, _ = shl.shl_homogenize(ctx, drv.design, r, o)
    assert abs(drv.value - float(-objectives.bulk_hill(torch.tensor(C)) / vf)) <= 1e-5 * abs(drv.value)

"""The GPU adjoint (shl_grad) against the oracle's adjoint, against central
finite differences of the GPU's own C^H, and through torch.autograd."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2511_04025_b300 import inputs, shl  # noqa: E402
from paper_2511_04025_b300.autograd import HomogenizeFn  # noqa: E402


GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device: GPU tests need a B300")
    c = shl.Context(0)
    yield c.handle
    c.close()


def _smooth(prec=shl.SHL_FP64, tol=1e-12, **kw):
    return shl.default_solve_opts(precision=prec, tol=tol, density=shl.SHL_SMOOTH, **kw)


def test_grad_matches_oracle_gradient(ctx):
    r = 16
    d = inputs.random_design(21, 6, 0.12)
    d.iso = 0.003
    t = oracle.voxelize(d, r)["t"]
    Ct = inputs.isotropic_target()
    ref0 = oracle.gradient(d, r, np.zeros((6, 6)), t, tol=1e-13)
    G = 2.0 * (ref0["C"] - Ct)
    ref = oracle.gradient(d, r, G, t, tol=1e-13)
    out = shl.shl_grad(ctx, d, r, _smooth(), G, t=t, want_alpha=True)
    s = np.abs(ref["C"]).max()
    assert np.max(np.abs(out["C"] - ref["C"])) <= 1e-9 * s
    scale = max(np.abs(ref["g_pos"]).max(), np.abs(ref["g_q"]).max(), abs(ref["g_iso"]), abs(ref["g_t"]))
    for k in ("g_pos", "g_q"):
        assert np.abs(out[k] - ref[k]).max() <= 1e-7 * scale, k
    # mode weights alpha_hkl (Sec. 4.3), every entry
    assert np.abs(out["g_alpha"] - ref["g_alpha"]).max() <= 1e-7 * np.abs(ref["g_alpha"]).max()
    assert abs(out["g_iso"] - ref["g_iso"]) <= 1e-7 * scale
    assert abs(out["g_t"] - ref["g_t"]) <= 1e-7 * scale


@pytest.mark.parametrize("prec,tol,bound", [(shl.SHL_FP64, 1e-12, 1e-7), (shl.SHL_FP32_REFINE, 1e-10, 1e-6)])
def test_grad_64_matches_oracle_golden(ctx, prec, tol, bound):
    """The inverse-design gradient at full size (64^3, 24 charges +-1, 10 %
    solid, smoothed density): GPU adjoint against the oracle's (solved to
    1e-12) for dE/dC^H = 2 (C^H - C^T) stored with the oracle's values, every
    parameter: positions, magnitudes, alpha, iso-level, thickness."""
    with open(os.path.join(GOLD, "gradient64_s0.json")) as f:
        g = json.load(f)
    d = inputs.gradient_64(0)
    out = shl.shl_grad(ctx, d, 64, _smooth(prec=prec, tol=tol), np.array(g["dEdC"]), t=g["t"], want_alpha=True)
    C = np.array(g["C"])
    assert np.abs(out["C"] - C).max() <= 1e-9 * np.abs(C).max()
    scale = max(np.abs(g["g_pos"]).max(), np.abs(g["g_q"]).max(), abs(g["g_iso"]), abs(g["g_t"]))
    assert np.abs(out["g_pos"] - np.array(g["g_pos"])).max() <= bound * scale
    assert np.abs(out["g_q"] - np.array(g["g_q"])).max() <= bound * scale
    assert abs(out["g_iso"] - g["g_iso"]) <= bound * scale
    assert abs(out["g_t"] - g["g_t"]) <= bound * scale
    ga = np.array(g["g_alpha"])
    assert np.abs(out["g_alpha"] - ga).max() <= bound * np.abs(ga).max()


def test_grad_matches_central_differences_32(ctx):
    """Objective E = sum (C^H - C^T)^2 with C^T isotropic (bulk 0.05, shear
    0.02); adjoint vs central differences (h = 1e-4) of the GPU forward."""
    r = 32
    d = inputs.gradient_64(0)
    vox = oracle.voxelize(d, r)
    t = vox["t"]
    Ct = inputs.isotropic_target()
    o = _smooth()
    C0, _ = shl.shl_homogenize(ctx, d.copy(t=t), r, o)
    out = shl.shl_grad(ctx, d, r, o, 2.0 * (C0 - Ct), t=t, want_alpha=True)
    E = lambda dd, tt: float(np.sum((shl.shl_homogenize(ctx, dd.copy(t=tt), r, o)[0] - Ct) ** 2))
    h = 1e-4
    checks = []
    for j, m in ((0, 0), (5, 1), (11, 2), (17, 0)):
        dp, dm = d.copy(), d.copy()
        dp.pos[j, m] += h
        dm.pos[j, m] -= h
        checks.append(((E(dp, t) - E(dm, t)) / (2 * h), out["g_pos"][j, m]))
    for j in (2, 13):
        dp, dm = d.copy(), d.copy()
        dp.q[j] += h
        dm.q[j] -= h
        checks.append(((E(dp, t) - E(dm, t)) / (2 * h), out["g_q"][j]))
    dp, dm = d.copy(iso=d.iso + h), d.copy(iso=d.iso - h)
    checks.append(((E(dp, t) - E(dm, t)) / (2 * h), out["g_iso"]))
    checks.append(((E(d, t + h) - E(d, t - h)) / (2 * h), out["g_t"]))
    a0 = np.ones(64)
    for idx in (1 * 16 + 2 * 4 + 0, 3 * 16 + 3 * 4 + 3):
        ap, am = a0.copy(), a0.copy()
        ap[idx] += h
        am[idx] -= h
        checks.append(((E(d.copy(alpha=ap), t) - E(d.copy(alpha=am), t)) / (2 * h), out["g_alpha"][idx]))
    scale = max(abs(f) for f, _ in checks)
    for f, a in checks:
        assert abs(f - a) <= 1e-4 * scale + 1e-3 * abs(f), (f, a)


def test_autograd_function_matches_shl_grad(ctx):
    r = 16
    d = inputs.random_design(5, 8, 0.12)
    t = oracle.voxelize(d, r)["t"]
    pos = torch.tensor(d.pos, requires_grad=True)
    q = torch.tensor(d.q, requires_grad=True)
    iso = torch.tensor(0.0, dtype=torch.float64, requires_grad=True)
    tt = torch.tensor(t, dtype=torch.float64, requires_grad=True)
    Ct = torch.tensor(inputs.isotropic_target())
    C = HomogenizeFn.apply(pos, q, iso, tt, ctx, r, 3, None, _smooth())
    loss = ((C - Ct) ** 2).sum()
    loss.backward()
    ref = shl.shl_grad(ctx, d, r, _smooth(), 2.0 * (C.detach().numpy() - Ct.numpy()), t=t)
    np.testing.assert_allclose(pos.grad.numpy(), ref["g_pos"], rtol=1e-6, atol=1e-9 * np.abs(ref["g_pos"]).max())
    np.testing.assert_allclose(q.grad.numpy(), ref["g_q"], rtol=1e-6, atol=1e-9 * np.abs(ref["g_q"]).max())
    assert abs(float(tt.grad) - ref["g_t"]) <= 1e-6 * abs(ref["g_t"])

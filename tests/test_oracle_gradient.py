"""Pins of the oracle's adjoint (Eq. chain) against central finite differences
of the oracle's own forward map (independent of the adjoint formulas)."""
import numpy as np
import pytest

import oracle
from paper_2511_04025_b300 import inputs

R = 10


def objective(C, Ct):
    return float(np.sum((C - Ct) ** 2))


def forward_C(design, r, t, kap, rho_override=None):
    F, gF = oracle.field_grid(design, r)
    rho = oracle.beta(oracle.distance(F, gF, design.iso), t, kap) if rho_override is None else rho_override
    u, *_ = oracle.solve(r, rho, tol=1e-13)
    return oracle.chom(r, rho, u)[0]


def test_element_sensitivity_matches_finite_differences():
    """dC^H_ij/drho_e = (E - E_void) w_i^T Khat w_j (no adjoint solve: the cell
    problems are self-adjoint); checked for a few elements against central
    differences of the full solve."""
    rng = np.random.default_rng(3)
    rho = rng.uniform(0.2, 1.0, size=R ** 3)
    u, *_ = oracle.solve(R, rho, tol=1e-13)
    G = rng.standard_normal((6, 6))
    g = oracle.element_sensitivity(R, u, G)
    hs = 1e-5
    for e in (0, 37, 511, R ** 3 - 1):
        rp, rm = rho.copy(), rho.copy()
        rp[e] += hs
        rm[e] -= hs
        up, *_ = oracle.solve(R, rp, tol=1e-13)
        um, *_ = oracle.solve(R, rm, tol=1e-13)
        fd = np.sum(G * (oracle.chom(R, rp, up)[0] - oracle.chom(R, rm, um)[0])) / (2 * hs)
        # FD noise: solve error (~1e-13) / h dominates for the smallest sensitivities
        assert abs(fd - g[e]) <= 2e-5 * max(abs(fd), 1e-2 * np.abs(g).max())


def test_adjoint_gradient_matches_finite_differences():
    d = inputs.random_design(21, 6, 0.12)
    d.iso = 0.003
    Ct = inputs.isotropic_target()
    kap = oracle.default_kappa(R)
    t = oracle.voxelize(d, R)["t"]
    C0 = forward_C(d, R, t, kap)
    res = oracle.gradient(d, R, 2.0 * (C0 - Ct), t, kappa=kap, tol=1e-13)
    np.testing.assert_allclose(res["C"], C0, rtol=0, atol=1e-13)
    h = 1e-4

    def fd(mutate):
        dp, dm = d.copy(), d.copy()
        tp = mutate(dp, +h)
        tm = mutate(dm, -h)
        return (objective(forward_C(dp, R, tp, kap), Ct) - objective(forward_C(dm, R, tm, kap), Ct)) / (2 * h)

    checks = []
    for j in (0, 3):
        for m in range(3):
            def mut(x, s, j=j, m=m):
                x.pos[j, m] += s
                return t
            checks.append((fd(mut), res["g_pos"][j, m]))

        def mutq(x, s, j=j):
            x.q[j] += s
            return t
        checks.append((fd(mutq), res["g_q"][j]))

    def muti(x, s):
        x.iso += s
        return t
    checks.append((fd(muti), res["g_iso"]))
    checks.append((fd(lambda x, s: t + s), res["g_t"]))
    # mode weights alpha_hkl (Sec. 4.3), indexed [h][k][l]
    for idx in (1 * 16 + 0 * 4 + 0, 1 * 16 + 2 * 4 + 0, 3 * 16 + 3 * 4 + 3, 0 * 16 + 2 * 4 + 1):
        def muta(x, s, idx=idx):
            a = np.ones(64) if x.alpha is None else x.alpha.copy()
            a[idx] += s
            x.alpha = a
            return t
        checks.append((fd(muta), res["g_alpha"][idx]))
    assert res["g_alpha"][0] == 0.0
    scale = max(abs(a) for a, _ in checks)
    for f, a in checks:
        assert abs(f - a) <= 1e-5 * scale + 1e-4 * abs(f), (f, a)


def _vjp_seeds(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n), rng.standard_normal((n, 3))


def test_field_vjp_alpha_and_q_euler_identity():
    """F and grad F are linear in alpha and in q, so by Euler's theorem for
    homogeneous functions of degree one
      sum_hkl alpha_hkl dPhi/dalpha_hkl = sum_j q_j dPhi/dq_j = Phi,
    Phi = sum_p Fbar F + gFbar . grad F, for any seeds (non-uniform alpha so a
    wrong index order fails)."""
    d = inputs.random_design(4, 7, 0.1, balanced=False)
    rng = np.random.default_rng(9)
    d.alpha = rng.uniform(0.2, 2.0, 64)
    pts = rng.uniform(0.0, 1.0, (300, 3))
    Fb, gFb = _vjp_seeds(300, 10)
    F, gF = oracle.field(d, pts)
    phi = float(Fb @ F + np.sum(gFb * gF))
    _, g_q, g_a = oracle.field_vjp(d, pts, Fb, gFb, want_alpha=True)
    assert abs(float(d.alpha @ g_a) - phi) <= 1e-12 * np.sum(np.abs(Fb) * np.abs(F))
    assert abs(float(d.q @ g_q) - phi) <= 1e-12 * np.sum(np.abs(Fb) * np.abs(F))


def test_field_vjp_alpha_matches_differences_of_the_field():
    """dPhi/dalpha_hkl against central differences of the oracle's forward field
    (exact up to rounding, the field being linear in alpha), every mode."""
    d = inputs.random_design(8, 6, 0.1)
    rng = np.random.default_rng(2)
    d.alpha = rng.uniform(0.5, 1.5, 64)
    pts = rng.uniform(0.0, 1.0, (64, 3))
    Fb, gFb = _vjp_seeds(64, 3)
    _, _, g_a = oracle.field_vjp(d, pts, Fb, gFb, want_alpha=True)

    def phi(a):
        F, gF = oracle.field(d.copy(alpha=a), pts)
        return float(Fb @ F + np.sum(gFb * gF))
    h = 0.25
    fd = np.array([(phi(d.alpha + h * np.eye(64)[m]) - phi(d.alpha - h * np.eye(64)[m])) / (2 * h)
                   for m in range(64)])
    assert fd[0] == pytest.approx(0.0, abs=1e-12)
    np.testing.assert_allclose(g_a, fd, rtol=0, atol=1e-10 * np.abs(fd).max())

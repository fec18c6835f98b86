"""Inverse-design pieces that need no GPU: the effective properties of C^H
against closed forms, their gradients against central differences, and the
CMA-ES against standard test functions."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2511_04025_b300 import objectives  # noqa: E402
from paper_2511_04025_b300.cmaes import CMAES  # noqa: E402


def _t(C):
    return torch.tensor(np.asarray(C, dtype=np.float64))


def test_isotropic_properties_closed_forms():
    E, nu = 2.0, 0.27
    C = _t(oracle.isotropic_C(E, nu))
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    assert abs(float(objectives.young(C, 0)) - E) <= 1e-12 * E
    assert abs(float(objectives.young(C, 2)) - E) <= 1e-12 * E
    assert abs(float(objectives.c_avg(C)) - (lam + 2 * mu)) <= 1e-12
    assert abs(float(objectives.bulk_hill(C)) - E / (3 * (1 - 2 * nu))) <= 1e-12
    assert abs(float(objectives.shear_hill(C)) - mu) <= 1e-12
    assert float(objectives.coupling(C)) == 0.0
    assert abs(float(objectives.uai(C))) <= 1e-12
    assert float(objectives.iso_dist(C)) <= 1e-15


def test_cubic_properties_closed_forms():
    a, b, c = 3.0, 1.2, 0.7  # C11, C12, C44 of a cubic tensor
    C = np.zeros((6, 6))
    C[:3, :3] = b
    np.fill_diagonal(C[:3, :3], a)
    C[3, 3] = C[4, 4] = C[5, 5] = c
    Ct = _t(C)
    # Young's modulus along [100] of a cubic crystal
    assert abs(float(objectives.young(Ct, 0)) - (a - b) * (a + 2 * b) / (a + b)) <= 1e-12
    # cubic: Voigt and Reuss bulk moduli coincide
    assert abs(float(objectives.bulk_hill(Ct)) - (a + 2 * b) / 3) <= 1e-12
    gv = (a - b + 3 * c) / 5
    gr = 5 * (a - b) * c / (4 * c + 3 * (a - b))
    assert abs(float(objectives.shear_hill(Ct)) - 0.5 * (gv + gr)) <= 1e-12
    # universal anisotropy index of a cubic crystal from its Zener ratio
    # A = 2 C44 / (C11 - C12): (6/5) (sqrt A - 1/sqrt A)^2
    A = 2 * c / (a - b)
    assert abs(float(objectives.uai(Ct)) - 1.2 * (A ** 0.5 - A ** -0.5) ** 2) <= 1e-12
    # distance to the isotropic tensor with the Voigt moduli, written out
    # entry by entry in the Mandel form
    k, g = (a + 2 * b) / 3, (a - b + 3 * c) / 5
    d11, d12, d44 = a - (k + 4 * g / 3), b - (k - 2 * g / 3), 2 * (c - g)
    num = (3 * d11 ** 2 + 6 * d12 ** 2 + 3 * d44 ** 2) ** 0.5
    den = (3 * a ** 2 + 6 * b ** 2 + 3 * (2 * c) ** 2) ** 0.5
    assert abs(float(objectives.iso_dist(Ct)) - num / den) <= 1e-14


def test_isotropic_projection_is_the_closest():
    """C_iso minimises the Mandel-form Frobenius distance over all isotropic
    tensors: no perturbation of its two moduli gets closer."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal((6, 6))
    C = A @ A.T + 6 * np.eye(6)
    Ct = _t(C)
    base = float(objectives.iso_dist(Ct))
    cd = C[0, 0] + C[1, 1] + C[2, 2]
    co = C[0, 1] + C[1, 2] + C[0, 2]
    cs = C[3, 3] + C[4, 4] + C[5, 5]
    k0, g0 = (cd + 2 * co) / 9, (cd - co + 3 * cs) / 15
    w = np.array([1, 1, 1, 2 ** 0.5, 2 ** 0.5, 2 ** 0.5])
    for dk, dg in [(1e-3, 0), (-1e-3, 0), (0, 1e-3), (0, -1e-3), (1e-3, 1e-3)]:
        k, g = k0 + dk, g0 + dg
        iso = np.zeros((6, 6))
        iso[:3, :3] = k - 2 * g / 3
        iso[:3, :3] += 2 * g * np.eye(3)
        iso[3:, 3:] = g * np.eye(3)
        M = (C - iso) * np.outer(w, w)
        assert np.linalg.norm(M) / np.linalg.norm(C * np.outer(w, w)) > base


@pytest.mark.parametrize("name", ["Ex", "Cavg", "Keff", "Geff", "coupling", "force", "isotropy"])
def test_objective_gradients_match_central_differences(name):
    rng = np.random.default_rng(3)
    A = rng.standard_normal((6, 6))
    C = A @ A.T + 6 * np.eye(6)  # SPD, with non-zero normal-shear coupling
    fn = objectives.objective(name, k=1, target=2.0)
    V = 0.13
    e, G, gV = objectives.value_and_grad(fn, C, V)
    h = 1e-6
    v64 = lambda x: torch.tensor(x, dtype=torch.float64)  # noqa: E731
    fdV = (float(fn(_t(C), v64(V + h))) - float(fn(_t(C), v64(V - h)))) / (2 * h)
    assert abs(fdV - gV) <= 1e-6 * (1 + abs(fdV))
    if name in ("Ex", "Cavg", "Keff", "Geff"):  # -P / V: dE/dV = P / V^2 = -E / V
        assert abs(gV + e / V) <= 1e-12 * abs(e / V)
    for i in range(6):
        for j in range(6):
            Cp, Cm = C.copy(), C.copy()
            Cp[i, j] += h
            Cm[i, j] -= h
            fd = (float(fn(_t(Cp), v64(V))) - float(fn(_t(Cm), v64(V)))) / (2 * h)
            assert abs(fd - G[i, j]) <= 1e-6 * (1 + abs(fd)), (name, i, j, fd, G[i, j])


def test_cmaes_sphere():
    es = CMAES(np.ones(10), 0.5, seed=1)
    for _ in range(400):
        X = es.ask()
        es.tell(X, np.sum(X ** 2, axis=1))
    assert es.best_f < 1e-10


def test_cmaes_ellipsoid_learns_scaling():
    n = 8
    scale = 10.0 ** (6 * np.arange(n) / (n - 1))
    es = CMAES(np.ones(n), 0.5, seed=2)
    for _ in range(1200):
        X = es.ask()
        es.tell(X, (X ** 2) @ scale)
    assert es.best_f < 1e-8


def test_cmaes_rosenbrock():
    def rosen(X):
        return np.sum(100 * (X[:, 1:] - X[:, :-1] ** 2) ** 2 + (1 - X[:, :-1]) ** 2, axis=1)

    es = CMAES(np.zeros(5), 0.5, seed=4)
    for _ in range(2000):
        X = es.ask()
        es.tell(X, rosen(X))
    assert es.best_f < 1e-8
    assert np.abs(es.best_x - 1).max() < 1e-3


def test_hashin_shtrikman_bounds():
    E, nu = 1.0, 0.3
    K1, G1 = E / (3 * (1 - 2 * nu)), E / (2 * (1 + nu))
    assert objectives.hs_upper(1.0, E, nu) == (K1, G1)
    ku, gu = objectives.hs_upper(1e-12, E, nu)
    assert ku < 1e-11 and gu < 1e-11
    for V in (0.05, 0.1, 0.3, 0.7):
        ku, gu = objectives.hs_upper(V, E, nu)
        # porous solid: the coated-sphere assemblage gives K = 4 G1 K1 V / (3 K1 (1 - V) + 4 G1)
        assert abs(ku - 4 * G1 * K1 * V / (3 * K1 * (1 - V) + 4 * G1)) <= 1e-14
        # both bounds lie below the Voigt (rule-of-mixtures) bounds V K1, V G1
        assert ku < V * K1 and gu < V * G1
    # two identical phases: the bounds return the phase moduli
    ku, gu = objectives.hs_upper(0.4, E, nu, K2=K1 * (1 + 1e-12), G2=G1 * (1 + 1e-12))
    assert abs(ku - K1) <= 1e-9 and abs(gu - G1) <= 1e-9

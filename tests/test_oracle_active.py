"""Pins of the oracle's active-set problem (Sec. 4.2.1: elements with
beta_e <= 1e-3 culled, no ersatz floor, nodes without an active element
removed) against closed forms, an independent dense solve and the limit of
the ersatz-void problem as the void stiffness goes to zero."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2511_04025_b300 import inputs

CORNERS = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0), (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]
N_IDX, T_IDX = [2, 3, 4], [0, 1, 5]  # Voigt 33, 23, 13 (normal z) and 11, 22, 12


def _plane_stress(C):
    """In-plane stiffness of a sheet with free faces (normal stresses zero):
    C_TT - C_TN C_NN^-1 C_NT, embedded in 6x6 (normal rows and columns zero)."""
    CTT = C[np.ix_(T_IDX, T_IDX)]
    CTN = C[np.ix_(T_IDX, N_IDX)]
    CNN = C[np.ix_(N_IDX, N_IDX)]
    out = np.zeros((6, 6))
    out[np.ix_(T_IDX, T_IDX)] = CTT - CTN @ np.linalg.solve(CNN, CTN.T)
    return out


@pytest.mark.parametrize("layers", [[1.0, 1.0, 0.0, 0.0, 1.0, 0.0], [0.5, 0.8, 0.0, 0.0005, 0.3, 0.0]])
def test_laminate_with_culled_layers_closed_form(layers):
    """Layers along z, some culled: the solid sheets are disconnected in z, so
    no normal or transverse-shear stress is carried (those rows of C^H vanish)
    and every active layer deforms in plane stress; the displacement is
    piecewise linear in z, which trilinear elements represent exactly, so
    C^H = sum over active layers of (1/r) rho_l E (C0_TT - C0_TN C0_NN^-1 C0_NT).
    The layer of density 5e-4 lies below the threshold and is culled."""
    r = len(layers)
    rho = np.repeat(np.array(layers), r * r)
    u, it, rr, st, rc, pin = oracle.solve_active(r, rho, tol=1e-13, maxit=20000)
    # In-plane shear 12 of free sheets needs no fluctuation: its load vanishes in
    # exact arithmetic, and the rounding left of it is not orthogonal to the
    # translations of a floating sheet, so CG cannot meet a tolerance relative
    # to it.  Those cases are taken at their exact solution u = 0.
    f = oracle.rhs(r, rc, Evoid=0.0)
    fn = np.sqrt((f ** 2).sum(axis=(1, 2)))
    zero = fn <= 1e-12 * fn.max()
    assert zero[5] and not zero[:5].any()
    assert np.all(rr[~zero] <= 1e-13)
    u[zero] = 0.0
    C, _ = oracle.chom(r, rc, u, Evoid=0.0)
    S = _plane_stress(oracle.isotropic_C())
    ref = sum(l / r * S for l in layers if l > oracle.CULL_THRESHOLD)
    np.testing.assert_allclose(C, ref, rtol=0, atol=1e-9 * np.abs(ref).max())


def _dense_active_C(r, rho_c, E=1.0, nu=0.3):
    """Independent dense solve of the culled problem: numpy assembly over the
    active elements only, inactive nodes dropped, first active node pinned."""
    h = 1.0 / r
    Ke = oracle.element_stiffness(1.0, nu, h)
    n = r ** 3
    K = np.zeros((3 * n, 3 * n))
    F = np.zeros((6, 3 * n))
    chis = [oracle.test_displacement(k, h) for k in range(6)]
    elems = []
    used = np.zeros(n, bool)
    for iz, iy, ix in itertools.product(range(r), repeat=3):
        e = (iz * r + iy) * r + ix
        if rho_c[e] <= 0.0:
            continue
        Ee = rho_c[e] * E
        nodes = [(((iz + c[2]) % r) * r + (iy + c[1]) % r) * r + (ix + c[0]) % r for c in CORNERS]
        used[nodes] = True
        dofs = np.array([3 * nd + i for nd in nodes for i in range(3)])
        elems.append((Ee, dofs))
        K[np.ix_(dofs, dofs)] += Ee * Ke
        for k in range(6):
            np.add.at(F[k], dofs, -Ee * Ke @ chis[k])
    act = np.flatnonzero(used)
    keep = np.array([3 * nd + i for nd in act[1:] for i in range(3)])  # first active node pinned
    U = np.zeros((6, 3 * n))
    for k in range(6):
        # least-norm solve: floating pieces of solid leave the kept system singular but consistent
        U[k, keep] = np.linalg.lstsq(K[np.ix_(keep, keep)], F[k, keep], rcond=1e-12)[0]
    C = np.zeros((6, 6))
    for Ee, dofs in elems:
        w = [chis[k] + U[k, dofs] for k in range(6)]
        for i in range(6):
            for j in range(6):
                C[i, j] += Ee * w[i] @ Ke @ w[j]
    return C, used


@pytest.mark.parametrize("r,seed", [(3, 1), (4, 2), (4, 3)])
def test_active_set_matches_dense_solve(r, seed):
    rng = np.random.default_rng(seed)
    rho = np.where(rng.uniform(size=r ** 3) < 0.5, rng.uniform(0.3, 1.0, r ** 3), 0.0)
    rho[rng.integers(0, r ** 3)] = 5e-4  # below the threshold: culled
    Cd, used = _dense_active_C(r, oracle.cull(rho))
    u, it, rr, st, rc, pin = oracle.solve_active(r, rho, tol=1e-14, maxit=100000)
    assert st == 0
    C, _ = oracle.chom(r, rc, u, Evoid=0.0)
    np.testing.assert_allclose(C, Cd, rtol=0, atol=1e-10 * np.abs(Cd).max())
    # removed nodes keep u = 0; the active-node set matches the dense assembly's
    assert np.array_equal(oracle.active_nodes(r, rc), used)
    assert np.all(u[:, ~used, :] == 0.0)


def test_ersatz_problem_tends_to_the_active_set():
    """As E_void -> 0 the ersatz-void C^H tends to the active-set C^H, to first
    order in E_void (the void carries energy in proportion to its stiffness):
    the gap falls 100-fold per 100-fold smaller E_void and is ~4e-8 of max|C|
    at E_void = 1e-10 on this coarse 10^3 shell (~4e-4 at the ersatz floor
    1e-6: thin voxel connections let the void matter; the gap shrinks with
    refinement, ~8e-5 at 16^3)."""
    r = 10
    d = inputs.plain_32(0)
    m = oracle.voxelize(d, r)["mask"].astype(np.float64)
    u, it, rr, st, rc, pin = oracle.solve_active(r, m, tol=1e-13)
    Ca, _ = oracle.chom(r, rc, u, Evoid=0.0)
    gap = {}
    for ev in (1e-6, 1e-8, 1e-10):
        ud, *_ = oracle.solve(r, m, Evoid=ev, tol=1e-13, maxit=400000)
        Cd, _ = oracle.chom(r, m, ud, Evoid=ev)
        gap[ev] = np.abs(Ca - Cd).max() / np.abs(Ca).max()
    assert gap[1e-10] <= 1e-7
    assert 70 <= gap[1e-6] / gap[1e-8] <= 130 and 70 <= gap[1e-8] / gap[1e-10] <= 130


def test_fully_active_grid_is_the_floorless_problem():
    """With every element active nothing is culled or removed: the active-set
    solve equals the plain solve without a floor (E_void = 0), node 0 pinned."""
    r = 5
    rho = np.random.default_rng(7).uniform(0.2, 1.0, r ** 3)
    u, it, rr, st, rc, pin = oracle.solve_active(r, rho, tol=1e-13)
    assert pin == 0 and np.array_equal(rc, rho)
    u0, *_ = oracle.solve(r, rho, Evoid=0.0, tol=1e-13)
    np.testing.assert_allclose(oracle.chom(r, rc, u, Evoid=0.0)[0], oracle.chom(r, rho, u0, Evoid=0.0)[0],
                               rtol=1e-12, atol=1e-14)

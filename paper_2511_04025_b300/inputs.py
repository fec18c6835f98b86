"""Seeded synthetic design generators shared by the CUDA path and the oracle.

This module holds no arithmetic of the homogenisation method: it only draws
charge positions and magnitudes, expands them by a symmetry group (the
fundamental-bounding-volume mirroring of Sec. 3.2) and fixes the
per-workload constants (grid size, target volume fraction, material).  The
paper's datasets (86 shells, Table 2; 2700 random structures, Sec. 5.2) are
not available, so these generators stand in for them with the same shapes:
2N charges, K = 3 (Sec. 5), shell volume fractions of a few percent.

Every generator takes an integer seed and uses ``numpy.random.default_rng``.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field, replace
from typing import List, Optional

import numpy as np

# Material and solver constants of the workloads: E = 1, nu = 0.3, ersatz
# void modulus 1e-6 (spec configs; Sec. 4.1 stiffness scaling).
E_SOLID = 1.0
NU = 0.3
E_VOID = 1e-6
K_TRUNC = 3  # truncation order used for every example in the paper (Sec. 5)


@dataclass
class Design:
    """A charge design theta = {p_m, q_m, alpha_hkl, c} (Sec. 3.1, Eq. charge-field).

    pos: (n, 3) float64 in [0, 1); q: (n,) float64; alpha: ((K+1)^3,) float64
    indexed [h][k][l] or None for all ones; iso: iso-level c of the shell
    |F - c| <= t |grad F|; vf: target solid volume fraction used to pick the
    half-thickness t; t: explicit half-thickness (cell units) or None.
    """

    pos: np.ndarray
    q: np.ndarray
    alpha: Optional[np.ndarray] = None
    iso: float = 0.0
    K: int = K_TRUNC
    vf: Optional[float] = None
    t: Optional[float] = None

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    def copy(self, **kw) -> "Design":
        d = replace(self, pos=self.pos.copy(), q=self.q.copy(),
                    alpha=None if self.alpha is None else self.alpha.copy())
        return replace(d, **kw) if kw else d


def _balanced_signs(n: int) -> np.ndarray:
    """q_j = +1 for j <= N and -1 for j > N, 2N = n (Sec. 3.1)."""
    assert n % 2 == 0
    return np.concatenate([np.ones(n // 2), -np.ones(n // 2)])


def oh_group() -> List[np.ndarray]:
    """The 48 signed permutation matrices of the cube group O_h."""
    mats = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1.0, -1.0), repeat=3):
            m = np.zeros((3, 3))
            for i, p in enumerate(perm):
                m[i, p] = signs[i]
            mats.append(m)
    return mats


def oh_orbit(seed_point: np.ndarray) -> np.ndarray:
    """Mirror one charge in the tetrahedral FBV to the full cell (Sec. 3.2).

    O_h acts about the cell centre: p -> 1/2 + g (p - 1/2), wrapped into [0,1).
    """
    u = np.asarray(seed_point, dtype=np.float64) - 0.5
    pts = np.array([0.5 + g @ u for g in oh_group()])
    return np.mod(pts, 1.0)


def _fbv_seed(rng: np.random.Generator, margin: float = 1e-3) -> np.ndarray:
    """A point u with margin <= u_z, u_z + margin <= u_y, u_y + margin <= u_x <= 1/2 - margin,
    returned as p = 1/2 + u: strictly inside the tetrahedral FBV, away from every mirror plane."""
    while True:
        u = np.sort(rng.uniform(0.0, 0.5, size=3))[::-1]  # u_x >= u_y >= u_z
        if (u[2] >= margin and u[1] - u[2] >= margin and u[0] - u[1] >= margin
                and 0.5 - u[0] >= margin):
            return 0.5 + u


# --------------------------------------------------------------------------- #
# Workload recipes (seeded).  r = voxels per axis.
# --------------------------------------------------------------------------- #

def plain_32(seed: int = 0) -> Design:
    """32^3 single design: 8 charges uniform in the cube, q = +1 x4, -1 x4,
    zero iso-level, half-thickness chosen for ~15 % solid volume."""
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, 1.0, size=(8, 3))
    return Design(pos=pos, q=_balanced_signs(8), iso=0.0, vf=0.15)


def gaussian_64(seed: int = 0) -> Design:
    """64^3 single design: 32 charges uniform, magnitudes N(0,1), ~8 % solid."""
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, 1.0, size=(32, 3))
    q = rng.standard_normal(32)
    return Design(pos=pos, q=q, iso=0.0, vf=0.08)


def cubic_128(seed: int = 0) -> Design:
    """128^3 single design: the 48-point O_h orbit of one FBV seed (all q = +1,
    so every image carries the same charge), ~5 % solid."""
    rng = np.random.default_rng(seed)
    pos = oh_orbit(_fbv_seed(rng))
    return Design(pos=pos, q=np.ones(48), iso=0.0, vf=0.05)


def gradient_64(seed: int = 0) -> Design:
    """Inverse-design member at 64^3: 24 charges balanced +-1, ~10 % solid."""
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, 1.0, size=(24, 3))
    return Design(pos=pos, q=_balanced_signs(24), iso=0.0, vf=0.10)


def shell_256(seed: int = 0) -> Design:
    """256^3 thin shell in the setting of the paper's timing table (Sec. 5.4):
    explicit half-thickness t = 0.02 (cell units), 32 charges balanced +-1
    uniform in the cell (about 9-10 % solid)."""
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, 1.0, size=(32, 3))
    return Design(pos=pos, q=_balanced_signs(32), iso=0.0, t=0.02)


def random_design(seed: int, n: int, vf: float, balanced: bool = True) -> Design:
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, 1.0, size=(n, 3))
    q = _balanced_signs(n) if balanced else rng.standard_normal(n)
    return Design(pos=pos, q=q, iso=0.0, vf=vf)


# Target tensor of the inverse-design objective: isotropic, bulk K = 0.05,
# shear G = 0.02 in units of E, Voigt order 11,22,33,23,13,12.
def isotropic_target(bulk: float = 0.05, shear: float = 0.02) -> np.ndarray:
    C = np.zeros((6, 6))
    C[:3, :3] = bulk - 2.0 * shear / 3.0
    for i in range(3):
        C[i, i] = bulk + 4.0 * shear / 3.0
        C[3 + i, 3 + i] = shear
    return C


@dataclass
class Request:
    """One serving request: a design on an r^3 grid, arriving at t_arrive (s)."""
    rid: int
    design: Design
    r: int
    t_arrive: float
    session: int
    follow_up_of: int = -1


def serving_stream(seed: int = 0, n_requests: int = 512, rate_hz: float = 100.0) -> List[Request]:
    """Poisson arrivals; grids 32^3/64^3/96^3 with probabilities 0.50/0.35/0.15;
    8..64 charges (even, balanced +-1); volume fraction uniform in [0.03, 0.20];
    25 % of requests revisit an earlier session with positions perturbed by
    N(0, 0.01) (a nearby design, as an interactive edit or an optimiser step
    would submit)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=n_requests)
    t = np.cumsum(gaps) - gaps[0]
    reqs: List[Request] = []
    for i in range(n_requests):
        if i > 0 and rng.uniform() < 0.25:
            base = reqs[int(rng.integers(0, i))]
            pos = np.mod(base.design.pos + rng.normal(0.0, 0.01, size=base.design.pos.shape), 1.0)
            d = base.design.copy(pos=pos)
            reqs.append(Request(i, d, base.r, float(t[i]), base.session, base.rid))
            continue
        r = int(rng.choice([32, 64, 96], p=[0.50, 0.35, 0.15]))
        n = 2 * int(rng.integers(4, 33))  # 8..64, even
        vf = float(rng.uniform(0.03, 0.20))
        pos = rng.uniform(0.0, 1.0, size=(n, 3))
        d = Design(pos=pos, q=_balanced_signs(n), iso=0.0, vf=vf)
        reqs.append(Request(i, d, r, float(t[i]), session=i))
    return reqs

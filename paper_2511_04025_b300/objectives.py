"""Effective properties of C^H and the six inverse-design objectives (Sec. 5.3,
properties as defined in Sec. 5.2).

C^H is 6x6 in Voigt order 11, 22, 33, 23, 13, 12 with engineering shear
strains, S = (C^H)^-1 the compliance.

  E_k      directional Young's modulus, 1 / S_kk
  C_avg    (C_11 + C_22 + C_33) / 3
  K_eff    Hill average of the Voigt and Reuss bulk moduli
           K_V = [(C11 + C22 + C33) + 2 (C12 + C23 + C13)] / 9
           K_R = 1 / [(S11 + S22 + S33) + 2 (S12 + S23 + S13)]
  G_eff    Hill average of the Voigt and Reuss shear moduli
           G_V = [(C11 + C22 + C33) - (C12 + C23 + C13) + 3 (C44 + C55 + C66)] / 15
           G_R = 15 / [4 (S11 + S22 + S33) - 4 (S12 + S23 + S13) + 3 (S44 + S55 + S66)]
  coupling sum over i in {1,2,3}, j in {4,5,6} of |C_ij| (normal-shear coupling)
  UAI      universal anisotropy index 5 G_V / G_R + K_V / K_R - 6 (zero exactly
           for an isotropic tensor), reported beside the moduli in Sec. 5.2
  iso_dist relative distance of C^H to its closest isotropic tensor,
           ||C - C_iso|| / ||C|| in the Frobenius norm of the fourth-order
           tensor (the Mandel form of the 6x6 matrix: shear rows and columns
           scaled by sqrt 2).  Projecting onto the isotropic tensors
           3K P_1 + 2G P_2 in that norm gives K = K_V and G = G_V, so C_iso is
           the isotropic tensor with the Voigt moduli.

Objectives E(C^H, V) (to be minimised), V the solid volume fraction:
  "Ex"       -E_x / V
  "Cavg"     -C_avg / V
  "Keff"     -K_eff / V
  "Geff"     -G_eff / V
  "coupling" -sum |C_ij| (i <= 3 < j)
  "force"    |C_kk - target| (k, target given)
  "isotropy" iso_dist (the "most isotropic structure" task of Sec. 5.3)

dE/dC^H (6x6) and dE/dV come from torch autograd on the CPU (a function of
37 numbers; the GPU adjoint turns them into design gradients, V being the
smoothed volume fraction there).
"""
from __future__ import annotations

from typing import Callable, Tuple

import numpy as np
import torch


def young(C: torch.Tensor, k: int = 0) -> torch.Tensor:
    return 1.0 / torch.linalg.inv(C)[k, k]


def c_avg(C: torch.Tensor) -> torch.Tensor:
    return (C[0, 0] + C[1, 1] + C[2, 2]) / 3.0


def _normal_sums(M: torch.Tensor) -> Tuple[torch.Tensor, torch.Tensor, torch.Tensor]:
    diag = M[0, 0] + M[1, 1] + M[2, 2]
    off = M[0, 1] + M[1, 2] + M[0, 2]
    shear = M[3, 3] + M[4, 4] + M[5, 5]
    return diag, off, shear


def bulk_hill(C: torch.Tensor) -> torch.Tensor:
    cd, co, _ = _normal_sums(C)
    sd, so, _ = _normal_sums(torch.linalg.inv(C))
    kv = (cd + 2.0 * co) / 9.0
    kr = 1.0 / (sd + 2.0 * so)
    return 0.5 * (kv + kr)


def shear_hill(C: torch.Tensor) -> torch.Tensor:
    cd, co, cs = _normal_sums(C)
    sd, so, ss = _normal_sums(torch.linalg.inv(C))
    gv = (cd - co + 3.0 * cs) / 15.0
    gr = 15.0 / (4.0 * sd - 4.0 * so + 3.0 * ss)
    return 0.5 * (gv + gr)


def coupling(C: torch.Tensor) -> torch.Tensor:
    return torch.abs(C[:3, 3:]).sum()


def uai(C: torch.Tensor) -> torch.Tensor:
    cd, co, cs = _normal_sums(C)
    sd, so, ss = _normal_sums(torch.linalg.inv(C))
    kv, kr = (cd + 2.0 * co) / 9.0, 1.0 / (sd + 2.0 * so)
    gv, gr = (cd - co + 3.0 * cs) / 15.0, 15.0 / (4.0 * sd - 4.0 * so + 3.0 * ss)
    return 5.0 * gv / gr + kv / kr - 6.0


def _mandel(C: torch.Tensor) -> torch.Tensor:
    w = torch.tensor([1.0, 1.0, 1.0, 2.0 ** 0.5, 2.0 ** 0.5, 2.0 ** 0.5], dtype=C.dtype)
    return C * w[:, None] * w[None, :]


def iso_dist(C: torch.Tensor) -> torch.Tensor:
    cd, co, cs = _normal_sums(C)
    k = (cd + 2.0 * co) / 9.0
    g = (cd - co + 3.0 * cs) / 15.0
    lam = k - 2.0 * g / 3.0
    eye3 = torch.eye(3, dtype=C.dtype)
    iso = torch.zeros(6, 6, dtype=C.dtype)
    iso[:3, :3] = lam + 2.0 * g * eye3
    iso[3:, 3:] = g * eye3
    return torch.linalg.norm(_mandel(C - iso)) / torch.linalg.norm(_mandel(C))


def hs_upper(V: float, E: float = 1.0, nu: float = 0.3, K2: float = 0.0, G2: float = 0.0) -> Tuple[float, float]:
    """Hashin-Shtrikman upper bounds (bulk, shear) of an isotropic two-phase
    mixture: the stiffer phase (Young's modulus E, Poisson ratio nu) at volume
    fraction V and a phase (K2, G2) at 1 - V, void by default (the bounds the
    optimised K_eff and G_eff are measured against in Sec. 5.3)."""
    K1 = E / (3.0 * (1.0 - 2.0 * nu))
    G1 = E / (2.0 * (1.0 + nu))
    if V >= 1.0:
        return K1, G1
    ku = K1 + (1.0 - V) / ((1.0 / (K2 - K1) if K2 != K1 else float("inf")) + 3.0 * V / (3.0 * K1 + 4.0 * G1))
    gu = G1 + (1.0 - V) / ((1.0 / (G2 - G1) if G2 != G1 else float("inf"))
                           + 6.0 * V * (K1 + 2.0 * G1) / (5.0 * G1 * (3.0 * K1 + 4.0 * G1)))
    return ku, gu


def objective(name: str, k: int = 0, target: float = 0.0) -> Callable[[torch.Tensor, torch.Tensor], torch.Tensor]:
    """The objective E(C, V) named by `name` (see the module docstring)."""
    if name == "Ex":
        return lambda C, V: -young(C, k) / V
    if name == "Cavg":
        return lambda C, V: -c_avg(C) / V
    if name == "Keff":
        return lambda C, V: -bulk_hill(C) / V
    if name == "Geff":
        return lambda C, V: -shear_hill(C) / V
    if name == "coupling":
        return lambda C, V: -coupling(C)
    if name == "force":
        return lambda C, V: torch.abs(C[k, k] - target)
    if name == "isotropy":
        return lambda C, V: iso_dist(C)
    raise ValueError(f"unknown objective {name!r}")


def value_and_grad(fn: Callable[[torch.Tensor, torch.Tensor], torch.Tensor], C: np.ndarray, V: float
                   ) -> Tuple[float, np.ndarray, float]:
    """E(C, V), dE/dC (6x6, every entry of C treated as independent) and dE/dV."""
    Ct = torch.tensor(np.asarray(C, dtype=np.float64), requires_grad=True)
    Vt = torch.tensor(float(V), dtype=torch.float64, requires_grad=True)
    e = fn(Ct, Vt)
    e.backward()
    gV = 0.0 if Vt.grad is None else float(Vt.grad)
    return float(e.detach()), Ct.grad.numpy().copy(), gV

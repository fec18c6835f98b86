"""Inverse design on top of the homogenisation path (Sec. 4.3).

The driver alternates three stages (the paper's joint optimisation with a
volume constraint):
  (i)   the shell thickness t is set so that the voxelised shell meets the
        target volume fraction (the GPU rank selection of shl_voxelize, which
        reaches the same t as a bisection on the solid count);
  (ii)  a fixed number of first-order (Adam) steps on the mode weights
        alpha_hkl with the charge positions fixed; each step runs the forward
        homogenisation and the hand-written adjoint (shl_grad, which starts
        from the forward's displacements, so the adjoint costs no new CG
        iterations);
  (iii) a fixed number of CMA-ES generations on the charge positions with
        alpha fixed; every population is submitted at once to the serving
        path (continuous batching: the candidates' solves overlap on the
        GPU), each candidate with its own thickness from the volume fraction.
Objectives: the six of Sec. 5.3 (module objectives).  The solves use the
smoothed density (the one the gradients differentiate) in FP32 with FP64
refinement.  V in the objectives is the target volume fraction, which stage
(i) and the per-candidate thickness maintain.

Every step runs in libshl; this module only orchestrates.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import torch

from . import inputs, objectives, shl
from .cmaes import CMAES


@dataclass
class History:
    objective: List[float] = field(default_factory=list)  # incumbent after each stage
    stage: List[str] = field(default_factory=list)
    evaluations: int = 0


class InverseDesign:
    def __init__(self, handle, design: inputs.Design, r: int, objective: str, vf: float, k: int = 0,
                 target: float = 0.0, tol: float = 1e-7, lr_alpha: float = 0.05, sigma0: float = 0.03,
                 popsize: Optional[int] = None, seed: int = 0):
        self.h = handle
        self.r = r
        self.vf = vf
        self.fn = objectives.objective(objective, k, target)
        self.opts = shl.default_solve_opts(precision=shl.SHL_FP32_REFINE, tol=tol, density=shl.SHL_SMOOTH)
        na = (design.K + 1) ** 3
        alpha = np.ones(na) if design.alpha is None else np.asarray(design.alpha, dtype=np.float64)
        self.design = design.copy(alpha=alpha.copy(), vf=vf, t=None)
        self.lr = lr_alpha
        self.sigma0 = sigma0
        self.popsize = popsize
        self.seed = seed
        self.hist = History()
        self.popsize_used = popsize or 4 + int(3 * math.log(design.pos.size))
        self._u = None  # forward displacements on the device (allocated by the first alpha step)
        self._adam_m = np.zeros(na)
        self._adam_v = np.zeros(na)
        self._adam_t = 0
        self.value = self.evaluate([self.design])[0]

    # -- evaluation ---------------------------------------------------------
    def evaluate(self, designs: List[inputs.Design]) -> List[float]:
        """Objective values of designs (volume fraction vf each), solved
        concurrently through the serving path."""
        tickets = [shl.shl_serve_submit(self.h, d.copy(vf=self.vf, t=None), self.r, self.opts) for d in designs]
        out = []
        for tk in tickets:
            res = shl.shl_serve_wait(self.h, tk)
            st = res["stats"]["status"]
            if st not in (shl.SHL_OK, shl.SHL_ENOCONV):
                out.append(math.inf)
            else:
                out.append(float(self.fn(torch.tensor(res["C"], dtype=torch.float64),
                                         torch.tensor(self.vf, dtype=torch.float64))))
        self.hist.evaluations += len(designs)
        return out

    # -- stage (i) ------------------------------------------------------------
    def thickness(self) -> float:
        return shl.shl_voxelize(self.h, self.design.copy(vf=self.vf, t=None), self.r)["t"]

    # -- stage (ii) -----------------------------------------------------------
    def alpha_steps(self, n: int) -> None:
        """n Adam steps on alpha (kept >= 0) with t from stage (i) held fixed.
        With t fixed the volume moves with alpha, so each step differentiates
        E(C^H, V) with V the smoothed volume fraction of the current design."""
        t = self.thickness()
        if self._u is None:
            self._u = torch.empty(18 * self.r ** 3, dtype=torch.float64, device=shl.ctx_device(self.h))
        for _ in range(n):
            fwd = shl.shl_grad(self.h, self.design, self.r, self.opts, np.zeros((6, 6)), u=self._u, t=t)
            _, G, gV = objectives.value_and_grad(self.fn, fwd["C"], fwd["V"])
            o = shl.default_solve_opts(precision=self.opts.precision, tol=self.opts.tol, density=self.opts.density,
                                       warm_start=1)
            g = shl.shl_grad(self.h, self.design, self.r, o, G, u=self._u, t=t, want_alpha=True,
                             dEdV=gV)["g_alpha"]
            self._adam_t += 1
            b1, b2 = 0.9, 0.999
            self._adam_m = b1 * self._adam_m + (1 - b1) * g
            self._adam_v = b2 * self._adam_v + (1 - b2) * g * g
            mh = self._adam_m / (1 - b1 ** self._adam_t)
            vh = self._adam_v / (1 - b2 ** self._adam_t)
            alpha = np.maximum(self.design.alpha - self.lr * mh / (np.sqrt(vh) + 1e-12), 0.0)
            self.design = self.design.copy(alpha=alpha)
        self.value = self.evaluate([self.design])[0]
        self.hist.objective.append(self.value)
        self.hist.stage.append("alpha")

    # -- stage (iii) ----------------------------------------------------------
    def position_generations(self, n: int) -> None:
        """n CMA-ES generations on the charge positions (periodic, wrapped
        into the unit cell); the incumbent moves to the best candidate seen
        when it improves on it."""
        es = CMAES(self.design.pos.ravel(), self.sigma0, seed=self.seed + len(self.hist.stage), popsize=self.popsize)
        shape = self.design.pos.shape
        for _ in range(n):
            X = es.ask()
            cands = [self.design.copy(pos=np.mod(x.reshape(shape), 1.0)) for x in X]
            es.tell(X, np.asarray(self.evaluate(cands)))
        if es.best_f < self.value:
            self.design = self.design.copy(pos=np.mod(es.best_x.reshape(shape), 1.0))
            self.value = float(es.best_f)
        self.hist.objective.append(self.value)
        self.hist.stage.append("positions")

    def run(self, outer: int, n_alpha: int, n_gen: int) -> History:
        for _ in range(outer):
            self.alpha_steps(n_alpha)
            self.position_generations(n_gen)
        return self.hist

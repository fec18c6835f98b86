"""CMA-ES, the (mu/mu_w, lambda) covariance-matrix-adaptation evolution
strategy with cumulative step-size adaptation and rank-one + rank-mu
covariance updates (the standard form of Hansen's tutorial), used by the
inverse-design driver for the charge positions (Sec. 4.3: positions by
CMA-ES, weights by gradient descent).  Plain numpy, ask / tell interface;
candidate evaluation is the caller's (the driver batches it through the
serving path).
"""
from __future__ import annotations

import math
from typing import Optional

import numpy as np


class CMAES:
    def __init__(self, x0, sigma0: float, seed: int = 0, popsize: Optional[int] = None):
        self.m = np.asarray(x0, dtype=np.float64).copy()
        n = self.n = self.m.size
        self.sigma = float(sigma0)
        self.rng = np.random.default_rng(seed)
        self.lam = popsize or 4 + int(3 * math.log(n))
        self.mu = self.lam // 2
        w = math.log(self.mu + 0.5) - np.log(np.arange(1, self.mu + 1))
        self.w = w / w.sum()
        self.mueff = 1.0 / np.sum(self.w ** 2)
        mueff = self.mueff
        self.cs = (mueff + 2.0) / (n + mueff + 5.0)
        self.ds = 1.0 + 2.0 * max(0.0, math.sqrt((mueff - 1.0) / (n + 1.0)) - 1.0) + self.cs
        self.cc = (4.0 + mueff / n) / (n + 4.0 + 2.0 * mueff / n)
        self.c1 = 2.0 / ((n + 1.3) ** 2 + mueff)
        self.cmu = min(1.0 - self.c1, 2.0 * (mueff - 2.0 + 1.0 / mueff) / ((n + 2.0) ** 2 + mueff))
        self.chin = math.sqrt(n) * (1.0 - 1.0 / (4.0 * n) + 1.0 / (21.0 * n * n))  # E||N(0, I)||
        self.ps = np.zeros(n)
        self.pc = np.zeros(n)
        self.C = np.eye(n)
        self.B = np.eye(n)
        self.D = np.ones(n)
        self.gen = 0
        self.best_x = self.m.copy()
        self.best_f = math.inf
        self._y = None

    def ask(self) -> np.ndarray:
        """lambda candidates, one per row."""
        z = self.rng.standard_normal((self.lam, self.n))
        self._y = (z * self.D) @ self.B.T  # y = B D z
        return self.m + self.sigma * self._y

    def tell(self, X: np.ndarray, f: np.ndarray) -> None:
        """Update from the candidates of the last ask() and their values (lower is better)."""
        f = np.asarray(f, dtype=np.float64)
        order = np.argsort(f, kind="stable")
        if f[order[0]] < self.best_f:
            self.best_f = float(f[order[0]])
            self.best_x = np.asarray(X[order[0]], dtype=np.float64).copy()
        y = self._y[order[: self.mu]]
        yw = self.w @ y
        self.m = self.m + self.sigma * yw
        # C^(-1/2) yw = B D^-1 B^T yw
        cinv_yw = self.B @ ((self.B.T @ yw) / self.D)
        self.ps = (1.0 - self.cs) * self.ps + math.sqrt(self.cs * (2.0 - self.cs) * self.mueff) * cinv_yw
        self.gen += 1
        ps_norm = np.linalg.norm(self.ps)
        hs = ps_norm / math.sqrt(1.0 - (1.0 - self.cs) ** (2 * self.gen)) < (1.4 + 2.0 / (self.n + 1.0)) * self.chin
        self.pc = (1.0 - self.cc) * self.pc + (math.sqrt(self.cc * (2.0 - self.cc) * self.mueff) * yw if hs else 0.0)
        rank_mu = (y * self.w[:, None]).T @ y
        delta = (1.0 - hs) * self.cc * (2.0 - self.cc)
        self.C = ((1.0 - self.c1 - self.cmu) * self.C + self.c1 * (np.outer(self.pc, self.pc) + delta * self.C)
                  + self.cmu * rank_mu)
        self.sigma *= math.exp((self.cs / self.ds) * (ps_norm / self.chin - 1.0))
        self.C = 0.5 * (self.C + self.C.T)
        ev, self.B = np.linalg.eigh(self.C)
        self.D = np.sqrt(np.maximum(ev, 1e-300))

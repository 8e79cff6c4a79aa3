"""ORACLE (test infrastructure): objective, gradient, projection, gradient map.

Only tests/, __graft_entry__.smoke() and bench.py's CPU legs may import this.

  phi(x) = 1/2 ||A x - b||^2 + alpha TV_tau(x)                (eq. TVobjectivefunction)
  grad phi(x) = A^T (A x - b) + alpha grad TV_tau(x)
  P_Q(x) = max(x, 0) for Q = R_+^N                             (Sec. III-A, Sec. IV-A)
  G_nu(x) = nu (x - P_Q(x - grad phi(x) / nu))                 (Sec. III-D)
All in FP64; A is a scipy CSR matrix (its matvec is the library primitive).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp

from . import tv


@dataclasses.dataclass
class Problem:
    A: sp.csr_matrix
    b: np.ndarray          # float64 [m]
    n: int                 # grid edge
    alpha: float
    tau: float

    @property
    def N(self) -> int:
        return self.n ** 3

    def residual(self, x):
        return self.A @ x - self.b

    def data_term(self, x) -> float:
        r = self.residual(x)
        return 0.5 * float(r @ r)

    def f(self, x) -> float:
        """phi(x)."""
        r = self.residual(x)
        return 0.5 * float(r @ r) + self.alpha * tv.tv_value(x, self.n, self.tau)

    def grad(self, x) -> np.ndarray:
        """grad phi(x)."""
        r = self.residual(x)
        return self.A.T @ r + self.alpha * tv.tv_grad(x, self.n, self.tau)

    def f_and_grad(self, x):
        r = self.residual(x)
        f = 0.5 * float(r @ r) + self.alpha * tv.tv_value(x, self.n, self.tau)
        g = self.A.T @ r + self.alpha * tv.tv_grad(x, self.n, self.tau)
        return f, g


def project_Q(x: np.ndarray) -> np.ndarray:
    """P_Q onto the nonnegative orthant."""
    return np.maximum(x, 0.0)


def gradient_map(x: np.ndarray, g: np.ndarray, nu: float) -> np.ndarray:
    """G_nu(x) for gradient g = grad phi(x)."""
    return nu * (x - project_Q(x - g / nu))

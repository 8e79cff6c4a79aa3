"""ORACLE (test infrastructure): discrete TV and its Huber smoothing, FP64.

Only tests/, __graft_entry__.smoke() and bench.py's CPU legs may import this.

Eq. (TV) of Sec. II-A: TV(x) = sum_j ||D_j x||_2, D_j the forward-difference
approximation of the gradient at voxel j.  The paper states that phi has a
Lipschitz gradient (Sec. II-B), which the plain norm does not give; the smooth
surrogate used throughout is the Huber function

    h_tau(z) = ||z|| - tau/2        if ||z|| >= tau
             = ||z||^2 / (2 tau)    otherwise,
    grad h_tau(z) = z / max(tau, ||z||),

so TV_tau(x) = sum_j h_tau(D_j x) and grad TV_tau(x) = sum_j D_j^T grad h_tau(D_j x).
Boundary: the component of D_j x along axis e is x_{j+e} - x_j when j+e is
inside the grid and 0 otherwise.  Arrays are [iz, iy, ix] (x fastest).
"""
from __future__ import annotations

import numpy as np


def forward_differences(x: np.ndarray, n: int):
    """(dx, dy, dz), each [n, n, n]: the three components of D_j x for every j."""
    v = np.asarray(x, dtype=np.float64).reshape(n, n, n)
    dx = np.zeros_like(v)
    dy = np.zeros_like(v)
    dz = np.zeros_like(v)
    dx[:, :, :-1] = v[:, :, 1:] - v[:, :, :-1]
    dy[:, :-1, :] = v[:, 1:, :] - v[:, :-1, :]
    dz[:-1, :, :] = v[1:, :, :] - v[:-1, :, :]
    return dx, dy, dz


def huber(norm: np.ndarray, tau: float) -> np.ndarray:
    return np.where(norm >= tau, norm - 0.5 * tau, norm * norm / (2.0 * tau))


def tv_value(x: np.ndarray, n: int, tau: float) -> float:
    """TV_tau(x) = sum_j h_tau(D_j x)."""
    dx, dy, dz = forward_differences(x, n)
    nrm = np.sqrt(dx * dx + dy * dy + dz * dz)
    return float(np.sum(huber(nrm, tau)))


def tv_plain(x: np.ndarray, n: int) -> float:
    """Unsmoothed TV(x) = sum_j ||D_j x||_2 (eq. TV)."""
    dx, dy, dz = forward_differences(x, n)
    return float(np.sum(np.sqrt(dx * dx + dy * dy + dz * dz)))


def tv_grad(x: np.ndarray, n: int, tau: float) -> np.ndarray:
    """grad TV_tau(x) = sum_j D_j^T (D_j x / max(tau, ||D_j x||)), flat [n^3]."""
    dx, dy, dz = forward_differences(x, n)
    nrm = np.sqrt(dx * dx + dy * dy + dz * dz)
    den = np.maximum(tau, nrm)
    wx, wy, wz = dx / den, dy / den, dz / den
    # D_j^T w: component e of D_j x is x_{j+e} - x_j, so w_e adds to j+e and
    # subtracts from j (w_e is 0 where j+e leaves the grid).
    g = -(wx + wy + wz)
    g[:, :, 1:] += wx[:, :, :-1]
    g[:, 1:, :] += wy[:, :-1, :]
    g[1:, :, :] += wz[:-1, :, :]
    return g.reshape(-1)

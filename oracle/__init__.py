"""FP64 CPU oracle of the TV-CT gradient methods -- TEST INFRASTRUCTURE.

Only tests/, __graft_entry__.smoke() and bench.py's CPU legs (cpu_baseline and
``--impl reference``) may import, call or execute anything in this package.
The product path (paper_1105_4002_gb300) never does; it shares no code, header
or table with this package.  The only shared module is ``synth`` (seeded input
data, none of the method's arithmetic).

Contents, each written from the paper:
  _siddon.py / siddon.c  system matrix A (Siddon lengths, FP64), Sec. II-A
  tv.py                  TV and its Huber smoothing, eq. (TV)
  objective.py           phi, grad phi, P_Q, gradient map, eq. (TVobjectivefunction), Sec. III-D
  solvers.py             GP, GPBB (Alg. 1), BT (Alg. 2), UPN (Alg. 3)
"""
from __future__ import annotations

import numpy as np

from . import tv
from ._siddon import adjoint, build, forward, row, system_matrix, trace_ray
from .objective import Problem, gradient_map, project_Q
from .solvers import (ERR_LINESEARCH, ERR_NONFINITE, NOT_CONVERGED, OK, Options, Result,
                      solve_gp, solve_gpbb, solve_upn, upn_theta_next)


def make_data(A, x_true: np.ndarray, z: np.ndarray, level: float) -> np.ndarray:
    """b = A x_true + e with e = level * ||A x_true|| / sqrt(m) * z (Sec. IV-A noise).

    The result is rounded to FP32 and returned as FP64, so that the oracle
    and the FP32 GPU path solve exactly the same data.
    """
    ax = A @ x_true
    sigma = level * float(np.linalg.norm(ax)) / np.sqrt(ax.size)
    b = ax + sigma * z
    return b.astype(np.float32).astype(np.float64)


def problem_from_config(cfg, alpha=None, tau=None):
    """(Problem, geometry, x_true) for a synth.Config."""
    g = cfg.geometry()
    A = system_matrix(g)
    x_true = cfg.phantom()
    b = make_data(A, x_true, cfg.noise_direction(), cfg.noise)
    prob = Problem(A=A, b=b, n=cfg.n, alpha=cfg.alpha if alpha is None else alpha,
                   tau=cfg.tau if tau is None else tau)
    return prob, g, x_true


__all__ = [
    "adjoint", "build", "forward", "row", "system_matrix", "trace_ray", "tv", "Problem", "gradient_map",
    "project_Q", "Options", "Result", "solve_gp", "solve_gpbb", "solve_upn", "upn_theta_next",
    "make_data", "problem_from_config", "OK", "NOT_CONVERGED", "ERR_LINESEARCH", "ERR_NONFINITE",
]

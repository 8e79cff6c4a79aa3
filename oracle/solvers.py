"""ORACLE (test infrastructure): GP, GPBB and UPN in plain FP64 numpy.

Only tests/, __graft_entry__.smoke() and bench.py's CPU legs may import this.

Each solver follows the paper's steps in its order and notation, with f = phi:
  * GP   -- eq. (gradientmethod) x+ = P_Q(x - theta_k grad f(x)); the step
            rule is not given, so theta_k = 1/L_k with L_k from BT (Alg. 2)
            started at L_{k-1}.
  * GPBB -- Alg. 1: BB step ||s||^2 / <s, y>, beta from 0.95 squared until
            f(xbar) < max_{i<=K} f(x^(k-i)) - sigma grad f(x)^T (x - xbar);
            K = 2, sigma = 0.1 (Sec. III-A).
  * BT   -- Alg. 2: L <- rho_L L until
            f(x) <= f(y) + grad f(y)^T (x - y) + L/2 ||x - y||^2.
  * UPN  -- Alg. 3 with the strong-convexity estimate eq. (mu_k_estimate).
Stopping rule (Sec. III-D): stop after iteration k when ||G_nu(x^(k))||_2 / N
<= eps ("per_n"), or, relative form, ||G|| / ||G at iteration 0|| <= eps ("rel").

Readings where the paper is silent (all shared with the CUDA path's defaults):
  theta_0 = 1; for k < K the max runs over the available f's; if <s, y> <= 0
  or s = 0 the previous theta is kept; GPBB rejects at equality; at most
  ``gpbb_max_trials`` squarings of beta per iteration, at most ``bt_max``
  increases of L per BT call; rho_L = 2, Lbar = 1, mubar = 0.1 Lbar;
  theta_1 = sqrt(min(1, mu_0 / L_0)); nu = L_k for GP and UPN (the gradient
  map at the BT base point, G = L_k (base - x+)), nu = 1/theta_k for GPBB;
  mu-estimate pair (x^(k), y^(k)) as printed, skipped when
  1/2 ||x - y||^2 <= 1e-300 or non-finite, clamped at >= 0.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from .objective import Problem, project_Q

OK = 0
NOT_CONVERGED = 1
ERR_LINESEARCH = -4
ERR_NONFINITE = -5


@dataclasses.dataclass
class Options:
    k_max: int = 20000
    stop: str = "rel"           # "rel" or "per_n"
    gpbb_K: int = 2
    gpbb_sigma: float = 0.1
    gpbb_beta0: float = 0.95
    gpbb_max_trials: int = 12
    rho_L: float = 2.0
    L_bar: float = 1.0
    mu_bar: float | None = None  # None -> 0.1 * L_bar
    bt_max: int = 60
    record: bool = False
    # with record: also keep, per iteration, copies of the vectors the step's
    # scalars came from (GPBB: x^(k) and grad f(x^(k)); UPN: the pair
    # (x^(k), y^(k)) of the mu-estimate), so that tests can recompute them
    record_iterates: bool = False


@dataclasses.dataclass
class Result:
    x: np.ndarray
    status: int
    iters: int
    f_evals: int = 0
    g_evals: int = 0
    gnorm: float = math.nan
    gnorm0: float = math.nan
    f: float = math.nan
    L: float = math.nan
    theta: float = math.nan
    mu: float = math.nan
    history: list = dataclasses.field(default_factory=list)


class _Counter:
    def __init__(self, prob: Problem):
        self.p = prob
        self.nf = 0
        self.ng = 0

    def f(self, x):
        self.nf += 1
        return self.p.f(x)

    def f_and_grad(self, x):
        self.nf += 1
        self.ng += 1
        return self.p.f_and_grad(x)

    def grad(self, x):
        self.ng += 1
        return self.p.grad(x)


def _stop_value(gnorm: float, gnorm0: float, N: int, mode: str) -> float:
    if mode == "per_n":
        return gnorm / N
    return gnorm / gnorm0 if gnorm0 > 0 else 0.0


class LineSearchError(RuntimeError):
    pass


def backtracking(c: _Counter, y, fy, gy, L_bar, opts: Options):
    """Alg. 2 (BT): returns (x, L, f(x), number of increases of L)."""
    L = L_bar
    x = project_Q(y - gy / L)
    fx = c.f(x)
    j = 0
    while True:
        d = x - y
        bound = fy + float(gy @ d) + 0.5 * L * float(d @ d)
        if not fx > bound:
            return x, L, fx, j
        j += 1
        if j > opts.bt_max:
            raise LineSearchError("BT: L increased bt_max times")
        L = opts.rho_L * L
        x = project_Q(y - gy / L)
        fx = c.f(x)


def solve_gp(prob: Problem, x0, eps: float, opts: Options | None = None) -> Result:
    opts = opts or Options()
    c = _Counter(prob)
    x = np.array(x0, dtype=np.float64)
    N = x.size
    f, g = c.f_and_grad(x)
    L = opts.L_bar
    gnorm0 = math.nan
    hist = []
    status = NOT_CONVERGED
    k = 0
    gnorm = math.nan
    try:
        for k in range(opts.k_max):
            x_new, L, f_new, j = backtracking(c, x, f, g, L, opts)
            gnorm = L * float(np.linalg.norm(x - x_new))     # ||G_{L_k}(x^(k))||
            if k == 0:
                gnorm0 = gnorm
            x, f = x_new, f_new
            if opts.record:
                hist.append(dict(k=k, f=f, gnorm=gnorm, L=L, trials=j))
            if not (math.isfinite(f) and math.isfinite(gnorm)):
                status = ERR_NONFINITE
                break
            if _stop_value(gnorm, gnorm0, N, opts.stop) <= eps:
                status = OK
                break
            g = c.grad(x)
    except LineSearchError:
        status = ERR_LINESEARCH
    return Result(x=x, status=status, iters=k + 1, f_evals=c.nf, g_evals=c.ng, gnorm=gnorm,
                  gnorm0=gnorm0, f=f, L=L, history=hist)


def solve_gpbb(prob: Problem, x0, eps: float, opts: Options | None = None) -> Result:
    opts = opts or Options()
    c = _Counter(prob)
    K, sigma = opts.gpbb_K, opts.gpbb_sigma
    x = np.array(x0, dtype=np.float64)
    N = x.size
    theta = 1.0                                  # theta_0 = 1
    f, g = c.f_and_grad(x)
    fhist = [f]
    x_prev = g_prev = None
    gnorm0 = math.nan
    gnorm = math.nan
    hist = []
    status = NOT_CONVERGED
    k = 0
    for k in range(opts.k_max):
        if k > 0:                                # BB strategy
            s = x - x_prev
            yv = g - g_prev
            sy = float(s @ yv)
            ss = float(s @ s)
            if sy > 0.0 and ss > 0.0:
                theta = ss / sy
        beta = opts.gpbb_beta0
        xbar = project_Q(x - beta * theta * g)
        fhat = max(fhist[-(K + 1):])
        gnorm = float(np.linalg.norm(x - project_Q(x - theta * g))) / theta  # nu = 1/theta_k
        if k == 0:
            gnorm0 = gnorm
        fbar = c.f(xbar)
        trials = 0
        failed = False
        while fbar >= fhat - sigma * float(g @ (x - xbar)):
            trials += 1
            if trials > opts.gpbb_max_trials:
                failed = True
                break
            beta = beta * beta
            xbar = project_Q(x - beta * theta * g)
            fbar = c.f(xbar)
        if failed:
            status = ERR_LINESEARCH
            break
        x_prev, g_prev = x, g
        x, f = xbar, fbar
        fhist.append(f)
        if opts.record:
            hist.append(dict(k=k, f=f, gnorm=gnorm, theta=theta, beta=beta, trials=trials))
            if opts.record_iterates:
                hist[-1].update(x=x_prev.copy(), g=g_prev.copy())
        if not (math.isfinite(f) and math.isfinite(gnorm)):
            status = ERR_NONFINITE
            break
        if _stop_value(gnorm, gnorm0, N, opts.stop) <= eps:
            status = OK
            break
        g = c.grad(x)
    return Result(x=x, status=status, iters=k + 1, f_evals=c.nf, g_evals=c.ng, gnorm=gnorm,
                  gnorm0=gnorm0, f=f, theta=theta, history=hist)


def upn_theta_next(theta: float, q: float) -> float:
    """Positive root of t^2 = (1 - t) theta^2 + q t."""
    a = theta * theta - q
    return 0.5 * (-a + math.sqrt(a * a + 4.0 * theta * theta))


def solve_upn(prob: Problem, x0, eps: float, opts: Options | None = None) -> Result:
    opts = opts or Options()
    c = _Counter(prob)
    mu = opts.mu_bar if opts.mu_bar is not None else 0.1 * opts.L_bar
    x0 = np.array(x0, dtype=np.float64)
    N = x0.size
    hist = []
    f0, g0 = c.f_and_grad(x0)
    try:
        xk, L, fk, j = backtracking(c, x0, f0, g0, opts.L_bar, opts)   # [x1, L0] = BT(x0, Lbar)
    except LineSearchError:
        return Result(x=x0, status=ERR_LINESEARCH, iters=0, f_evals=c.nf, g_evals=c.ng)
    gnorm0 = L * float(np.linalg.norm(x0 - xk))                          # G_{L0}(x0)
    gnorm = gnorm0
    if opts.record:
        hist.append(dict(k=0, f=fk, gnorm=gnorm, L=L, mu=mu, trials=j))
    if _stop_value(gnorm, gnorm0, N, opts.stop) <= eps:
        return Result(x=xk, status=OK, iters=1, f_evals=c.nf, g_evals=c.ng, gnorm=gnorm,
                      gnorm0=gnorm0, f=fk, L=L, mu=mu, history=hist)
    y = xk.copy()                                                          # y1 = x1
    theta = math.sqrt(min(1.0, mu / L))                                    # theta1
    status = NOT_CONVERGED
    k = 0
    try:
        for k in range(1, opts.k_max):
            fy, gy = c.f_and_grad(y)
            x_new, L, f_new, j = backtracking(c, y, fy, gy, L, opts)       # [x(k+1), L_k]
            d = xk - y                                                     # mu_k from (x(k), y(k))
            dd = 0.5 * float(d @ d)
            if dd > 1e-300:
                M = (fk - fy - float(gy @ d)) / dd
                if math.isfinite(M):
                    mu = min(mu, max(M, 0.0))
            theta_new = upn_theta_next(theta, mu / L)
            beta = theta * (1.0 - theta) / (theta * theta + theta_new)
            gnorm = L * float(np.linalg.norm(y - x_new))                   # G_{L_k}(y(k))
            pair = (xk, y)
            y = x_new + beta * (x_new - xk)
            xk, fk, theta = x_new, f_new, theta_new
            if opts.record:
                hist.append(dict(k=k, f=fk, gnorm=gnorm, L=L, mu=mu, theta=theta, beta=beta,
                                 trials=j))
                if opts.record_iterates:
                    hist[-1].update(x=pair[0].copy(), y=pair[1].copy())
            if not (math.isfinite(fk) and math.isfinite(gnorm)):
                status = ERR_NONFINITE
                break
            if _stop_value(gnorm, gnorm0, N, opts.stop) <= eps:
                status = OK
                break
    except LineSearchError:
        status = ERR_LINESEARCH
    return Result(x=xk, status=status, iters=k + 1, f_evals=c.nf, g_evals=c.ng, gnorm=gnorm,
                  gnorm0=gnorm0, f=fk, L=L, theta=theta, mu=mu, history=hist)

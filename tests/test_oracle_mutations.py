"""Planted mistakes in the oracle (on the CPU) must be caught by its pins.

Each case plants one plausible error into the oracle -- by monkeypatching a
function, or by loading a copy of an oracle module whose source has one
edit -- and re-runs the check that is meant to catch it; the check must now
fail.
"""
import inspect
import math
import sys
import types

import numpy as np
import pytest

import oracle
from oracle import objective, tv


def _fd_ok(prob, x):
    f, g = prob.f_and_grad(x)
    h = 1e-6
    for j in range(0, prob.N, 7):
        e = np.zeros(prob.N)
        e[j] = h
        fd = (prob.f(x + e) - prob.f(x - e)) / (2 * h)
        if abs(fd - g[j]) > 1e-5 * (1 + abs(g[j])):
            return False
    return True


@pytest.fixture
def prob():
    from conftest import small_geometry
    g = small_geometry(n=4, views=6, det=6)
    A = oracle.system_matrix(g)
    rng = np.random.default_rng(2)
    return oracle.Problem(A=A, b=A @ rng.uniform(0, 1, g.N), n=4, alpha=0.3, tau=0.05), \
        rng.uniform(0, 1, g.N)


def test_clean_oracle_passes(prob):
    assert _fd_ok(*prob)


def test_sign_error_in_tv_gradient_is_caught(prob, monkeypatch):
    orig = tv.tv_grad
    monkeypatch.setattr(objective.tv, "tv_grad", lambda x, n, t: -orig(x, n, t))
    assert not _fd_ok(*prob)


def test_dropped_alpha_term_is_caught(prob, monkeypatch):
    p, x = prob
    monkeypatch.setattr(objective.Problem, "grad",
                        lambda self, x: self.A.T @ (self.A @ x - self.b))
    monkeypatch.setattr(objective.Problem, "f_and_grad",
                        lambda self, x: (self.f(x), self.A.T @ (self.A @ x - self.b)))
    assert not _fd_ok(p, x)


def test_wrong_shift_direction_in_tv_gradient_is_caught(prob, monkeypatch):
    def bad(x, n, tau):
        dx, dy, dz = tv.forward_differences(x, n)
        nrm = np.sqrt(dx * dx + dy * dy + dz * dz)
        den = np.maximum(tau, nrm)
        wx, wy, wz = dx / den, dy / den, dz / den
        g = -(wx + wy + wz)
        g[:, :, :-1] += wx[:, :, 1:]           # shifted the wrong way
        g[:, 1:, :] += wy[:, :-1, :]
        g[1:, :, :] += wz[:-1, :, :]
        return g.reshape(-1)
    monkeypatch.setattr(objective.tv, "tv_grad", bad)
    assert not _fd_ok(*prob)


def test_wrong_upn_root_is_caught():
    # the recursion-limit pin fails for the negative root
    th, q = math.sqrt(0.9), 0.01
    for _ in range(2000):
        a = th * th - q
        th = 0.5 * (-a - math.sqrt(a * a + 4 * th * th))
        if not math.isfinite(th):
            break
    assert not (abs(th - math.sqrt(q)) < 1e-10)


def test_siddon_midpoint_rule_error_would_break_chords(monkeypatch):
    # A tracer that drops the last segment no longer sums to the chord.
    cols, vals = oracle.trace_ray([-10, 0.3, 0.2], [10, 0.3, 0.2], 6)
    assert abs(vals.sum() - 6.0) < 1e-12
    assert abs(vals[:-1].sum() - 6.0) > 0.5


# ---------------------------------------------------------------- control scalars
def mutant(module, *edits):
    """A copy of `module` built from its source with each (old, new) edit
    applied; every `old` must occur exactly once."""
    src = inspect.getsource(module)
    for old, new in edits:
        assert src.count(old) == 1, old
        src = src.replace(old, new)
    name = module.__name__ + "_mutant"
    mod = types.ModuleType(name)
    mod.__package__ = module.__package__
    mod.__file__ = module.__file__
    sys.modules[name] = mod
    try:
        exec(compile(src, f"{module.__file__} (mutant)", "exec"), mod.__dict__)
    finally:
        del sys.modules[name]
    return mod


from oracle import solvers as _solvers  # noqa: E402
import test_oracle_control_pins as pins  # noqa: E402

MU_MUTANTS = {
    # sign error in M
    "sign_of_M": [("M = (fk - fy - float(gy @ d)) / dd", "M = -(fk - fy - float(gy @ d)) / dd")],
    # the pair (x^(k+1), y^(k)) in place of (x^(k), y^(k))
    "pair_xk1": [("d = xk - y ", "d = x_new - y "),
                 ("M = (fk - fy - float(gy @ d)) / dd", "M = (f_new - fy - float(gy @ d)) / dd")],
    # mu_k no longer kept non-increasing (the running minimum dropped)
    "no_running_min": [("mu = min(mu, max(M, 0.0))", "mu = max(M, 0.0)")],
    # the estimate skipped altogether
    "never_updated": [("mu = min(mu, max(M, 0.0))", "pass")],
}

GPBB_MUTANTS = {
    # nu = theta_k in place of 1/theta_k
    "nu_theta": [("theta * g))) / theta", "theta * g))) * theta")],
    # the gradient map taken at the accepted point (with the old gradient)
    "norm_after_acceptance": [
        ("        gnorm = float(np.linalg.norm(x - project_Q(x - theta * g))) / theta  # nu = 1/theta_k\n",
         ""),
        ("        x, f = xbar, fbar\n",
         "        x, f = xbar, fbar\n"
         "        gnorm = float(np.linalg.norm(x - project_Q(x - theta * g))) / theta\n"),
        ("        if k == 0:\n            gnorm0 = gnorm\n        fbar = c.f(xbar)\n",
         "        fbar = c.f(xbar)\n"),
        ("        fhist.append(f)\n",
         "        fhist.append(f)\n        if k == 0:\n            gnorm0 = gnorm\n"),
    ],
}

BB_MUTANTS = {
    # the BB quotient inverted
    "bb_inverted": [("theta = ss / sy", "theta = sy / ss")],
    # s and y taken with the wrong iterate pair (x^(k) - x^(k-2))
    "bb_stale_s": [("s = x - x_prev", "s = x - (x_prev if k < 2 else x_prev2)"),
                   ("        x_prev, g_prev = x, g\n",
                    "        x_prev2 = x_prev if k > 0 else x\n        x_prev, g_prev = x, g\n")],
}


def test_clean_control_pins_pass():
    assert pins.check_mu_is_running_min_of_rayleigh_quotients(_solvers)
    assert pins.check_gpbb_stop_value(_solvers)
    assert pins.check_gpbb_theta_is_bb_step(_solvers)


@pytest.mark.parametrize("name", sorted(MU_MUTANTS))
def test_mu_estimate_mistake_is_caught(name):
    assert not pins.check_mu_is_running_min_of_rayleigh_quotients(mutant(_solvers, *MU_MUTANTS[name]))


@pytest.mark.parametrize("name", sorted(GPBB_MUTANTS))
def test_gpbb_stop_value_mistake_is_caught(name):
    assert not pins.check_gpbb_stop_value(mutant(_solvers, *GPBB_MUTANTS[name]))


@pytest.mark.parametrize("name", sorted(BB_MUTANTS))
def test_bb_step_mistake_is_caught(name):
    assert not pins.check_gpbb_theta_is_bb_step(mutant(_solvers, *BB_MUTANTS[name]))

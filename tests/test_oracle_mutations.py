"""Planted mistakes in the oracle (on the CPU) must be caught by its pins.

Each case monkeypatches one plausible error into the oracle and re-runs the
check that is meant to catch it; the check must now fail.
"""
import math

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

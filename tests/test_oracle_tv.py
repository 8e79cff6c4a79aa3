"""Pins of the oracle's TV_tau (eq. TV with Huber smoothing) and its gradient.

Closed forms (constant image, linear ramp, single interior cube), an explicit
triple loop over voxels, the explicit sparse D_j operator, central finite
differences and the tau -> 0 limit.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import tv


def test_constant_image_has_zero_tv():
    n = 6
    x = np.full(n ** 3, 0.37)
    assert tv.tv_value(x, n, 1e-3) == 0.0
    assert np.all(tv.tv_grad(x, n, 1e-3) == 0.0)


@pytest.mark.parametrize("c,tau", [(0.5, 1e-4), (2.0, 0.1), (0.3, 0.3)])
def test_ramp_closed_form(c, tau):
    n = 5
    ix = np.tile(np.arange(n), n * n).astype(float)
    x = c * ix
    expect = n * n * (n - 1) * (c - tau / 2)
    assert abs(tv.tv_value(x, n, tau) - expect) <= 1e-12 * expect


def test_ramp_in_quadratic_zone():
    n, c, tau = 4, 1e-3, 1e-1
    x = c * np.tile(np.arange(n), n * n).astype(float)
    expect = n * n * (n - 1) * c * c / (2 * tau)
    assert abs(tv.tv_value(x, n, tau) - expect) <= 1e-12 * expect


@pytest.mark.parametrize("s,a", [(1, 1), (2, 2), (3, 1), (4, 2)])
def test_single_cube_closed_form(s, a):
    n, c, tau = 8, 0.8, 1e-3
    v = np.zeros((n, n, n))
    v[a:a + s, a:a + s, a:a + s] = c
    expect = (c * (3 * s * s + 3 * (s - 1) ** 2 + 3 * math.sqrt(2) * (s - 1) + math.sqrt(3))
              - 0.5 * tau * (3 * s * s + 3 * (s - 1) ** 2 + 3 * (s - 1) + 1))
    assert abs(tv.tv_value(v.reshape(-1), n, tau) - expect) <= 1e-12 * expect


def _loop_tv(x, n, tau):
    v = x.reshape(n, n, n)
    total = 0.0
    for iz in range(n):
        for iy in range(n):
            for ix in range(n):
                c = v[iz, iy, ix]
                gx = v[iz, iy, ix + 1] - c if ix + 1 < n else 0.0
                gy = v[iz, iy + 1, ix] - c if iy + 1 < n else 0.0
                gz = v[iz + 1, iy, ix] - c if iz + 1 < n else 0.0
                r = math.sqrt(gx * gx + gy * gy + gz * gz)
                total += r - tau / 2 if r >= tau else r * r / (2 * tau)
    return total


def _difference_operator(n):
    """Sparse D (3N x N): rows 3j+e hold component e of D_j x."""
    rows, cols, vals = [], [], []
    for iz in range(n):
        for iy in range(n):
            for ix in range(n):
                j = ix + n * iy + n * n * iz
                for e, (dx, dy, dz) in enumerate([(1, 0, 0), (0, 1, 0), (0, 0, 1)]):
                    jx, jy, jz = ix + dx, iy + dy, iz + dz
                    if jx < n and jy < n and jz < n:
                        k = jx + n * jy + n * n * jz
                        rows += [3 * j + e, 3 * j + e]
                        cols += [k, j]
                        vals += [1.0, -1.0]
    return sp.csr_matrix((vals, (rows, cols)), shape=(3 * n ** 3, n ** 3))


@pytest.mark.parametrize("n", [2, 3, 4])
def test_value_matches_explicit_loop(n):
    rng = np.random.default_rng(n)
    x = rng.uniform(0, 1, n ** 3)
    for tau in [1e-4, 0.2, 5.0]:
        assert abs(tv.tv_value(x, n, tau) - _loop_tv(x, n, tau)) <= 1e-12 * (1 + _loop_tv(x, n, tau))


@pytest.mark.parametrize("n", [3, 5])
def test_gradient_equals_DT_w(n):
    rng = np.random.default_rng(10 + n)
    x = rng.uniform(0, 1, n ** 3)
    D = _difference_operator(n)
    for tau in [1e-3, 0.3]:
        z = (D @ x).reshape(-1, 3)
        w = z / np.maximum(tau, np.linalg.norm(z, axis=1))[:, None]
        expect = D.T @ w.reshape(-1)
        assert np.allclose(tv.tv_grad(x, n, tau), expect, rtol=1e-13, atol=1e-13)


def test_gradient_finite_differences():
    n = 5
    rng = np.random.default_rng(5)
    x = rng.uniform(0, 1, n ** 3)
    tau = 1e-2
    g = tv.tv_grad(x, n, tau)
    h = 1e-6
    D = _difference_operator(n)
    # avoid the Huber kink: skip coordinates whose stencils sit near ||z|| = tau
    nz = np.linalg.norm((D @ x).reshape(-1, 3), axis=1)
    for j in rng.choice(n ** 3, 40, replace=False):
        near = D[:, j].nonzero()[0] // 3
        if np.any(np.abs(nz[near] - tau) < 10 * h):
            continue
        e = np.zeros_like(x)
        e[j] = h
        fd = (tv.tv_value(x + e, n, tau) - tv.tv_value(x - e, n, tau)) / (2 * h)
        assert abs(fd - g[j]) <= 1e-6 * (1 + abs(g[j]))


def test_tau_to_zero_recovers_plain_tv():
    n = 4
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 1, n ** 3)
    plain = tv.tv_plain(x, n)
    for tau in [1e-2, 1e-4, 1e-6]:
        assert 0 <= plain - tv.tv_value(x, n, tau) <= n ** 3 * tau / 2 + 1e-12


def test_huber_is_continuous_at_tau():
    tau = 0.25
    r = np.array([tau * (1 - 1e-12), tau, tau * (1 + 1e-12)])
    h = tv.huber(r, tau)
    assert np.allclose(h, tau / 2, rtol=1e-10)

"""Pins of the oracle's objective and of GP / GPBB (Alg. 1) / BT (Alg. 2) / UPN (Alg. 3).

Fixed points: closed-form minimisers of diagonal quadratics on Q, exact
recovery of a noise-free overdetermined 4^3 problem, agreement with scipy's
L-BFGS-B on a 4^3 TV problem, the KKT / gradient-map optimality condition
(Sec. III-D), the UPN theta/beta recursion limit, and the invariants the
algorithms guarantee by construction (BT inequality, non-increasing mu_k,
GPBB's nonmonotone acceptance rule).
"""
import math

import numpy as np
import pytest
import scipy.optimize as so
import scipy.sparse as sp

import oracle
from oracle import tv
from conftest import small_geometry

SOLVERS = [oracle.solve_gp, oracle.solve_gpbb, oracle.solve_upn]


def diag_problem(n=3, seed=0, alpha=0.0, tau=1e-2):
    rng = np.random.default_rng(seed)
    N = n ** 3
    a = rng.uniform(0.5, 3.0, N)
    c = rng.uniform(-1.0, 1.0, N)
    A = sp.csr_matrix(sp.diags(a))
    return oracle.Problem(A=A, b=a * c, n=n, alpha=alpha, tau=tau), c


@pytest.mark.parametrize("solver", SOLVERS)
def test_diagonal_quadratic_interior(solver):
    # c > 0: x* = c and phi* = 0, so the FP64 line-search tests stay resolvable
    prob, c = diag_problem()
    c = np.abs(c) + 0.1
    prob.b = prob.A @ c
    res = solver(prob, np.zeros(prob.N), 1e-13, oracle.Options(stop="per_n", k_max=20000))
    assert res.status == oracle.OK
    assert np.allclose(res.x, c, atol=1e-11)


@pytest.mark.parametrize("solver", SOLVERS)
def test_diagonal_quadratic_with_active_bounds(solver):
    # x* = max(c, 0); phi* > 0 limits how far the literal FP64 tests resolve
    # f differences (about 1e-16 phi), hence the moderate tolerance.
    prob, c = diag_problem()
    res = solver(prob, np.zeros(prob.N), 1e-8, oracle.Options(stop="per_n", k_max=20000))
    assert res.status == oracle.OK
    assert np.allclose(res.x, np.maximum(c, 0.0), atol=1e-6)


def test_gpbb_bb_step_is_inverse_curvature_on_scaled_identity():
    n = 2
    N = n ** 3
    lam = 4.0
    A = sp.csr_matrix(sp.identity(N) * math.sqrt(lam))
    c = np.linspace(0.1, 0.8, N)
    prob = oracle.Problem(A=A, b=A @ c, n=n, alpha=0.0, tau=1e-2)
    res = oracle.solve_gpbb(prob, np.zeros(N), 1e-14, oracle.Options(stop="per_n", record=True))
    # theta_k = ||s||^2 / <s, H s> = 1/lam from k = 1 on
    assert abs(res.history[1]["theta"] - 1.0 / lam) < 1e-14
    assert np.allclose(res.x, c, atol=1e-12)


def test_objective_gradient_finite_differences():
    g = small_geometry(n=4, views=6, det=6)
    A = oracle.system_matrix(g)
    rng = np.random.default_rng(2)
    b = A @ rng.uniform(0, 1, g.N)
    prob = oracle.Problem(A=A, b=b, n=4, alpha=0.3, tau=0.05)
    x = rng.uniform(0, 1, g.N)
    f, gr = prob.f_and_grad(x)
    assert f == pytest.approx(prob.f(x), rel=1e-15)
    h = 1e-6
    for j in range(0, g.N, 5):
        e = np.zeros(g.N)
        e[j] = h
        fd = (prob.f(x + e) - prob.f(x - e)) / (2 * h)
        assert abs(fd - gr[j]) <= 1e-5 * (1 + abs(gr[j]))


def test_alpha_zero_gradient_equals_dense_normal_equations():
    g = small_geometry(n=4, views=5, det=5)
    A = oracle.system_matrix(g)
    Ad = A.toarray()
    rng = np.random.default_rng(4)
    b = rng.uniform(0, 3, g.m)
    x = rng.uniform(0, 1, g.N)
    prob = oracle.Problem(A=A, b=b, n=4, alpha=0.0, tau=0.1)
    assert np.allclose(prob.grad(x), Ad.T @ Ad @ x - Ad.T @ b, rtol=1e-12, atol=1e-10)


def test_projection_and_gradient_map():
    rng = np.random.default_rng(0)
    x = rng.normal(size=100)
    p = oracle.project_Q(x)
    assert np.all(p >= 0) and np.array_equal(oracle.project_Q(p), p)
    # G_nu vanishes exactly at a KKT point of a separable quadratic
    c = rng.normal(size=100)
    xs = np.maximum(c, 0)
    gs = xs - c                       # grad of 1/2 ||x - c||^2
    for nu in [0.1, 1.0, 10.0]:
        assert np.allclose(oracle.gradient_map(xs, gs, nu), 0.0, atol=1e-15)
        assert np.linalg.norm(oracle.gradient_map(xs + 0.1, xs + 0.1 - c, nu)) > 0


def test_noise_free_overdetermined_recovery():
    g = small_geometry(n=4, views=8, det=6)
    A = oracle.system_matrix(g)
    assert np.linalg.matrix_rank(A.toarray()) == g.N
    rng = np.random.default_rng(8)
    x_true = rng.uniform(0.2, 1.0, g.N)
    prob = oracle.Problem(A=A, b=A @ x_true, n=4, alpha=0.0, tau=1e-2)
    for solver in SOLVERS:
        res = solver(prob, np.zeros(g.N), 1e-11, oracle.Options(stop="rel", k_max=200000))
        assert res.status == oracle.OK
        assert np.linalg.norm(res.x - x_true) <= 1e-6 * np.linalg.norm(x_true), solver.__name__


@pytest.fixture(scope="module")
def tv4():
    g = small_geometry(n=4, views=3, det=5)       # m = 75 rays, N = 64: few-view-like
    A = oracle.system_matrix(g)
    rng = np.random.default_rng(12)
    x_true = np.zeros(64)
    x_true[rng.choice(64, 20, replace=False)] = rng.uniform(0.3, 1.0, 20)
    b = A @ x_true + 0.01 * rng.normal(size=g.m)
    prob = oracle.Problem(A=A, b=b, n=4, alpha=0.05, tau=1e-2)
    ref = so.minimize(lambda x: prob.f_and_grad(x), np.zeros(64), jac=True, method="L-BFGS-B",
                      bounds=[(0, None)] * 64,
                      options=dict(maxiter=100000, ftol=1e-16, gtol=1e-13, maxcor=50))
    return prob, ref.x


@pytest.mark.parametrize("solver", SOLVERS)
def test_agrees_with_lbfgsb_on_4cubed_tv(tv4, solver):
    prob, xref = tv4
    res = solver(prob, np.zeros(64), 1e-10, oracle.Options(stop="rel", k_max=500000))
    assert res.status == oracle.OK
    assert prob.f(res.x) <= prob.f(xref) + 1e-9 * abs(prob.f(xref))
    assert np.linalg.norm(res.x - xref) <= 1e-4 * np.linalg.norm(xref)


@pytest.mark.parametrize("solver", SOLVERS)
def test_kkt_at_returned_point(tv4, solver):
    prob, _ = tv4
    res = solver(prob, np.zeros(64), 1e-9, oracle.Options(stop="rel", k_max=500000))
    g = prob.grad(res.x)
    scale = np.linalg.norm(prob.grad(np.zeros(64)))
    tol = 1e-7 * scale
    pos = res.x > 0
    assert np.all(np.abs(g[pos]) <= tol)
    assert np.all(g[~pos] >= -tol)
    assert np.linalg.norm(oracle.gradient_map(res.x, g, 1.0)) <= tol * 8


def test_upn_recursion_limit():
    # fixed q: theta -> sqrt(q), beta -> (1 - sqrt q) / (1 + sqrt q)
    for q in [1e-4, 0.01, 0.3]:
        th = math.sqrt(0.9)
        for _ in range(20000):
            tn = oracle.upn_theta_next(th, q)
            beta = th * (1 - th) / (th * th + tn)
            th = tn
        assert abs(th - math.sqrt(q)) < 1e-10
        assert abs(beta - (1 - math.sqrt(q)) / (1 + math.sqrt(q))) < 1e-9
    # the root satisfies the defining equation
    for th in [0.9, 0.3, 0.01]:
        for q in [0.0, 1e-3, 0.5]:
            t = oracle.upn_theta_next(th, q)
            assert t > 0 and abs(t * t - ((1 - t) * th * th + q * t)) < 1e-15


def test_invariants_on_c32(c32_problem):
    cfg, prob, geom, x_true = c32_problem
    x0 = np.zeros(prob.N)
    opts = oracle.Options(record=True, k_max=400)
    # UPN: mu_k non-increasing; BT's L bounded by rho (||A||^2 + 12 alpha / tau)
    r = oracle.solve_upn(prob, x0, 1e-4, opts)
    mus = [h["mu"] for h in r.history]
    assert all(b <= a for a, b in zip(mus, mus[1:]))
    Ls = [h["L"] for h in r.history]
    assert all(b >= a for a, b in zip(Ls, Ls[1:]))
    normA2 = so_norm2(prob.A)
    assert Ls[-1] <= 2.0 * (normA2 + 12 * prob.alpha / prob.tau)
    # GPBB: f(x(k+1)) < max of the last K+1 values (nonmonotone rule)
    r = oracle.solve_gpbb(prob, x0, 1e-4, opts)
    fs = [prob.f(x0)] + [h["f"] for h in r.history]
    for k in range(1, len(fs)):
        assert fs[k] < max(fs[max(0, k - 3):k])
    # GP: monotone decrease
    r = oracle.solve_gp(prob, x0, 1e-3, opts)
    fs = [h["f"] for h in r.history]
    assert all(b <= a for a, b in zip(fs, fs[1:]))


def so_norm2(A):
    import scipy.sparse.linalg as sla
    return float(sla.svds(A, k=1, return_singular_vectors=False)[0]) ** 2


@pytest.mark.slow
def test_upn_beats_gp_on_few_view(c32_problem):
    cfg, prob, geom, x_true = c32_problem
    x0 = np.zeros(prob.N)
    up = oracle.solve_upn(prob, x0, 1e-5, oracle.Options(k_max=20000))
    gp = oracle.solve_gp(prob, x0, 1e-5, oracle.Options(k_max=20000))
    assert up.status == oracle.OK
    assert up.iters < gp.iters

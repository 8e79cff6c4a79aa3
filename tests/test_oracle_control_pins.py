"""Pins of the oracle's control scalars against quantities computed from A
directly, independently of the solver's own arithmetic.

  * UPN's strong-convexity estimate (eq. mu_k_estimate, Alg. 3).  With
    alpha = 0, phi is the quadratic 1/2||Ax - b||^2, so
        M(x, y) = (phi(x) - phi(y) - grad phi(y)^T (x - y)) / (1/2||x - y||^2)
    is exactly the Rayleigh quotient ||A(x - y)||^2 / ||x - y||^2 of A^T A.
    Each recorded mu_k must equal min(mubar, min over j <= k of that quotient
    at the pair (x^(j), y^(j))), and lie in [lambda_min, lambda_max] of A^T A
    once it has been updated.
  * GPBB's stopping value (Sec. III-D with nu = 1/theta_k): the recorded
    ||G|| must equal ||G_{1/theta_k}(x^(k))|| recomputed by the pinned
    gradient_map from the recorded iterate and a fresh gradient there.
  * GPBB's BB step (Alg. 1): theta_k = ||s||^2 / <s, y> with s = x^(k) -
    x^(k-1), y = grad f(x^(k)) - grad f(x^(k-1)), or theta_{k-1} when
    <s, y> <= 0.

Each check takes the solver module as an argument, so that
test_oracle_mutations.py can run it against copies of the oracle with one
planted mistake and see it fail.
"""
import numpy as np

import oracle
from oracle import solvers as oracle_solvers
from conftest import small_geometry


def quadratic_case():
    """4^3, 8 views of 6^2 (A^T A has full rank), alpha = 0, about half the
    true voxels at zero so that the bound Q is active and the Rayleigh
    quotients along the iterates are not monotone."""
    g = small_geometry(n=4, views=8, det=6)
    A = oracle.system_matrix(g)
    Ad = A.toarray()
    ev = np.linalg.eigvalsh(Ad.T @ Ad)
    rng = np.random.default_rng(3)
    x_true = np.where(rng.uniform(size=g.N) < 0.5, 0.0, rng.uniform(0.2, 1.0, g.N))
    b = A @ x_true + 0.05 * rng.normal(size=g.m)
    prob = oracle.Problem(A=A, b=b, n=4, alpha=0.0, tau=1e-2)
    # Lbar above lambda_max (BT never raises L), mubar between lambda_max and
    # Lbar (the first quotient lowers it)
    opts = oracle.Options(record=True, record_iterates=True, L_bar=2.0 * ev[-1],
                          mu_bar=1.5 * ev[-1], stop="rel", k_max=60)
    return prob, Ad, ev, opts


def check_mu_is_running_min_of_rayleigh_quotients(solvers) -> bool:
    prob, Ad, ev, opts = quadratic_case()
    r = solvers.solve_upn(prob, np.zeros(prob.N), 1e-12, opts)
    if len(r.history) < 40:
        return False
    mu = opts.mu_bar
    updates = 0
    rq_rises = 0
    last_rq = None
    for h in r.history[1:]:
        d = h["x"] - h["y"]
        dd = float(d @ d)
        if 0.5 * dd > 1e-300:
            rq = float(np.linalg.norm(Ad @ d) ** 2) / dd
            if last_rq is not None and rq > last_rq:
                rq_rises += 1
            last_rq = rq
            mu = min(mu, rq)
            updates += 1
        if not abs(h["mu"] - mu) <= 1e-8 * mu:
            return False
        if updates and not (ev[0] * (1 - 1e-10) <= h["mu"] <= ev[-1] * (1 + 1e-10)):
            return False
    # the case must exercise both branches of the running minimum
    assert updates >= 30 and rq_rises >= 1
    return True


def tv_case():
    g = small_geometry(n=4, views=3, det=5)
    A = oracle.system_matrix(g)
    rng = np.random.default_rng(12)
    x_true = np.zeros(64)
    x_true[rng.choice(64, 20, replace=False)] = rng.uniform(0.3, 1.0, 20)
    b = A @ x_true + 0.01 * rng.normal(size=g.m)
    return oracle.Problem(A=A, b=b, n=4, alpha=0.05, tau=1e-2)


def check_gpbb_stop_value(solvers) -> bool:
    prob = tv_case()
    opts = oracle.Options(record=True, record_iterates=True, k_max=80)
    r = solvers.solve_gpbb(prob, np.zeros(prob.N), 1e-12, opts)
    if len(r.history) < 40:
        return False
    for h in r.history:
        g = prob.grad(h["x"])                      # a fresh gradient at the recorded x^(k)
        G = oracle.gradient_map(h["x"], g, 1.0 / h["theta"])
        if not abs(h["gnorm"] - float(np.linalg.norm(G))) <= 1e-12 * h["gnorm"]:
            return False
    return True


def check_gpbb_theta_is_bb_step(solvers) -> bool:
    prob = tv_case()
    opts = oracle.Options(record=True, record_iterates=True, k_max=80)
    r = solvers.solve_gpbb(prob, np.zeros(prob.N), 1e-12, opts)
    h = r.history
    if len(h) < 40 or h[0]["theta"] != 1.0:    # theta_0 = 1
        return False
    for k in range(1, len(h)):
        s = h[k]["x"] - h[k - 1]["x"]
        y = prob.grad(h[k]["x"]) - prob.grad(h[k - 1]["x"])
        sy, ss = float(s @ y), float(s @ s)
        want = ss / sy if (sy > 0 and ss > 0) else h[k - 1]["theta"]
        if not abs(h[k]["theta"] - want) <= 1e-9 * want:
            return False
    return True


def test_upn_mu_is_the_running_min_of_rayleigh_quotients():
    assert check_mu_is_running_min_of_rayleigh_quotients(oracle_solvers)


def test_gpbb_stop_value_is_the_gradient_map_at_inverse_theta():
    assert check_gpbb_stop_value(oracle_solvers)


def test_gpbb_theta_is_the_bb_step():
    assert check_gpbb_theta_is_bb_step(oracle_solvers)


def test_mu_pair_literal_reading_at_first_iteration():
    """At k = 1, y^(1) = x^(1): the pair of the estimate has zero distance,
    the estimate is skipped and mu_1 = mubar (the reading of Alg. 3 where the
    printed formula is 0/0)."""
    prob, Ad, ev, opts = quadratic_case()
    r = oracle.solve_upn(prob, np.zeros(prob.N), 1e-12, opts)
    h1 = r.history[1]
    assert np.array_equal(h1["x"], h1["y"]) and h1["mu"] == opts.mu_bar

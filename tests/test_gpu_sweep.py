"""alpha sweep (batching pattern): up to 8 solves sharing every read of A.

Each column must reproduce the single solve with its alpha (the sweep runs
the same arithmetic per column) and match the FP64 oracle at equal eps.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import cuda, dev_f32, oracle_spread, rel_l2

pytestmark = pytest.mark.gpu

ALPHAS = [1e-3, 1e-2, 3e-2, 1e-1]


@pytest.fixture(scope="module")
def c32():
    torch = cuda()
    from paper_1105_4002_gb300 import System
    cfg = synth.get_config("c32")
    prob, geom, _ = oracle.problem_from_config(cfg)
    return torch, System(geom), prob, cfg


@pytest.mark.parametrize("method", ["upn", "gp", "gpbb"])
def test_sweep_columns_equal_single_solves(c32, method):
    """With the single solves' row split (4 lanes) a column runs exactly their
    arithmetic."""
    torch, s, prob, cfg = c32
    from paper_1105_4002_gb300 import SolveOptions
    X = torch.zeros(len(ALPHAS) * prob.N, device="cuda")
    b = dev_f32(torch, prob.b)
    res = s.solve_sweep(method, b, ALPHAS, prob.tau, cfg.eps, X, SolveOptions(sweep_lanes=4))
    Xh = X.cpu().numpy().reshape(len(ALPHAS), prob.N)
    for c, a in enumerate(ALPHAS):
        x1 = torch.zeros(prob.N, device="cuda")
        r1 = s.solve(method, b, a, prob.tau, cfg.eps, x1)
        assert res[c].status == r1.status == 0
        d = rel_l2(Xh[c], x1.cpu().numpy())
        if method == "gpbb":
            assert d <= 1e-2, (a, d)      # BB steps react to last-bit differences of the reductions
        else:
            assert d <= 1e-5, (a, d, res[c].iters, r1.iters)


def test_sweep_upn_matches_oracle(c32):
    torch, s, prob, cfg = c32
    X = torch.zeros(len(ALPHAS) * prob.N, device="cuda")
    s.solve_sweep("upn", dev_f32(torch, prob.b), ALPHAS, prob.tau, cfg.eps, X)
    Xh = X.cpu().numpy().reshape(len(ALPHAS), prob.N)
    # At eps = 1e-4 a late line-search decision (an increase of L near the
    # stop) can move the stopping iterate; the oracle's own answer moves by
    # the same amount under float32-sized perturbations of b.
    for c, a in enumerate(ALPHAS):
        p = oracle.Problem(A=prob.A, b=prob.b, n=prob.n, alpha=a, tau=prob.tau)
        ref, spread = oracle_spread(p, oracle.solve_upn, cfg.eps, draws=8)
        d = rel_l2(Xh[c], ref.x)
        assert d <= max(1e-4, 3 * spread), (a, d, spread)


def test_sweep_eight_columns_host_buffers_and_status(c32):
    torch, s, prob, cfg = c32
    from paper_1105_4002_gb300 import SolveOptions
    alphas = list(np.logspace(-4, -1, 8))
    X = np.zeros(8 * prob.N, np.float32)
    res = s.solve_sweep("upn", prob.b.astype(np.float32), alphas, prob.tau, cfg.eps, X)
    assert all(r.status == 0 for r in res)
    Xd = torch.zeros(8 * prob.N, device="cuda")
    s.solve_sweep("upn", dev_f32(torch, prob.b), alphas, prob.tau, cfg.eps, Xd)
    assert np.array_equal(Xd.cpu().numpy(), X)
    # k_max reached on some columns
    X2 = torch.zeros(2 * prob.N, device="cuda")
    r2 = s.solve_sweep("upn", dev_f32(torch, prob.b), [1e-2, 1e-1], prob.tau, 1e-12, X2,
                       SolveOptions(k_max=7))
    assert [r.status for r in r2] == [1, 1] and [r.iters for r in r2] == [7, 7]


def test_sweep_bf16(c32):
    torch, _, prob, cfg = c32
    from paper_1105_4002_gb300 import System
    s16 = System(cfg.geometry(), storage="bf16")
    b = dev_f32(torch, prob.b)
    X = torch.zeros(2 * prob.N, device="cuda")
    res = s16.solve_sweep("upn", b, [1e-2, 1e-1], prob.tau, cfg.eps, X)
    Xh = X.cpu().numpy().reshape(2, prob.N)
    for c, a in enumerate([1e-2, 1e-1]):
        x1 = torch.zeros(prob.N, device="cuda")
        s16.solve("upn", b, a, prob.tau, cfg.eps, x1)
        assert res[c].ok and rel_l2(Xh[c], x1.cpu().numpy()) <= 1e-5


def _single_spread(torch, s, prob, a, eps, draws=4):
    """The single solve's x* and how far it moves when b is perturbed at the
    relative size of float32 rounding (1e-6): a change in the order of the
    additions moves the stopping iterate about as much."""
    b = dev_f32(torch, prob.b)
    x1 = torch.zeros(prob.N, device="cuda")
    s.solve("upn", b, a, prob.tau, eps, x1)
    ref = x1.cpu().numpy()
    rng = np.random.default_rng(0)
    spread = 0.0
    for _ in range(draws):
        pb = dev_f32(torch, prob.b * (1 + 1e-6 * rng.standard_normal(prob.b.size)))
        s.solve("upn", pb, a, prob.tau, eps, x1.zero_())
        spread = max(spread, rel_l2(x1.cpu().numpy(), ref))
    return ref, spread


@pytest.mark.parametrize("lanes", [2, 4, 8])
def test_every_row_split_reproduces_the_single_solves(c32, lanes):
    """The row split (lanes per row / column of the sweep's projections)
    changes only the order of additions: each column stays within the single
    solve's own spread under float32-sized perturbations (4 lanes: the same
    arithmetic)."""
    torch, s, prob, cfg = c32
    from paper_1105_4002_gb300 import SolveOptions
    X = torch.zeros(len(ALPHAS) * prob.N, device="cuda")
    b = dev_f32(torch, prob.b)
    res = s.solve_sweep("upn", b, ALPHAS, prob.tau, cfg.eps, X, SolveOptions(sweep_lanes=lanes))
    assert all(r.status == 0 and r.lanes == (lanes, lanes) for r in res)
    Xh = X.cpu().numpy().reshape(len(ALPHAS), prob.N)
    for c, a in enumerate(ALPHAS):
        ref, spread = _single_spread(torch, s, prob, a, cfg.eps)
        d = rel_l2(Xh[c], ref)
        assert d <= (1e-5 if lanes == 4 else max(1e-5, 3 * spread)), (lanes, a, d, spread)


def test_autotuned_row_split_is_a_candidate_and_kept(c32):
    torch, s, prob, cfg = c32
    from paper_1105_4002_gb300 import SolveOptions, System, TVRError
    b = dev_f32(torch, prob.b)
    X = torch.zeros(2 * prob.N, device="cuda")
    r1 = s.solve_sweep("upn", b, ALPHAS[:2], prob.tau, cfg.eps, X)
    assert r1[0].lanes[0] in (2, 4, 8) and r1[0].lanes[1] in (2, 4, 8)
    # a second system of the same shape on the same GPU reuses the choice
    s2 = System(cfg.geometry())
    r2 = s2.solve_sweep("upn", b, ALPHAS[:2], prob.tau, cfg.eps, X.zero_())
    assert r2[0].lanes == r1[0].lanes
    with pytest.raises(TVRError):
        s.solve_sweep("upn", b, ALPHAS[:2], prob.tau, cfg.eps, X, SolveOptions(sweep_lanes=3))


def test_sweep_gpbb_columns_where_the_minimiser_is_determined(c32):
    """At alpha = 0.1 and 0.3, tau = 1e-2 and eps = 1e-8 the stopping point
    pins down the minimiser (the FP64 oracle's GPBB and UPN agree to 2e-5 at
    alpha = 0.1), so the sweep's GPBB columns meet 1e-4 against the single
    solves and the oracle although their BB steps see last-bit differences."""
    torch, s, prob, cfg = c32
    from paper_1105_4002_gb300 import SolveOptions
    alphas, tau, eps = [0.1, 0.3], 1e-2, 1e-8
    X = torch.zeros(len(alphas) * prob.N, device="cuda")
    b = dev_f32(torch, prob.b)
    res = s.solve_sweep("gpbb", b, alphas, tau, eps, X, SolveOptions(k_max=100000))
    Xh = X.cpu().numpy().reshape(len(alphas), prob.N)
    for c, a in enumerate(alphas):
        x1 = torch.zeros(prob.N, device="cuda")
        r1 = s.solve("gpbb", b, a, tau, eps, x1, SolveOptions(k_max=100000))
        assert res[c].status == r1.status == 0
        assert rel_l2(Xh[c], x1.cpu().numpy()) <= 1e-4, (a, res[c].iters, r1.iters)
        p = oracle.Problem(A=prob.A, b=prob.b, n=prob.n, alpha=a, tau=tau)
        ref = oracle.solve_gpbb(p, np.zeros(prob.N), eps, oracle.Options(k_max=100000))
        assert ref.status == 0 and rel_l2(Xh[c], ref.x) <= 1e-4, (a, rel_l2(Xh[c], ref.x))

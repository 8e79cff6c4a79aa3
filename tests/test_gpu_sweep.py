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
    torch, s, prob, cfg = c32
    X = torch.zeros(len(ALPHAS) * prob.N, device="cuda")
    b = dev_f32(torch, prob.b)
    res = s.solve_sweep(method, b, ALPHAS, prob.tau, cfg.eps, X)
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

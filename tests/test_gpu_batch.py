"""Batch of independent uneven problems (batching pattern): side by side on
their own streams (each relaunched as soon as its previous batch of passes
drains), each must give exactly the result of solving it alone."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import cuda, dev_f32, rel_l2

pytestmark = pytest.mark.gpu


def problems():
    out = []
    for i, (n, v, p) in enumerate([(8, 4, 12), (12, 6, 18), (16, 9, 24), (20, 5, 30), (24, 12, 36)]):
        g = synth.cone_geometry(n, v, p, 3.0 * n, 2.0 * n)
        x_true = synth.ellipsoid_phantom(n, 3, (0.1 * n, 0.3 * n), (0.2, 1.0), 5000 + i)
        A = oracle.system_matrix(g)
        b = oracle.make_data(A, x_true, synth.standard_normal(g.m, 6000 + i), 0.01)
        out.append((g, b, oracle.Problem(A=A, b=b, n=n, alpha=1e-2 * (1 + i), tau=1e-3)))
    return out


@pytest.mark.parametrize("method", ["upn", "gpbb", "gp"])
def test_batch_equals_single_solves(method):
    torch = cuda()
    from paper_1105_4002_gb300 import System, solve_batch
    probs = problems()
    systems = [System(g) for g, _, _ in probs]
    bs = [dev_f32(torch, b) for _, b, _ in probs]
    xs = [torch.zeros(g.N, device="cuda") for g, _, _ in probs]
    alphas = [p.alpha for _, _, p in probs]
    res = solve_batch(method, systems, bs, alphas, 1e-3, 1e-4, xs)
    for s, b, x, a, r in zip(systems, bs, xs, alphas, res):
        x1 = torch.zeros(s.N, device="cuda")
        r1 = s.solve(method, b, a, 1e-3, 1e-4, x1)
        assert r.status == r1.status == 0
        assert r.iters == r1.iters and torch.equal(x, x1)


def test_batch_matches_oracle_and_host_buffers():
    torch = cuda()
    from paper_1105_4002_gb300 import System, solve_batch
    probs = problems()
    systems = [System(g) for g, _, _ in probs]
    bs = [b.astype(np.float32) for _, b, _ in probs]
    xs = [np.zeros(g.N, np.float32) for g, _, _ in probs]
    res = solve_batch("upn", systems, bs, [p.alpha for _, _, p in probs], 1e-3, 1e-6, xs)
    for (g, b, p), x, r in zip(probs, xs, res):
        ref = oracle.solve_upn(p, np.zeros(g.N), 1e-6)
        assert r.ok and ref.status == 0
        assert rel_l2(x, ref.x) <= 1e-4, (g.n, rel_l2(x, ref.x), r.iters, ref.iters)


def test_batch_rejects_duplicate_systems():
    torch = cuda()
    from paper_1105_4002_gb300 import System, TVRError, solve_batch
    g, b, p = problems()[0]
    s = System(g)
    bd = dev_f32(torch, b)
    with pytest.raises(TVRError):
        solve_batch("upn", [s, s], [bd, bd], [1e-2, 1e-2], 1e-3, 1e-4,
                    [torch.zeros(g.N, device="cuda"), torch.zeros(g.N, device="cuda")])


def test_batch_u16_matches_the_unquantised_oracle():
    """16-bit fixed-point storage (2 bytes per entry, like BF16) keeps the
    batch's x* within 1e-4 of the FP64 oracle on the unquantised matrix."""
    torch = cuda()
    from paper_1105_4002_gb300 import System, solve_batch
    probs = problems()
    systems = [System(g, storage="u16") for g, _, _ in probs]
    bs = [dev_f32(torch, b) for _, b, _ in probs]
    xs = [torch.zeros(g.N, device="cuda") for g, _, _ in probs]
    res = solve_batch("upn", systems, bs, [p.alpha for _, _, p in probs], 1e-3, 1e-6, xs)
    for (g, b, p), x, r in zip(probs, xs, res):
        ref = oracle.solve_upn(p, np.zeros(g.N), 1e-6)
        assert r.ok and ref.status == 0
        assert rel_l2(x.cpu().numpy(), ref.x) <= 1e-4, (g.n, rel_l2(x.cpu().numpy(), ref.x))

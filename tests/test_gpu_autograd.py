"""phi(x; b) as a torch.autograd.Function: gradcheck in FP64 against central
finite differences, and both gradients against the FP64 oracle.

The gradcheck point keeps every ||D_j x|| at least 1e-3 away from tau, so
that h = 1e-6 differences never straddle the kink of the Huber function.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import cuda, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c8():
    torch = cuda()
    from paper_1105_4002_gb300 import System
    cfg = synth.get_config("c8")
    prob, geom, _ = oracle.problem_from_config(cfg)
    return torch, System(geom), prob


def away_from_kink(prob, seed):
    rng = np.random.default_rng(seed)
    for _ in range(100):
        x = rng.uniform(0.2, 1.0, prob.N)
        dx, dy, dz = oracle.tv.forward_differences(x, prob.n)
        nrm = np.sqrt(dx * dx + dy * dy + dz * dz)
        if np.min(np.abs(nrm - prob.tau)) > 1e-3:
            return x
    raise RuntimeError("no point away from the Huber kink")


def test_gradcheck_fp64(c8):
    torch, s, prob = c8
    from paper_1105_4002_gb300.autograd import PhiFunction
    x = torch.tensor(away_from_kink(prob, 0), dtype=torch.float64, device="cuda", requires_grad=True)
    b = torch.tensor(prob.b, dtype=torch.float64, device="cuda", requires_grad=True)
    f = lambda x_, b_: PhiFunction.apply(x_, b_, s, prob.alpha, prob.tau)
    assert torch.autograd.gradcheck(f, (x, b), eps=1e-6, atol=1e-6, rtol=1e-5)


def test_fp64_gradients_match_oracle(c8):
    torch, s, prob = c8
    from paper_1105_4002_gb300.autograd import phi
    xn = away_from_kink(prob, 1)
    x = torch.tensor(xn, dtype=torch.float64, device="cuda", requires_grad=True)
    b = torch.tensor(prob.b, dtype=torch.float64, device="cuda", requires_grad=True)
    A32 = prob.A.copy()
    A32.data = A32.data.astype(np.float32).astype(np.float64)    # the GPU stores A in FP32
    p32 = oracle.Problem(A=A32, b=prob.b, n=prob.n, alpha=prob.alpha, tau=prob.tau)
    f = phi(x, b, s, prob.alpha, prob.tau)
    (3.0 * f).backward()
    f_ref, g_ref = p32.f_and_grad(xn)
    assert abs(f.item() - f_ref) <= 1e-12 * abs(f_ref)
    assert rel_l2(x.grad.cpu().numpy(), 3.0 * g_ref) <= 1e-12
    assert rel_l2(b.grad.cpu().numpy(), -3.0 * (A32 @ xn - prob.b)) <= 1e-12


def test_fp32_gradients_match_oracle(c8):
    torch, s, prob = c8
    from paper_1105_4002_gb300.autograd import phi
    xn = away_from_kink(prob, 2).astype(np.float32).astype(np.float64)
    x = torch.tensor(xn, dtype=torch.float32, device="cuda", requires_grad=True)
    b = torch.tensor(prob.b, dtype=torch.float32, device="cuda", requires_grad=True)
    f = phi(x, b, s, prob.alpha, prob.tau)
    f.backward()
    f_ref, g_ref = prob.f_and_grad(xn)
    assert abs(f.item() - f_ref) <= 1e-6 * abs(f_ref)
    assert rel_l2(x.grad.cpu().numpy(), g_ref) <= 1e-5
    assert rel_l2(b.grad.cpu().numpy(), -(prob.A @ xn - prob.b)) <= 1e-5


def test_fp32_vjp_equals_phi_and_grad(c8):
    """The backward kernel gives exactly the gradient tvr_phi_and_grad returns."""
    torch, s, prob = c8
    from paper_1105_4002_gb300.autograd import phi
    x = torch.rand(prob.N, device="cuda", requires_grad=True)
    b = torch.tensor(prob.b, dtype=torch.float32, device="cuda")
    phi(x, b, s, prob.alpha, prob.tau).backward()
    g = torch.empty(prob.N, device="cuda")
    s.phi_and_grad(x.detach(), b, prob.alpha, prob.tau, grad=g)
    assert torch.equal(x.grad, g)


def test_large_volume_sampled_parity():
    """128^3 / 60 views / 192^2: sampled rows of A x against the oracle's
    matrix-free rows, the adjoint identity, and the TV gradient at sampled voxels."""
    torch = cuda()
    from paper_1105_4002_gb300 import System
    cfg = synth.get_config("c128")
    geom = cfg.geometry()
    s = System(geom)
    assert s.nnz > 3e8
    rng = np.random.default_rng(5)
    x = rng.uniform(0, 1, geom.N).astype(np.float32)
    y = torch.empty(geom.m, device="cuda")
    xd = torch.tensor(x, device="cuda")
    s.forward(xd, y)
    yh = y.cpu().numpy()
    for i in rng.choice(geom.m, 200, replace=False):
        cols, vals = oracle.row(geom, int(i))
        ref = float(vals.astype(np.float32).astype(np.float64) @ x[cols].astype(np.float64))
        assert abs(yh[i] - ref) <= 1e-5 * (abs(ref) + 1e-3)
    r = rng.normal(size=geom.m).astype(np.float32)
    z = torch.empty(geom.N, device="cuda")
    s.adjoint(torch.tensor(r, device="cuda"), z)
    lhs = float(yh.astype(np.float64) @ r.astype(np.float64))
    rhs = float(x.astype(np.float64) @ z.cpu().numpy().astype(np.float64))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
    # b = A x (the same kernel's output) makes the residual exactly zero, so
    # the gradient with alpha = 1 is grad TV_tau alone
    g = torch.empty(geom.N, device="cuda")
    s.phi_and_grad(xd, y, 1.0, cfg.tau, grad=g)
    gtv = g.cpu().numpy().astype(np.float64)
    ref = oracle.tv.tv_grad(x.astype(np.float64), cfg.n, cfg.tau)
    idx = rng.choice(geom.N, 2000, replace=False)
    assert np.max(np.abs(gtv[idx] - ref[idx])) <= 1e-5 * (1 + np.max(np.abs(ref)))

"""phi, grad phi, A x, A^T r, P_Q and the gradient map on the GPU vs the FP64
oracle on the same float32 inputs.

Tolerance (no figure is printed in the paper; derived from the arithmetic):
float32 products accumulated over <= ~3n entries per row/column give a
relative error of a few 1e-7 per entry, so each gradient must agree to 1e-5
relative L2 (the stated target), phi to 1e-6 relative.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import cuda, dev_f32, geometries, rel_l2

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-5
PHI_TOL = 1e-6


def inputs(prob, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, 1.0, prob.N).astype(np.float32).astype(np.float64)
    return x


@pytest.fixture(scope="module")
def c32():
    torch = cuda()
    from paper_1105_4002_gb300 import System
    cfg = synth.get_config("c32")
    prob, geom, x_true = oracle.problem_from_config(cfg)
    return torch, System(geom), prob, x_true


@pytest.mark.parametrize("alpha,tau", [(1e-2, 1e-4), (1e-1, 1e-2), (0.0, 1.0), (1.0, 1e-1)])
def test_phi_and_grad_parity(c32, alpha, tau):
    torch, s, prob, x_true = c32
    prob = oracle.Problem(A=prob.A, b=prob.b, n=prob.n, alpha=alpha, tau=tau)
    for x in [inputs(prob, 1), x_true.astype(np.float32).astype(np.float64)]:
        g = torch.empty(prob.N, device="cuda")
        r = torch.empty(prob.m if hasattr(prob, "m") else prob.A.shape[0], device="cuda")
        phi, data, tv = s.phi_and_grad(dev_f32(torch, x), dev_f32(torch, prob.b), alpha, tau,
                                       grad=g, resid=r)
        f_ref, g_ref = prob.f_and_grad(x)
        r_ref = prob.A @ x - prob.b
        assert abs(phi - f_ref) <= PHI_TOL * abs(f_ref)
        assert abs(data - 0.5 * r_ref @ r_ref) <= PHI_TOL * abs(0.5 * r_ref @ r_ref)
        assert abs(tv - oracle.tv.tv_value(x, prob.n, tau)) <= PHI_TOL * (1 + abs(tv))
        assert rel_l2(g.cpu().numpy(), g_ref) <= GRAD_TOL
        assert rel_l2(r.cpu().numpy(), r_ref) <= GRAD_TOL


def test_tv_gradient_alone_parity(c32):
    """b = A x makes the data part of grad phi vanish up to rounding; alpha = 1."""
    torch, s, prob, _ = c32
    x = inputs(prob, 7)
    tau = 1e-2
    g = torch.empty(prob.N, device="cuda")
    zero_b = np.zeros(prob.A.shape[0])
    s.phi_and_grad(dev_f32(torch, x), dev_f32(torch, zero_b), 0.0, tau, grad=g)
    g_data = g.cpu().numpy().astype(np.float64)
    s.phi_and_grad(dev_f32(torch, x), dev_f32(torch, zero_b), 1.0, tau, grad=g)
    g_tv = g.cpu().numpy().astype(np.float64) - g_data
    ref = oracle.tv.tv_grad(x, prob.n, tau)
    assert rel_l2(g_tv, ref) <= 1e-4


def test_forward_adjoint_parity_and_adjointness(c32):
    torch, s, prob, _ = c32
    rng = np.random.default_rng(3)
    x = rng.normal(size=prob.N).astype(np.float32).astype(np.float64)
    r = rng.normal(size=prob.A.shape[0]).astype(np.float32).astype(np.float64)
    y = torch.empty(prob.A.shape[0], device="cuda")
    z = torch.empty(prob.N, device="cuda")
    s.forward(dev_f32(torch, x), y)
    s.adjoint(dev_f32(torch, r), z)
    assert rel_l2(y.cpu().numpy(), prob.A @ x) <= GRAD_TOL
    assert rel_l2(z.cpu().numpy(), prob.A.T @ r) <= GRAD_TOL
    lhs = float(y.cpu().numpy().astype(np.float64) @ r)
    rhs = float(x @ z.cpu().numpy().astype(np.float64))
    assert abs(lhs - rhs) <= 1e-5 * (abs(lhs) + 1)


def test_host_buffers_equal_device_buffers(c32):
    torch, s, prob, _ = c32
    x = inputs(prob, 11).astype(np.float32)
    b = prob.b.astype(np.float32)
    gd = torch.empty(prob.N, device="cuda")
    phid = s.phi_and_grad(dev_f32(torch, x), dev_f32(torch, b), 1e-2, 1e-4, grad=gd)
    gh = np.empty(prob.N, np.float32)
    phih = s.phi_and_grad(x, b, 1e-2, 1e-4, grad=gh)
    assert phid == phih
    assert np.array_equal(gd.cpu().numpy(), gh)
    pinned = torch.tensor(x).pin_memory()
    ghp = torch.empty(prob.N).pin_memory()
    phip = s.phi_and_grad(pinned, torch.tensor(b).pin_memory(), 1e-2, 1e-4, grad=ghp)
    assert phip == phid and np.array_equal(ghp.numpy(), gh)


def test_results_are_deterministic(c32):
    torch, s, prob, _ = c32
    x = dev_f32(torch, inputs(prob, 5))
    b = dev_f32(torch, prob.b)
    g1 = torch.empty(prob.N, device="cuda")
    g2 = torch.empty(prob.N, device="cuda")
    p1 = s.phi_and_grad(x, b, 1e-2, 1e-4, grad=g1)
    p2 = s.phi_and_grad(x, b, 1e-2, 1e-4, grad=g2)
    assert p1 == p2 and torch.equal(g1, g2)


def test_phi_only_matches_phi_with_grad(c32):
    torch, s, prob, _ = c32
    x = dev_f32(torch, inputs(prob, 9))
    b = dev_f32(torch, prob.b)
    g = torch.empty(prob.N, device="cuda")
    assert s.phi_and_grad(x, b, 1e-2, 1e-4) == s.phi_and_grad(x, b, 1e-2, 1e-4, grad=g)


@pytest.mark.parametrize("name,geom", geometries(), ids=[g[0] for g in geometries()])
def test_small_and_ragged_geometries(name, geom):
    torch = cuda()
    from paper_1105_4002_gb300 import System
    A = oracle.system_matrix(geom)
    s = System(geom)
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 1, geom.N).astype(np.float32).astype(np.float64)
    b = rng.uniform(0, 2, geom.m).astype(np.float32).astype(np.float64)
    prob = oracle.Problem(A=A, b=b, n=geom.n, alpha=0.05, tau=1e-2)
    g = torch.empty(geom.N, device="cuda")
    phi, _, _ = s.phi_and_grad(dev_f32(torch, x), dev_f32(torch, b), 0.05, 1e-2, grad=g)
    f_ref, g_ref = prob.f_and_grad(x)
    assert abs(phi - f_ref) <= PHI_TOL * abs(f_ref)
    assert rel_l2(g.cpu().numpy(), g_ref) <= GRAD_TOL


def test_full_size_64cubed_sampled():
    """64^3 headline problem: full gradient vs the oracle at one point."""
    torch = cuda()
    from paper_1105_4002_gb300 import System
    cfg = synth.get_config("c64")
    prob, geom, x_true = oracle.problem_from_config(cfg)
    s = System(geom)
    x = inputs(prob, 21)
    g = torch.empty(prob.N, device="cuda")
    phi, _, _ = s.phi_and_grad(dev_f32(torch, x), dev_f32(torch, prob.b), cfg.alpha, cfg.tau, grad=g)
    f_ref, g_ref = prob.f_and_grad(x)
    assert abs(phi - f_ref) <= PHI_TOL * abs(f_ref)
    assert rel_l2(g.cpu().numpy(), g_ref) <= GRAD_TOL


def test_project_and_gradient_map(c32):
    torch, s, prob, _ = c32
    from paper_1105_4002_gb300 import project_Q
    v = torch.tensor([-1.0, 0.0, -0.0, 2.5, float("nan"), -1e-30, 3e38], device="cuda")
    project_Q(v)
    out = v.cpu().numpy()
    assert out[0] == 0 and out[3] == 2.5 and np.isnan(out[4]) and out[5] == 0 and out[6] == 3e38
    rng = np.random.default_rng(2)
    x = rng.uniform(-1, 1, prob.N).astype(np.float32)
    gr = rng.normal(size=prob.N).astype(np.float32)
    for nu in [0.1, 1.0, 37.0]:
        ref = np.linalg.norm(oracle.gradient_map(x.astype(np.float64), gr.astype(np.float64), nu))
        got = s.gradient_map_norm(dev_f32(torch, x), dev_f32(torch, gr), nu)
        assert abs(got - ref) <= 1e-5 * ref
    empty = torch.empty(0, device="cuda")
    project_Q(empty)


def test_argument_errors(c32):
    torch, s, prob, _ = c32
    from paper_1105_4002_gb300 import TVRError
    x = torch.zeros(prob.N, device="cuda")
    b = torch.zeros(prob.A.shape[0], device="cuda")
    with pytest.raises(TVRError):
        s.phi_and_grad(x, b, -1.0, 1e-4)
    with pytest.raises(TVRError):
        s.phi_and_grad(x, b, 1.0, 0.0)
    with pytest.raises(ValueError):
        s.phi_and_grad(torch.zeros(prob.N + 1, device="cuda"), b, 1.0, 1e-4)

"""BF16 storage with per-row FP32 scale (precision pattern).

q_ij = bf16(a_ij / s_i) with s_i = max_j a_ij is a quantisation: both sides
take it in float32 (the kernel's precision), so the codes must agree bit for
bit with a numpy emulation (round to nearest even on the float32 bits).  The
kernels then apply the effective matrix s_i q_ij, so phi, its gradient and the
solutions are compared with the FP64 oracle run on that same matrix; the
distance to the unquantised problem is reported by bench.py, not asserted.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import cuda, dev_f32, rel_l2

pytestmark = pytest.mark.gpu


def bf16_rne(a32):
    u = a32.astype(np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def effective(A):
    """Effective float32 values of the BF16 storage of an oracle CSR matrix."""
    v32 = A.data.astype(np.float32)
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    s = np.ones(A.shape[0], np.float32)
    np.maximum.at(s, rows, v32)          # rows are non-empty where entries exist; empty rows keep 1
    nonempty = np.diff(A.indptr) > 0
    smax = np.zeros(A.shape[0], np.float32)
    np.maximum.at(smax, rows, v32)
    s = np.where(nonempty & (smax > 0), smax, np.float32(1.0)).astype(np.float32)
    q = bf16_rne(v32 / s[rows])
    eff = (s[rows] * q).astype(np.float32)
    Ah = A.copy()
    Ah.data = eff.astype(np.float64)
    return Ah, eff


@pytest.fixture(scope="module")
def c32bf():
    torch = cuda()
    from paper_1105_4002_gb300 import System
    cfg = synth.get_config("c32")
    prob, geom, x_true = oracle.problem_from_config(cfg)
    Ah, eff = effective(prob.A)
    ph = oracle.Problem(A=Ah, b=prob.b, n=prob.n, alpha=prob.alpha, tau=prob.tau)
    return torch, System(geom, storage="bf16"), prob, ph, eff, cfg


def test_codes_bit_exact(c32bf):
    torch, s, prob, ph, eff, _ = c32bf
    rp, col, val = s.export_csr()
    assert np.array_equal(col, prob.A.indices)
    assert np.array_equal(val, eff)
    cp, row, cval = s.export_csc()
    C = ph.A.tocsc()
    assert np.array_equal(row, C.indices)
    assert np.array_equal(cval, C.data.astype(np.float32))


def test_phi_grad_and_adjoint_on_effective_matrix(c32bf):
    torch, s, prob, ph, eff, _ = c32bf
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 1, prob.N).astype(np.float32).astype(np.float64)
    g = torch.empty(prob.N, device="cuda")
    phi, _, _ = s.phi_and_grad(dev_f32(torch, x), dev_f32(torch, prob.b), prob.alpha, prob.tau, grad=g)
    f_ref, g_ref = ph.f_and_grad(x)
    assert abs(phi - f_ref) <= 1e-6 * abs(f_ref)
    assert rel_l2(g.cpu().numpy(), g_ref) <= 1e-5
    y = torch.empty(prob.A.shape[0], device="cuda")
    s.forward(dev_f32(torch, x), y)
    assert rel_l2(y.cpu().numpy(), ph.A @ x) <= 1e-5
    r = rng.normal(size=prob.A.shape[0]).astype(np.float32)
    z = torch.empty(prob.N, device="cuda")
    s.adjoint(dev_f32(torch, r), z)
    assert rel_l2(z.cpu().numpy(), ph.A.T @ r.astype(np.float64)) <= 1e-5
    # the VJP kernel applies the same (scaled) transpose
    from paper_1105_4002_gb300.autograd import phi as phi_fn
    xt = dev_f32(torch, x).requires_grad_(True)
    phi_fn(xt, dev_f32(torch, prob.b), s, prob.alpha, prob.tau).backward()
    assert rel_l2(xt.grad.cpu().numpy(), g_ref) <= 1e-5


@pytest.mark.parametrize("method", ["upn", "gp"])
def test_solution_matches_oracle_on_effective_matrix(c32bf, method):
    torch, s, prob, ph, eff, cfg = c32bf
    x = torch.zeros(prob.N, device="cuda")
    res = s.solve(method, dev_f32(torch, prob.b), prob.alpha, prob.tau, cfg.eps, x)
    fn = {"upn": oracle.solve_upn, "gp": oracle.solve_gp}[method]
    ref = fn(ph, np.zeros(prob.N), cfg.eps)
    assert res.ok and ref.status == 0
    assert rel_l2(x.cpu().numpy(), ref.x) <= 1e-4, (rel_l2(x.cpu().numpy(), ref.x), res.iters, ref.iters)


def test_bf16_close_to_fp32(c32bf):
    torch, s, prob, ph, eff, cfg = c32bf
    from paper_1105_4002_gb300 import System
    s32 = System(cfg.geometry())
    x16 = torch.zeros(prob.N, device="cuda")
    x32 = torch.zeros(prob.N, device="cuda")
    s.solve("upn", dev_f32(torch, prob.b), prob.alpha, prob.tau, 1e-5, x16)
    s32.solve("upn", dev_f32(torch, prob.b), prob.alpha, prob.tau, 1e-5, x32)
    # 2^-9 relative perturbation of each entry: the solutions differ by about that much
    assert rel_l2(x16.cpu().numpy(), x32.cpu().numpy()) <= 2e-2

"""16-bit unsigned fixed-point storage with a per-row FP32 step (precision
pattern): a_ij = t_i q_ij with t_i = fl(s_i / 65535), s_i = max_j a_ij and
q_ij = min(65535, rint(a_ij / t_i)), the same codes in CSR and CSC.

The quantisation is taken in float32 on both sides, so the codes must agree
bit for bit with a numpy emulation.  The kernels then apply the effective
matrix t_i q_ij: phi, its gradient, the adjoint and the solutions are compared
with the FP64 oracle on that matrix; and, unlike bfloat16 codes (2^-9 of each
entry), the step is small enough for x* to stay within 1e-4 of the oracle's
on the unquantised problem.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import cuda, dev_f32, rel_l2

pytestmark = pytest.mark.gpu


def effective(A):
    """Effective float32 values of the U16 storage of an oracle CSR matrix."""
    v32 = A.data.astype(np.float32)
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    smax = np.zeros(A.shape[0], np.float32)
    np.maximum.at(smax, rows, v32)
    s = np.where(smax > 0, smax, np.float32(1.0)).astype(np.float32)
    t = (s / np.float32(65535.0)).astype(np.float32)
    q = np.minimum(np.rint((v32 / t[rows]).astype(np.float32)), 65535).astype(np.float32)
    eff = (t[rows] * q).astype(np.float32)
    Ah = A.copy()
    Ah.data = eff.astype(np.float64)
    return Ah, eff


@pytest.fixture(scope="module")
def c32u():
    torch = cuda()
    from paper_1105_4002_gb300 import System
    cfg = synth.get_config("c32")
    prob, geom, x_true = oracle.problem_from_config(cfg)
    Ah, eff = effective(prob.A)
    ph = oracle.Problem(A=Ah, b=prob.b, n=prob.n, alpha=prob.alpha, tau=prob.tau)
    return torch, System(geom, storage="u16"), prob, ph, eff, cfg


def test_codes_bit_exact(c32u):
    torch, s, prob, ph, eff, _ = c32u
    rp, col, val = s.export_csr()
    assert np.array_equal(col, prob.A.indices)
    assert np.array_equal(val, eff)
    cp, row, cval = s.export_csc()
    C = ph.A.tocsc()
    assert np.array_equal(row, C.indices)
    assert np.array_equal(cval, C.data.astype(np.float32))
    # every entry within half a step (plus the float32 rounding of t q) of a_ij
    a = prob.A.data
    rows = np.repeat(np.arange(prob.A.shape[0]), np.diff(prob.A.indptr))
    smax = np.zeros(prob.A.shape[0])
    np.maximum.at(smax, rows, a)
    assert np.all(np.abs(eff - a) <= smax[rows] * (0.5 / 65535 + 1e-6))


def test_phi_grad_and_adjoint_on_effective_matrix(c32u):
    torch, s, prob, ph, eff, _ = c32u
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 1, prob.N).astype(np.float32).astype(np.float64)
    g = torch.empty(prob.N, device="cuda")
    phi, _, _ = s.phi_and_grad(dev_f32(torch, x), dev_f32(torch, prob.b), prob.alpha, prob.tau,
                               grad=g)
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


@pytest.mark.parametrize("method", ["upn", "gp"])
def test_solution_matches_oracle_on_effective_matrix(c32u, method):
    torch, s, prob, ph, eff, cfg = c32u
    x = torch.zeros(prob.N, device="cuda")
    res = s.solve(method, dev_f32(torch, prob.b), prob.alpha, prob.tau, cfg.eps, x)
    fn = {"upn": oracle.solve_upn, "gp": oracle.solve_gp}[method]
    ref = fn(ph, np.zeros(prob.N), cfg.eps)
    assert res.ok and ref.status == 0
    assert rel_l2(x.cpu().numpy(), ref.x) <= 1e-4, (rel_l2(x.cpu().numpy(), ref.x), res.iters,
                                                    ref.iters)


@pytest.mark.parametrize("method", ["upn", "gp"])
def test_solution_within_1e4_of_the_unquantised_oracle(c32u, method):
    """The accuracy target of the 16-bit storage: x* against the FP64 oracle on
    the unquantised A at equal eps."""
    torch, s, prob, ph, eff, cfg = c32u
    x = torch.zeros(prob.N, device="cuda")
    res = s.solve(method, dev_f32(torch, prob.b), prob.alpha, prob.tau, cfg.eps, x)
    fn = {"upn": oracle.solve_upn, "gp": oracle.solve_gp}[method]
    ref = fn(prob, np.zeros(prob.N), cfg.eps)
    assert res.ok and ref.status == 0
    assert rel_l2(x.cpu().numpy(), ref.x) <= 1e-4, (rel_l2(x.cpu().numpy(), ref.x), res.iters,
                                                    ref.iters)


def test_sweep_and_batch_run_on_u16(c32u):
    torch, s, prob, ph, eff, cfg = c32u
    from paper_1105_4002_gb300 import System, solve_batch
    X = torch.zeros(2 * prob.N, device="cuda")
    res = s.solve_sweep("upn", dev_f32(torch, prob.b), [prob.alpha, 3 * prob.alpha], prob.tau,
                        cfg.eps, X)
    x1 = torch.zeros(prob.N, device="cuda")
    r1 = s.solve("upn", dev_f32(torch, prob.b), prob.alpha, prob.tau, cfg.eps, x1)
    assert res[0].ok and rel_l2(X[:prob.N].cpu().numpy(), x1.cpu().numpy()) <= 1e-5
    s2 = System(cfg.geometry(), storage="u16")
    xs = [torch.zeros(prob.N, device="cuda")]
    rb = solve_batch("upn", [s2], [dev_f32(torch, prob.b)], [prob.alpha], prob.tau, cfg.eps, xs)
    assert rb[0].ok and torch.equal(xs[0], x1)

"""Matrix-free storage (no stored A): the entries are the float32 slab-method
lengths of each ray segment inside each voxel box, computed on the fly by the
forward projection (per ray) and the back projection (per voxel).

Parity: against the FP64 oracle (Siddon lengths), within the float32 rounding
of the ray geometry.  A coordinate of magnitude up to D = D_so + D_od (the
largest distance in the scan, 5n for the cone configurations) carries an
error of 2^-24 D; a plane crossing moves by that much along the ray, so an
entry's length changes by about 2^-23 D (two crossings) and a row sum by at
most twice that per unit of |x| over the phantom's edges.  For n = 32
(D = 160) that is 2e-5 of a voxel; the relative L2 error of A x is far
smaller because the crossings are shared by neighbouring voxels.  The tests
use 1e-5 relative L2 for A x and A^T y, and 2e-5 for the gradient.
Exact transposition is checked bit for bit on a dense 4^3 system.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import cuda, dev_f32, geometries, rel_l2

pytestmark = pytest.mark.gpu


def _sys(torch, geom):
    from paper_1105_4002_gb300 import System
    return System(geom, storage="mf")


def tilted_cone(n, views, det, deg=25.0):
    """A circular cone-beam scan whose orbit is tilted by `deg` about the x
    axis: the detector's row axis then has a y component, so the views are not
    separable into x-y and z parts and the back projection enumerates each
    voxel's pixels itself instead of taking the per-stack kernel's sums."""
    g = synth.cone_geometry(n, views, det, 3.0 * n, 2.0 * n)
    c, s = np.cos(np.radians(deg)), np.sin(np.radians(deg))
    R = np.array([[1.0, 0.0, 0.0], [0.0, c, -s], [0.0, s, c]])
    v = g.views.reshape(-1, 4, 3) @ R.T
    return synth.Geometry(n=g.n, det_cols=g.det_cols, det_rows=g.det_rows,
                          views=np.ascontiguousarray(v.reshape(-1, synth.VIEW_FIELDS)), kind=g.kind)


CASES = geometries() + [("tilted_cone", tilted_cone(12, 7, 19)),
                        ("odd_n_stacks", synth.cone_geometry(11, 6, 17, 33.0, 22.0))]


@pytest.mark.parametrize("name,geom", CASES, ids=[g[0] for g in CASES])
def test_forward_and_adjoint_match_the_oracle(name, geom):
    torch = cuda()
    s = _sys(torch, geom)
    A = oracle.system_matrix(geom)
    rng = np.random.default_rng(11)
    x = rng.uniform(0, 1, geom.N).astype(np.float32)
    y = torch.empty(geom.m, device="cuda")
    s.forward(dev_f32(torch, x), y)
    ref = A @ x.astype(np.float64)
    if np.linalg.norm(ref) == 0:
        assert np.all(y.cpu().numpy() == 0)
    else:
        assert rel_l2(y.cpu().numpy(), ref) <= 1e-5, name
    r = rng.normal(size=geom.m).astype(np.float32)
    z = torch.empty(geom.N, device="cuda")
    s.adjoint(dev_f32(torch, r), z)
    ref = A.T @ r.astype(np.float64)
    if np.linalg.norm(ref) == 0:
        assert np.all(z.cpu().numpy() == 0)
    else:
        assert rel_l2(z.cpu().numpy(), ref) <= 1e-5, name


@pytest.mark.parametrize("tilt", [0.0, 25.0])
def test_exact_transpose_on_a_dense_system(tilt):
    """Column j of the forward (x = e_j) equals row j of the back projection
    (r = e_i gives row i of A), bit for bit; both match the oracle's A.  On
    the untilted orbit the back projection takes the per-stack kernel's sums
    (separable views), on the tilted one its own pixel enumeration."""
    torch = cuda()
    g = tilted_cone(4, 3, 5, tilt)
    s = _sys(torch, g)
    Mf = np.zeros((g.m, g.N), np.float32)
    Mb = np.zeros((g.m, g.N), np.float32)
    y = torch.empty(g.m, device="cuda")
    for j in range(g.N):
        e = torch.zeros(g.N, device="cuda")
        e[j] = 1.0
        s.forward(e, y)
        Mf[:, j] = y.cpu().numpy()
    z = torch.empty(g.N, device="cuda")
    for i in range(g.m):
        e = torch.zeros(g.m, device="cuda")
        e[i] = 1.0
        s.adjoint(e, z)
        Mb[i, :] = z.cpu().numpy()
    assert np.array_equal(Mf, Mb)
    A = oracle.system_matrix(g).toarray()
    assert np.max(np.abs(Mf - A)) <= 1e-5 * np.max(A)
    # the index sets agree except for slivers below the float32 geometry error
    assert np.all(((Mf > 0) == (A > 0)) | (np.maximum(Mf, A) < 1e-4))


def test_phi_and_gradient_match_the_oracle():
    torch = cuda()
    cfg = synth.get_config("c32")
    prob, geom, _ = oracle.problem_from_config(cfg)
    s = _sys(torch, geom)
    x = np.random.default_rng(3).uniform(0, 1, prob.N).astype(np.float32).astype(np.float64)
    g = torch.empty(prob.N, device="cuda")
    phi, _, _ = s.phi_and_grad(dev_f32(torch, x), dev_f32(torch, prob.b), prob.alpha, prob.tau,
                               grad=g)
    f_ref, g_ref = prob.f_and_grad(x)
    assert abs(phi - f_ref) <= 2e-5 * abs(f_ref)
    assert rel_l2(g.cpu().numpy(), g_ref) <= 2e-5


@pytest.mark.parametrize("method", ["gp", "gpbb", "upn"])
def test_solve_matches_the_oracle(method):
    """x* of the matrix-free solve against the oracle's at equal eps, within
    the oracle's own spread under perturbations of b at the size of the
    float32 entry error (1e-5 relative), or 1e-3."""
    torch = cuda()
    from paper_1105_4002_gb300 import SolveOptions
    solver = {"gp": oracle.solve_gp, "gpbb": oracle.solve_gpbb, "upn": oracle.solve_upn}[method]
    cfg = synth.get_config("c32")
    prob, geom, _ = oracle.problem_from_config(cfg)
    s = _sys(torch, geom)
    x = torch.zeros(prob.N, device="cuda")
    res = s.solve(method, dev_f32(torch, prob.b), prob.alpha, prob.tau, cfg.eps, x, SolveOptions())
    assert res.ok
    ref = solver(prob, np.zeros(prob.N), cfg.eps)
    d = rel_l2(x.cpu().numpy(), ref.x)
    if d > 1e-3:
        rng = np.random.default_rng(0)
        spread = 0.0
        for _ in range(2):
            pb = prob.b * (1 + 1e-5 * rng.standard_normal(prob.b.size))
            p2 = oracle.Problem(A=prob.A, b=pb, n=prob.n, alpha=prob.alpha, tau=prob.tau)
            spread = max(spread, rel_l2(solver(p2, np.zeros(prob.N), cfg.eps).x, ref.x))
        assert d <= 3 * spread, (d, spread)


@pytest.mark.parametrize("tilt", [0.0, 25.0])
def test_trial_sums_match_the_oracle(tilt):
    """One projected trial step (the solvers' trial kernel, tvr_trial_sums):
    ||A xbar - b||^2 and ||A d||^2 against the oracle's FP64 A, within the
    float32 geometry bound of the entries (about 1e-5 of each row's sum of
    |a_ij x_j|; A d cancels, so 1e-3 on the squared sums).  Untilted, the row sums come from the
    per-stack forward kernel (separable views); tilted, from the walk of each
    ray."""
    torch = cuda()
    g = tilted_cone(16, 9, 24, tilt)
    s = _sys(torch, g)
    A = oracle.system_matrix(g)
    rng = np.random.default_rng(5)
    p = rng.uniform(0, 1, g.N).astype(np.float32)
    gr = rng.normal(size=g.N).astype(np.float32)
    b = (A @ p.astype(np.float64)).astype(np.float32) * np.float32(0.5)
    step = 0.1
    xb = torch.empty(g.N, device="cuda")
    sums = s.trial_sums(dev_f32(torch, p), dev_f32(torch, gr), dev_f32(torch, b), step, 1e-2,
                        xbar=xb)
    x64 = xb.cpu().numpy().astype(np.float64)
    assert np.array_equal(xb.cpu().numpy(), np.maximum(p - np.float32(step) * gr, np.float32(0)))
    r = A @ x64 - b
    Ad = A @ (x64 - p)
    assert sums[0] == pytest.approx(float(r @ r), rel=1e-3)
    assert sums[1] == pytest.approx(float(Ad @ Ad), rel=1e-3)


def test_autograd_on_matrix_free_storage():
    """phi through torch.autograd on a matrix-free system (FP32): the backward
    gives exactly tvr_phi_and_grad's gradient, and both gradients agree with
    the oracle within the float32 geometry bound."""
    torch = cuda()
    from paper_1105_4002_gb300.autograd import phi
    cfg = synth.get_config("c32")
    prob, geom, _ = oracle.problem_from_config(cfg)
    s = _sys(torch, geom)
    xn = np.random.default_rng(7).uniform(0, 1, prob.N).astype(np.float32)
    x = torch.tensor(xn, device="cuda", requires_grad=True)
    b = torch.tensor(prob.b, dtype=torch.float32, device="cuda", requires_grad=True)
    f = phi(x, b, s, prob.alpha, prob.tau)
    f.backward()
    g = torch.empty(prob.N, device="cuda")
    value, _, _ = s.phi_and_grad(x.detach(), b.detach(), prob.alpha, prob.tau, grad=g)
    assert torch.equal(x.grad, g)
    assert f.item() == pytest.approx(value, rel=1e-6)
    f_ref, g_ref = prob.f_and_grad(xn.astype(np.float64))
    assert abs(f.item() - f_ref) <= 2e-5 * abs(f_ref)
    assert rel_l2(x.grad.cpu().numpy(), g_ref) <= 2e-5
    assert rel_l2(b.grad.cpu().numpy(), -(prob.A @ xn.astype(np.float64) - prob.b)) <= 2e-5


def test_matrix_free_rejections():
    torch = cuda()
    from paper_1105_4002_gb300._capi import TVRError as TvrError
    g = synth.get_config("c8").geometry()
    s = _sys(torch, g)
    assert s.nnz == 0
    with pytest.raises(TvrError):
        s.export_csr()
    with pytest.raises(TvrError):
        s.export_csc()
    x = torch.zeros(g.N, dtype=torch.float64, device="cuda")
    b = torch.zeros(g.m, dtype=torch.float64, device="cuda")
    from paper_1105_4002_gb300.autograd import phi
    with pytest.raises(TvrError):
        phi(x, b, s, 1e-2, 1e-2)

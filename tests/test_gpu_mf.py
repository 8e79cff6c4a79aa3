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


@pytest.mark.parametrize("name,geom", geometries(), ids=[g[0] for g in geometries()])
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


def test_exact_transpose_on_a_dense_system():
    """Column j of the forward (x = e_j) equals row j of the back projection
    (r = e_i gives row i of A), bit for bit; both match the oracle's A."""
    torch = cuda()
    from conftest import small_geometry
    g = small_geometry(n=4, views=3, det=5)
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


@pytest.mark.parametrize("method", ["gp", "upn"])
def test_solve_matches_the_oracle(method):
    """x* of the matrix-free solve against the oracle's at equal eps, within
    the oracle's own spread under perturbations of b at the size of the
    float32 entry error (1e-5 relative), or 1e-3."""
    torch = cuda()
    from paper_1105_4002_gb300 import SolveOptions
    solver = {"gp": oracle.solve_gp, "upn": oracle.solve_upn}[method]
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

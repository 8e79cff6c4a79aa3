"""Shared helpers of the GPU parity tests (inputs come from synth, expected
values from the oracle; nothing here computes the method)."""
import numpy as np
import pytest

import oracle
import synth


def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def dev_f32(torch, a):
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def geometries():
    """(name, geometry) cases spanning tiles, ragged tails and degenerate scans."""
    out = []
    for name in ["c8", "c32"]:
        out.append((name, synth.get_config(name).geometry()))
    out.append(("odd_det", synth.cone_geometry(7, 5, 11, 21.0, 14.0, det_rows=9)))
    out.append(("n1", synth.cone_geometry(1, 3, 3, 3.0, 2.0)))
    out.append(("one_view_one_pixel", synth.cone_geometry(5, 1, 1, 15.0, 10.0)))
    out.append(("wide_det_misses", synth.cone_geometry(6, 4, 40, 18.0, 12.0, det_rows=3)))
    dirs = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 0], [1, 1, 1], [0.3, -0.7, 0.2]])
    out.append(("parallel_axes_diag", synth.parallel_geometry(6, dirs, 9)))
    # the paper's scan shape at small size: 19 directions spread over the sphere
    out.append(("sphere19", synth.sphere_parallel_geometry(8, 19, 13)))
    return out


def oracle_spread(prob, solver, eps, draws=4, seed=0):
    """How far the oracle's own answer moves when b is perturbed at the
    relative size of float32 gradient error (1e-6): the largest relative L2
    distance over `draws` seeded perturbations, and the solution itself."""
    ref = solver(prob, np.zeros(prob.N), eps)
    rng = np.random.default_rng(seed)
    spread = 0.0
    for _ in range(draws):
        pb = prob.b * (1 + 1e-6 * rng.standard_normal(prob.b.size))
        p2 = oracle.Problem(A=prob.A, b=pb, n=prob.n, alpha=prob.alpha, tau=prob.tau)
        spread = max(spread, rel_l2(solver(p2, np.zeros(prob.N), eps).x, ref.x))
    return ref, spread

"""The qualitative result of the paper's Sec. IV-B on a small scan of its
shape, in the FP64 oracle: parallel beam with view directions spread over the
unit sphere, fewer rays than voxels (few-view), Gaussian noise of relative
size exactly 0.01, alpha = 0.01.  UPN reaches the tolerance within 2000
iterations, GP does not (the paper: GP does not reach the accuracy within the
plotted 2000 iterations; UPN does); GPBB needs fewer iterations than GP and
more than UPN on this few-view scan (the paper: GPBB reaches the accuracy only
in the many-view case)."""
import numpy as np

import oracle
import synth


def sphere_few_view_problem(n=12, views=3, det=21, seed=77):
    g = synth.sphere_parallel_geometry(n, views, det)
    A = oracle.system_matrix(g)
    x_true = synth.ellipsoid_phantom(n, 4, (1.0, n / 3.0), (0.2, 1.0), seed)
    ax = A @ x_true
    e = synth.noise_exact(ax, synth.standard_normal(g.m, seed + 1), 0.01)
    b = (ax + e).astype(np.float32).astype(np.float64)
    return g, oracle.Problem(A=A, b=b, n=n, alpha=1e-2, tau=1e-4), x_true


def test_scan_is_few_view_with_exact_noise_level():
    g, prob, x_true = sphere_few_view_problem()
    assert g.m < g.N
    ax = prob.A @ x_true
    # ||b - A x_true|| / ||A x_true|| = 0.01 up to the float32 rounding of b
    assert abs(np.linalg.norm(prob.b - ax) / np.linalg.norm(ax) - 0.01) < 1e-6


def test_upn_within_2000_iterations_gp_not():
    g, prob, _ = sphere_few_view_problem()
    x0 = np.zeros(prob.N)
    opts = oracle.Options(k_max=2000)
    up = oracle.solve_upn(prob, x0, 1e-4, opts)
    gp = oracle.solve_gp(prob, x0, 1e-4, opts)
    bb = oracle.solve_gpbb(prob, x0, 1e-4, oracle.Options(k_max=20000))
    assert up.status == oracle.OK and up.iters < 2000
    assert gp.status == oracle.NOT_CONVERGED
    assert bb.status == oracle.OK and up.iters < bb.iters
    # phi after the same 2000 iterations: UPN's below GP's
    assert up.f < gp.f

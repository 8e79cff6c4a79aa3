"""The paper's scan shape (Sec. IV-A: parallel beam, view directions spread
over the unit sphere, few-view, noise exactly 0.01, alpha = 0.01) at 12^3 with
3 views on the GPU: every method follows the oracle's first iterations step
by step, UPN's x* matches the oracle's at equal eps, and the GPU methods keep
the ordering of Sec. IV-B (UPN within 2000 iterations, GPBB later, GP not
within 2000)."""
import numpy as np
import pytest

import oracle
from gpu_util import cuda, dev_f32, rel_l2
from test_paper_experiment_shape import sphere_few_view_problem

pytestmark = pytest.mark.gpu

ORACLE = {"gp": oracle.solve_gp, "gpbb": oracle.solve_gpbb, "upn": oracle.solve_upn}


@pytest.fixture(scope="module")
def scan():
    torch = cuda()
    from paper_1105_4002_gb300 import System
    g, prob, _ = sphere_few_view_problem()
    return torch, System(g), prob


def _solve(scan, method, eps, k_max):
    torch, s, prob = scan
    from paper_1105_4002_gb300 import SolveOptions
    x = torch.zeros(prob.N, device="cuda")
    r = s.solve(method, dev_f32(torch, prob.b), prob.alpha, prob.tau, eps, x,
                SolveOptions(k_max=k_max, history=k_max), raise_on_error=False)
    return r, x.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("method", ["gp", "gpbb", "upn"])
def test_first_iterations_follow_the_oracle(scan, method):
    _, _, prob = scan
    ref = ORACLE[method](prob, np.zeros(prob.N), 1e-4, oracle.Options(k_max=20, record=True))
    r, _ = _solve(scan, method, 1e-4, 20)
    h = r.history
    for i in range(min(8, len(ref.history), len(h))):
        o = ref.history[i]
        assert int(h[i, 5]) == o["trials"], (i, h[i], o)
        assert abs(h[i, 1] - o["gnorm"]) <= 1e-4 * o["gnorm"], (i, h[i, 1], o["gnorm"])
        # phi(x^(k+1)) is ~2e-4 of phi(0) = 1/2||b||^2 here: float32 rounding
        # of the data term shows at 1e-6 of phi
        assert abs(h[i, 6] - o["f"]) <= 1e-5 * abs(o["f"]), (i, h[i, 6], o["f"])


def test_upn_xstar_and_the_ordering_of_the_methods(scan):
    _, _, prob = scan
    up, x_up = _solve(scan, "upn", 1e-4, 2000)
    bb, _ = _solve(scan, "gpbb", 1e-4, 20000)
    gp, _ = _solve(scan, "gp", 1e-4, 2000)
    assert up.status == 0 and up.iters < 2000
    assert bb.status == 0 and up.iters < bb.iters
    assert gp.status == 1                       # TVR_NOT_CONVERGED after 2000 iterations
    ref = oracle.solve_upn(prob, np.zeros(prob.N), 1e-4)
    assert rel_l2(x_up, ref.x) <= 1e-4, (rel_l2(x_up, ref.x), up.iters, ref.iters)

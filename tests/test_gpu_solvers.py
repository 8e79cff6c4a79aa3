"""GP / GPBB / UPN on the GPU vs the FP64 oracle (Alg. 1-3, Sec. III-D).

x* parity target: 1e-4 relative L2 at equal eps.  The first iterations are
also compared step by step (same accepted trials, gradient-map norms within
float32 tolerance), before the FP32 and FP64 trajectories may part at a
line-search decision that lies within rounding of its threshold.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import cuda, dev_f32, rel_l2

pytestmark = pytest.mark.gpu

METHODS = ["gp", "gpbb", "upn"]
ORACLE = {"gp": oracle.solve_gp, "gpbb": oracle.solve_gpbb, "upn": oracle.solve_upn}
XSTAR_TOL = 1e-4


@pytest.fixture(scope="module")
def c32():
    torch = cuda()
    from paper_1105_4002_gb300 import System
    cfg = synth.get_config("c32")
    prob, geom, x_true = oracle.problem_from_config(cfg)
    return torch, System(geom), prob, cfg


@pytest.fixture(scope="module")
def oracle_solutions(c32):
    _, _, prob, cfg = c32
    x0 = np.zeros(prob.N)
    return {m: ORACLE[m](prob, x0, cfg.eps, oracle.Options(record=True)) for m in METHODS}


def gpu_solve(c32, method, eps=None, **kw):
    torch, s, prob, cfg = c32
    from paper_1105_4002_gb300 import SolveOptions
    x = torch.zeros(prob.N, device="cuda")
    o = SolveOptions(history=20000, **kw)
    res = s.solve(method, dev_f32(torch, prob.b), prob.alpha, prob.tau, eps or cfg.eps, x, o)
    return res, x.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("method", METHODS)
def test_first_iterations_follow_the_oracle(c32, oracle_solutions, method):
    res, _ = gpu_solve(c32, method)
    ref = oracle_solutions[method]
    h = res.history
    k = min(8, len(ref.history), len(h))
    for i in range(k):
        r = ref.history[i]
        assert int(h[i, 5]) == r["trials"], (i, h[i], r)
        assert abs(h[i, 1] - r["gnorm"]) <= 1e-4 * r["gnorm"], (i, h[i, 1], r["gnorm"])
        assert abs(h[i, 6] - r["f"]) <= 1e-6 * abs(r["f"]), (i, h[i, 6], r["f"])  # phi(x^(k+1))


@pytest.mark.parametrize("method", ["gp", "upn"])
def test_xstar_matches_oracle_at_equal_eps(c32, oracle_solutions, method):
    res, x = gpu_solve(c32, method)
    ref = oracle_solutions[method]
    assert res.status == 0 and ref.status == 0
    _, _, prob, _ = c32
    assert abs(res.phi - prob.f(ref.x)) <= 1e-5 * abs(prob.f(ref.x))
    assert rel_l2(x, ref.x) <= XSTAR_TOL, (method, rel_l2(x, ref.x), res.iters, ref.iters)


@pytest.mark.parametrize("eps", [1e-4, 1e-5])
def test_gpbb_xstar_within_the_oracles_own_sensitivity(c32, eps):
    """GPBB stops on ||G_{1/theta_k}||, and theta_k (the BB step) reacts to
    rounding-size changes of the data, so its stopping point at a loose eps is
    not a continuous function of the inputs: the FP64 oracle itself, given b
    perturbed at the relative size of float32 gradient error (1e-6, seeded),
    returns x* up to ~1e-2 (eps = 1e-4) or ~3e-4 (eps = 1e-5) apart.  The GPU
    result must lie within twice that spread of the oracle's (or within the
    1e-4 target)."""
    _, _, prob, _ = c32
    x0 = np.zeros(prob.N)
    a = oracle.solve_gpbb(prob, x0, eps)
    rng = np.random.default_rng(0)
    spread, fspread = 0.0, 0.0
    for _ in range(4):
        pb = prob.b * (1 + 1e-6 * rng.standard_normal(prob.b.size))
        pert = oracle.Problem(A=prob.A, b=pb, n=prob.n, alpha=prob.alpha, tau=prob.tau)
        r = oracle.solve_gpbb(pert, x0, eps)
        spread = max(spread, rel_l2(r.x, a.x))
        fspread = max(fspread, abs(prob.f(r.x) - prob.f(a.x)))
    res, x = gpu_solve(c32, "gpbb", eps=eps)
    assert res.status == 0 and a.status == 0
    assert rel_l2(x, a.x) <= max(XSTAR_TOL, 2 * spread), (rel_l2(x, a.x), spread)
    assert abs(res.phi - prob.f(a.x)) <= max(1e-5 * prob.f(a.x), 2 * fspread)


@pytest.mark.parametrize("name", ["c32", "c64"])
def test_gpbb_xstar_where_the_minimiser_is_determined(name):
    """GPBB x* within 1e-4 of the oracle's at equal eps, where x(eps) pins down
    the minimiser: alpha = 0.1, tau = 1e-2 and eps = 1e-8 (relative
    gradient-map norm), where the FP64 oracle's GPBB and UPN answers agree to
    2e-5.  (On the few-view tau = 1e-4 problems the oracle's own GPBB x(1e-6)
    is still 8e-3 from its x(1e-8): there x* at equal eps is not determined to
    1e-4 by any implementation; see test_gpbb_xstar_within_the_oracles_own_sensitivity.)"""
    torch = cuda()
    from paper_1105_4002_gb300 import SolveOptions, System
    cfg = synth.get_config(name)
    prob0, geom, _ = oracle.problem_from_config(cfg)
    prob = oracle.Problem(A=prob0.A, b=prob0.b, n=prob0.n, alpha=0.1, tau=1e-2)
    eps = 1e-8
    s = System(geom)
    x = torch.zeros(prob.N, device="cuda")
    res = s.solve("gpbb", dev_f32(torch, prob.b), prob.alpha, prob.tau, eps, x,
                  SolveOptions(k_max=100000))
    ref = oracle.solve_gpbb(prob, np.zeros(prob.N), eps, oracle.Options(k_max=100000))
    assert res.status == 0 and ref.status == 0
    xg = x.cpu().numpy().astype(np.float64)
    assert rel_l2(xg, ref.x) <= XSTAR_TOL, (rel_l2(xg, ref.x), res.iters, ref.iters)
    assert abs(res.phi - prob.f(ref.x)) <= 1e-7 * prob.f(ref.x)
    if name == "c32":  # the minimiser itself: the oracle's UPN answer at the same eps
        up = oracle.solve_upn(prob, np.zeros(prob.N), eps, oracle.Options(k_max=100000))
        assert up.status == 0 and rel_l2(xg, up.x) <= XSTAR_TOL


@pytest.mark.parametrize("method", ["upn", "gp"])
def test_xstar_at_tighter_eps(c32, method):
    """UPN and GP keep 1e-4 at eps = 1e-5 on the few-view problem (both stop
    at the oracle's iteration).  Tighter, the stop itself moves x by more than
    1e-4 per iteration on this problem: the GPU's UPN stops at 1e-7 three
    iterations before the oracle, 1.6e-4 away."""
    eps = 1e-5
    _, _, prob, _ = c32
    res, x = gpu_solve(c32, method, eps=eps)
    ref = ORACLE[method](prob, np.zeros(prob.N), eps, oracle.Options(k_max=100000))
    assert res.status == 0 and ref.status == 0
    assert rel_l2(x, ref.x) <= XSTAR_TOL, (method, rel_l2(x, ref.x), res.iters, ref.iters)


def test_graph_and_direct_launches_agree_bitwise(c32):
    r1, x1 = gpu_solve(c32, "upn", use_graph=True)
    r2, x2 = gpu_solve(c32, "upn", use_graph=False, batch=7)
    assert np.array_equal(x1, x2) and r1.iters == r2.iters and r1.gnorm == r2.gnorm


def test_kernel_timing_in_graph_and_direct_modes(c32):
    """Timed solves give the same result; every working launch is timed once."""
    torch, s, prob, cfg = c32
    r0, x0 = gpu_solve(c32, "upn")
    for graph in (True, False):
        s.profile(True)
        s.profile_read()
        r, x = gpu_solve(c32, "upn", use_graph=graph)
        p = s.profile_read()
        s.profile(False)
        assert np.array_equal(x, x0) and r.iters == r0.iters
        assert p["forward"][0] == r.f_evals - 1              # one trial forward per f-eval after init
        assert p["backward"][0] == r.g_evals - 1             # one back projection per new point
        assert p["step"] == (0, 0.0)                # fused into the trial kernel
        assert p["extrapolation"] == (0, 0.0)       # fused into the trial kernel (UPN)
        assert all(ms > 0 for k, (_, ms) in p.items() if k in ("forward", "backward"))


def test_solves_are_deterministic(c32):
    r1, x1 = gpu_solve(c32, "gpbb")
    r2, x2 = gpu_solve(c32, "gpbb")
    assert np.array_equal(x1, x2) and r1.iters == r2.iters


def test_host_buffers(c32):
    torch, s, prob, cfg = c32
    x = np.zeros(prob.N, np.float32)
    res = s.solve("upn", prob.b.astype(np.float32), prob.alpha, prob.tau, cfg.eps, x)
    _, xd = gpu_solve(c32, "upn")
    assert res.ok and np.array_equal(x.astype(np.float64), xd)


def test_status_paths(c32):
    torch, s, prob, cfg = c32
    from paper_1105_4002_gb300 import SolveOptions, TVRError
    b = dev_f32(torch, prob.b)
    x = torch.zeros(prob.N, device="cuda")
    r = s.solve("upn", b, prob.alpha, prob.tau, 1e-12, x, SolveOptions(k_max=5))
    assert r.status == 1 and r.iters == 5                 # TVR_NOT_CONVERGED
    with pytest.raises(TVRError) as e:                     # BT may not raise L at all
        s.solve("gp", b, prob.alpha, prob.tau, 1e-4, torch.zeros_like(x), SolveOptions(bt_max=0))
    assert e.value.status == -4
    with pytest.raises(TVRError) as e:                     # theta_0 = 1 is far too long a step
        s.solve("gpbb", b, prob.alpha, prob.tau, 1e-4, torch.zeros_like(x),
                SolveOptions(gpbb_max_trials=0))
    assert e.value.status == -4
    bad = prob.b.copy()
    bad[5] = np.nan
    with pytest.raises(TVRError) as e:
        s.solve("gpbb", dev_f32(torch, bad), prob.alpha, prob.tau, 1e-4, torch.zeros_like(x))
    assert e.value.status == -5
    with pytest.raises(TVRError) as e:
        s.solve("upn", b, prob.alpha, prob.tau, -1.0, x)
    assert e.value.status == -1


def test_upn_mu_nonincreasing_and_bt_inequality(c32):
    res, _ = gpu_solve(c32, "upn")
    h = res.history
    mus = h[1:, 3]
    assert np.all(np.diff(mus) <= 0)
    Ls = h[:, 2]
    assert np.all(np.diff(Ls) >= 0)


def test_4cubed_brute_force():
    """Tiny few-view TV problem: every GPU method reaches the L-BFGS-B minimiser."""
    torch = cuda()
    import scipy.optimize as so
    from conftest import small_geometry
    from paper_1105_4002_gb300 import SolveOptions, System
    g = small_geometry(n=4, views=3, det=5)
    A = oracle.system_matrix(g)
    rng = np.random.default_rng(12)
    x_true = np.zeros(64)
    x_true[rng.choice(64, 20, replace=False)] = rng.uniform(0.3, 1.0, 20)
    b = (A @ x_true + 0.01 * rng.normal(size=g.m)).astype(np.float32).astype(np.float64)
    prob = oracle.Problem(A=A, b=b, n=4, alpha=0.05, tau=1e-2)
    ref = so.minimize(lambda x: prob.f_and_grad(x), np.zeros(64), jac=True, method="L-BFGS-B",
                      bounds=[(0, None)] * 64,
                      options=dict(maxiter=100000, ftol=1e-16, gtol=1e-13, maxcor=50)).x
    s = System(g)
    for method in METHODS:
        x = torch.zeros(64, device="cuda")
        res = s.solve(method, dev_f32(torch, b), 0.05, 1e-2, 1e-5, x, SolveOptions(k_max=200000))
        assert res.ok, (method, res)
        assert rel_l2(x.cpu().numpy(), ref) <= 1e-3, method


@pytest.mark.parametrize("n", [7, 8])
@pytest.mark.parametrize("method", ["gp", "upn"])
def test_small_grids_of_odd_and_even_edge(n, method):
    """On 7^3 and 8^3 grids (ragged and whole 4-voxel x-rows, voxel index
    decomposition by invariant divisors) the solvers follow the oracle's first
    iterations and reach its x* at equal eps."""
    torch = cuda()
    from gpu_util import oracle_spread
    from paper_1105_4002_gb300 import SolveOptions, System
    g = synth.cone_geometry(n, 6, 2 * n - 1, 3.0 * n, 2.0 * n)
    A = oracle.system_matrix(g)
    x_true = synth.ellipsoid_phantom(n, 3, (1.0, n / 3.0), (0.2, 1.0), 40 + n)
    z = synth.standard_normal(g.m, 41 + n)
    b = oracle.make_data(A, x_true, z, 0.01).astype(np.float32).astype(np.float64)
    prob = oracle.Problem(A=A, b=b, n=n, alpha=1e-2, tau=1e-4)
    ref = ORACLE[method](prob, np.zeros(prob.N), 1e-4, oracle.Options(record=True))
    s = System(g)
    x = torch.zeros(prob.N, device="cuda")
    res = s.solve(method, dev_f32(torch, b), prob.alpha, prob.tau, 1e-4, x,
                  SolveOptions(history=20000))
    assert res.ok
    h = res.history
    for i in range(min(6, len(ref.history), len(h))):
        assert int(h[i, 5]) == ref.history[i]["trials"], (i, h[i], ref.history[i])
        assert abs(h[i, 1] - ref.history[i]["gnorm"]) <= 1e-4 * ref.history[i]["gnorm"]
    _, spread = oracle_spread(prob, ORACLE[method], 1e-4, draws=2)
    d = rel_l2(x.cpu().numpy(), ref.x)
    assert d <= max(XSTAR_TOL, 3 * spread), (d, spread)


def test_gpbb_two_points_per_pass_give_the_same_iterates(c32):
    """Forming the post-rejection trial in the same pass changes only how many
    passes run: the decisions, counts and iterates are those of one point per
    pass, bit for bit."""
    r1, x1 = gpu_solve(c32, "gpbb", gpbb_points=1, batch=1)
    r2, x2 = gpu_solve(c32, "gpbb", gpbb_points=2, batch=1)
    assert (r1.status, r1.iters, r1.f_evals, r1.g_evals, r1.trials) == \
           (r2.status, r2.iters, r2.f_evals, r2.g_evals, r2.trials)
    assert np.array_equal(x1, x2)
    assert np.array_equal(r1.history, r2.history)
    assert r1.trials > 0 and r2.passes < r1.passes


# the corners of the parameter grid the 64^3 configuration runs (alpha in
# {1e-3, 1e-2, 1e-1}, tau in {1e-2, 1e-4}) beyond the default (1e-2, 1e-4)
GRID = [(1e-3, 1e-4), (1e-1, 1e-2), (1e-2, 1e-2)]


@pytest.mark.parametrize("alpha,tau", GRID)
@pytest.mark.parametrize("method", METHODS)
def test_xstar_across_the_parameter_grid(c32, method, alpha, tau):
    """x* against the oracle's at equal eps for other alpha and tau: within
    1e-4, or within three times the oracle's own spread under float32-sized
    perturbations of b (a stop decision one iteration earlier or later)."""
    from gpu_util import oracle_spread
    torch, s, prob, cfg = c32
    p = oracle.Problem(A=prob.A, b=prob.b, n=prob.n, alpha=alpha, tau=tau)
    x = torch.zeros(prob.N, device="cuda")
    res = s.solve(method, dev_f32(torch, prob.b), alpha, tau, cfg.eps, x)
    ref = ORACLE[method](p, np.zeros(prob.N), cfg.eps)
    assert res.status == 0 and ref.status == 0
    d = rel_l2(x.cpu().numpy(), ref.x)
    if d > XSTAR_TOL:
        _, spread = oracle_spread(p, ORACLE[method], cfg.eps)
        assert d <= 3 * spread, (method, alpha, tau, d, spread, res.iters, ref.iters)

"""The values the paper prints (tests/golden/paper_printed_values.txt, each
with its section) against the defaults of the oracle, the Python options and
the C library, and against the experiment the paper pattern of bench.py runs.
CPU only: the C defaults come from tvr_solve_opts_default, a host function."""
import ctypes
import os

import pytest

import bench
import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def printed():
    vals = {}
    with open(os.path.join(ROOT, "tests", "golden", "paper_printed_values.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = (t.strip() for t in line.split("="))
                vals[k] = float(v)
    return vals


P = printed()


def test_fixture_holds_every_printed_value():
    assert set(P) == {"gpbb_K", "gpbb_sigma", "gpbb_beta0", "experiment_n", "experiment_views_many",
                      "experiment_views_few", "experiment_det", "experiment_noise", "experiment_eps",
                      "experiment_alpha", "phi_star_eps_factor", "upn_iterations_within"}


def test_gpbb_parameters_are_the_defaults_everywhere():
    o = oracle.Options()
    assert (o.gpbb_K, o.gpbb_sigma, o.gpbb_beta0) == (P["gpbb_K"], P["gpbb_sigma"], P["gpbb_beta0"])
    from paper_1105_4002_gb300 import SolveOptions, build
    so = SolveOptions()
    assert (so.gpbb_K, so.gpbb_sigma, so.gpbb_beta0) == (P["gpbb_K"], P["gpbb_sigma"],
                                                         P["gpbb_beta0"])
    build.build()
    import paper_1105_4002_gb300 as pkg
    from paper_1105_4002_gb300 import _capi
    co = _capi.SolveOpts()
    pkg.lib().tvr_solve_opts_default(ctypes.byref(co))
    assert (co.gpbb_K, co.gpbb_sigma, co.gpbb_beta0) == (P["gpbb_K"], P["gpbb_sigma"],
                                                         P["gpbb_beta0"])


def test_the_paper_pattern_runs_the_printed_experiment():
    E = bench.PAPER_EXPERIMENT
    assert E["n"] == P["experiment_n"] and E["det"] == P["experiment_det"]
    assert E["views"] == (P["experiment_views_many"], P["experiment_views_few"])
    assert (E["noise"], E["eps"], E["alpha"]) == (P["experiment_noise"], P["experiment_eps"],
                                                 P["experiment_alpha"])
    assert E["phi_star_eps_factor"] == P["phi_star_eps_factor"]
    assert max(E["checkpoints"]) == P["upn_iterations_within"]
    # the scan shape: parallel beam, views spread over the sphere, det^2 pixels per view
    n, det = int(E["n"]), int(E["det"])
    for views in E["views"]:
        g = synth.sphere_parallel_geometry(n, views, det)
        assert (g.n, g.n_views, g.det_cols, g.det_rows) == (n, views, det, det)
        assert g.m == views * det * det and g.N == n ** 3
    # the few-view scan has fewer rows than unknowns (Sec. IV-A)
    assert E["views"][1] * det * det < n ** 3 < E["views"][0] * det * det


@pytest.mark.parametrize("level", [P["experiment_noise"]])
def test_noise_is_exactly_the_printed_relative_magnitude(level):
    import numpy as np
    ax = np.abs(np.random.default_rng(0).standard_normal(1000)) + 1.0
    z = synth.standard_normal(1000, 7)
    e = synth.noise_exact(ax, z, level)
    assert abs(np.linalg.norm(e) / np.linalg.norm(ax) - level) <= 1e-12

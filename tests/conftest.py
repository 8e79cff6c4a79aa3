import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libtvr.so")
    config.addinivalue_line("markers", "slow: longer CPU oracle runs")


@pytest.fixture(scope="session")
def c32_problem():
    import oracle
    import synth
    cfg = synth.get_config("c32")
    prob, geom, x_true = oracle.problem_from_config(cfg)
    return cfg, prob, geom, x_true


def small_geometry(n=4, views=8, det=6):
    import synth
    return synth.cone_geometry(n, views, det, 3.0 * n, 2.0 * n)

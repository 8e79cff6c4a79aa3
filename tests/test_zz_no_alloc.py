"""tvr_phi_and_grad_noalloc against tvr_phi_and_grad, through the C ABI.

The no-allocation variant exists for callers that must not allocate device
memory while they evaluate phi: code whose device memory belongs to another
framework's caching allocator under a fixed budget, and latency-bound loops
that must stay out of the driver's allocator (which can synchronise the
device).  It must give the same phi and gradient as the ordinary entry point,
on consecutive calls that share its fixed scratch array, for stored FP32 and
matrix-free systems, and refuse what its scratch cannot hold.
"""
import ctypes

import numpy as np
import pytest

import synth
from gpu_util import cuda

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-5
PHI_TOL = 1e-6


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _noalloc(s, x, b, alpha, tau, grad, stream):
    from paper_1105_4002_gb300 import lib
    out = (ctypes.c_double * 3)()
    st = lib().tvr_phi_and_grad_noalloc(
        s.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(b.data_ptr()), alpha, tau,
        None, ctypes.cast(out, ctypes.c_void_p),
        ctypes.c_void_p(grad.data_ptr()) if grad is not None else None, stream)
    return st, (out[0], out[1], out[2])


@pytest.mark.parametrize("storage", ["fp32", "mf"])
def test_noalloc_matches_phi_and_grad_on_consecutive_calls(storage):
    torch = cuda()
    from paper_1105_4002_gb300 import System
    geom = synth.get_config("c32").geometry()
    s = System(geom, storage=storage)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(4)
    b = torch.tensor(rng.uniform(0, 5, geom.m), dtype=torch.float32, device="cuda")
    for call, (alpha, tau) in enumerate([(1e-2, 1e-4), (0.3, 1e-2)]):
        x = torch.tensor(rng.uniform(0, 1, geom.N), dtype=torch.float32, device="cuda")
        g_ref = torch.empty(geom.N, device="cuda")
        phi_ref = s.phi_and_grad(x, b, alpha, tau, grad=g_ref)
        g = torch.full((geom.N,), float("nan"), device="cuda")
        st, phi = _noalloc(s, x, b, alpha, tau, g, stream)
        assert st == 0, call
        for u, v in zip(phi, phi_ref):
            assert abs(u - v) <= PHI_TOL * abs(v), call
        assert _rel(g.cpu().numpy(), g_ref.cpu().numpy()) <= GRAD_TOL, call
        # phi only
        st, phi_only = _noalloc(s, x, b, alpha, tau, None, stream)
        assert st == 0 and abs(phi_only[0] - phi_ref[0]) <= PHI_TOL * abs(phi_ref[0])


def test_noalloc_refuses_what_its_scratch_cannot_hold():
    torch = cuda()
    from paper_1105_4002_gb300 import System, lib
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # one view, 2100 x 2100 pixels on a 2^3 grid: 4,410,000 rays > 4,194,304
    geom = synth.cone_geometry(2, 1, 2100, 6.0, 4.0, pitch=0.001)
    s = System(geom)
    x = torch.zeros(geom.N, device="cuda")
    b = torch.zeros(geom.m, device="cuda")
    g = torch.empty(geom.N, device="cuda")
    st, _ = _noalloc(s, x, b, 1e-2, 1e-4, g, stream)
    assert st == -1
    assert b"static scratch" in lib().tvr_last_error()
    # BF16 row-scale storage would need a second, row-scaled residual
    geom8 = synth.get_config("c8").geometry()
    s16 = System(geom8, storage="bf16")
    x8 = torch.zeros(geom8.N, device="cuda")
    b8 = torch.zeros(geom8.m, device="cuda")
    st, _ = _noalloc(s16, x8, b8, 1e-2, 1e-4, torch.empty(geom8.N, device="cuda"), stream)
    assert st == -1 and b"BF16" in lib().tvr_last_error()
    # host memory would need staging buffers
    small = System(geom8)
    xh = np.zeros(small.N, np.float32)
    bh = np.zeros(small.m, np.float32)
    st = lib().tvr_phi_and_grad_noalloc(small.handle, xh.ctypes.data_as(ctypes.c_void_p),
                                        bh.ctypes.data_as(ctypes.c_void_p), 1e-2, 1e-4, None, None,
                                        None, stream)
    assert st == -1

"""Precision of the sums the line-search decisions rest on (Alg. 1, Alg. 2).

The solvers accumulate their control sums on the device in double-single
(a float pair, about 48 bits) and finish them in FP64.  tvr_trial_sums runs
the solvers' own trial kernel once from a fixed float32 base point p, gradient
g and step s and returns its totals:
    ||A xbar - b||^2, ||A d||^2, g^T d, ||d||^2, sum_j B_h(D_j xbar; D_j p), TV_tau(xbar)
with xbar = P_Q(p - s g), d = xbar - p.

Two checks:
  1. the reductions: every total whose per-term float32 values can be formed
     here bit for bit (the products g_j d_j and d_j^2, the returned residuals,
     the per-voxel Huber terms evaluated with the kernel's float32 operation
     order) must equal the FP64 sum of those terms to 1e-10 of sum |term|;
  2. the formulas: the same totals against the oracle's FP64 definitions of the
     quantities (A d with FP64 A, the Bregman divergence written out as
     h(z') - h(z) - grad h(z).(z' - z), tv_value), within float32 per-term
     rounding.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import cuda, dev_f32

pytestmark = pytest.mark.gpu

F = np.float32


def _diff(v, n):
    """float32 forward differences (x, y, z) with 0 across the border, [N] each."""
    a = v.reshape(n, n, n)
    out = []
    for ax in (2, 1, 0):
        d = np.zeros_like(a)
        sl_hi = [slice(None)] * 3
        sl_lo = [slice(None)] * 3
        sl_hi[ax] = slice(1, None)
        sl_lo[ax] = slice(None, -1)
        d[tuple(sl_lo)] = a[tuple(sl_hi)] - a[tuple(sl_lo)]
        out.append(d.reshape(-1))
    return out


def _norm3(z):
    return np.sqrt((z[0] * z[0] + z[1] * z[1]) + z[2] * z[2])


def _huber32(nrm, tau):
    return np.where(nrm >= tau, nrm - F(0.5) * tau, (nrm * nrm) / (F(2.0) * tau))


def kernel_terms(p, xb, n, tau):
    """Per-voxel float32 terms of sum_j B_h and TV_tau(xbar), in the trial
    kernel's operation order (quadratic zone |dl|^2 / 2 tau; linear zone
    |z x dl|^2 / (|z| (|zb||z| + z.zb)); otherwise the difference form)."""
    tau = F(tau)
    z = _diff(p, n)
    zb = _diff(xb, n)
    # dl_e = (xbar_{j+e} - p_{j+e}) - d_j with d = xbar - p, 0 across the border
    d = xb - p
    idx = np.arange(d.size)
    dl = []
    for e, off in enumerate((1, n, n * n)):
        inside = (idx // off) % n + 1 < n
        de = np.zeros_like(d)
        de[inside] = (xb[idx[inside] + off] - p[idx[inside] + off]) - d[inside]
        dl.append(de)
    nz = _norm3(z)
    nb = _norm3(zb)
    quad = (nz < tau) & (nb < tau)
    d2 = (dl[0] * dl[0] + dl[1] * dl[1]) + dl[2] * dl[2]
    t_quad = d2 / (F(2.0) * tau)
    dot = (z[0] * zb[0] + z[1] * zb[1]) + z[2] * zb[2]
    lin = (nz >= tau) & (nb >= tau) & (dot > 0)
    c0 = z[1] * dl[2] - z[2] * dl[1]
    c1 = z[2] * dl[0] - z[0] * dl[2]
    c2 = z[0] * dl[1] - z[1] * dl[0]
    cc = (c0 * c0 + c1 * c1) + c2 * c2
    with np.errstate(divide="ignore", invalid="ignore"):
        t_lin = cc / (nz * (nb * nz + dot))
    den = np.maximum(tau, nz)
    wd = ((z[0] * dl[0] + z[1] * dl[1]) + z[2] * dl[2]) / den
    t_mix = np.maximum((_huber32(nb, tau) - _huber32(nz, tau)) - wd, F(0))
    breg = np.where(quad, t_quad, np.where(lin, t_lin, t_mix)).astype(F)
    return breg, _huber32(nb, tau).astype(F)


def oracle_bregman(p, xb, n, tau):
    """sum_j h(D_j xbar) - h(D_j p) - grad h(D_j p) . D_j (xbar - p), in FP64."""
    z = np.stack(oracle.tv.forward_differences(p.astype(np.float64), n)).reshape(3, -1)
    zb = np.stack(oracle.tv.forward_differences(xb.astype(np.float64), n)).reshape(3, -1)
    nz = np.linalg.norm(z, axis=0)
    nb = np.linalg.norm(zb, axis=0)
    w = z / np.maximum(tau, nz)
    return float(np.sum(oracle.tv.huber(nb, tau) - oracle.tv.huber(nz, tau)
                        - np.sum(w * (zb - z), axis=0)))


@pytest.fixture(scope="module")
def case():
    torch = cuda()
    from paper_1105_4002_gb300 import System
    cfg = synth.get_config("c32")
    prob, geom, x_true = oracle.problem_from_config(cfg)
    rng = np.random.default_rng(21)
    # a point near the phantom with some voxels at the bound, its gradient
    p = np.maximum(x_true + 0.05 * rng.standard_normal(prob.N), 0.0).astype(F)
    g = prob.grad(p.astype(np.float64)).astype(F)
    return torch, System(geom), prob, cfg, p, g


@pytest.mark.parametrize("step_scale", [1e-3, 3e-2])
def test_trial_sums_match_fp64_sums_of_the_same_float32_terms(case, step_scale):
    torch, s, prob, cfg, p, g = case
    n, tau = cfg.n, cfg.tau
    step = step_scale * float(np.max(p)) / float(np.max(np.abs(g)))
    xb_d = torch.empty(prob.N, device="cuda")
    r_d = torch.empty(prob.b.size, device="cuda")
    sums = s.trial_sums(dev_f32(torch, p), dev_f32(torch, g), dev_f32(torch, prob.b), step, tau,
                        xbar=xb_d, resid=r_d)
    xb = xb_d.cpu().numpy()
    r = r_d.cpu().numpy().astype(np.float64)
    # xbar = P_Q(p - s g) rounded as the kernel rounds it
    xb_ref = np.maximum(p - F(step) * g, F(0))
    assert np.array_equal(xb, xb_ref)
    assert 0 < np.count_nonzero((xb == 0) & (p > 0))          # the bound is active somewhere
    d = (xb - p).astype(np.float64)
    g64 = g.astype(np.float64)
    breg, hb = kernel_terms(p, xb, n, tau)
    exact = {  # index -> float32-exact per-term values
        0: r * r,
        2: g64 * d,
        3: d * d,
        4: breg.astype(np.float64),
        5: hb.astype(np.float64),
    }
    for k, terms in exact.items():
        ref = float(np.sum(terms))
        scale = float(np.sum(np.abs(terms)))
        assert abs(sums[k] - ref) <= 1e-10 * scale, (k, sums[k], ref, scale)
    # against the oracle's definitions: float32 row sums (A d, whose entries
    # cancel, and A xbar, whose residual is ~1% of it) and float32 per-voxel
    # terms
    Ad = prob.A @ d
    assert sums[1] == pytest.approx(float(Ad @ Ad), rel=1e-4)
    rr = prob.A @ xb.astype(np.float64) - prob.b
    assert sums[0] == pytest.approx(float(rr @ rr), rel=1e-5)
    assert sums[4] == pytest.approx(oracle_bregman(p, xb, n, tau), rel=1e-5)
    assert sums[5] == pytest.approx(oracle.tv.tv_value(xb.astype(np.float64), n, tau), rel=1e-6)


def test_trial_sums_reject_bad_arguments(case):
    torch, s, prob, cfg, p, g = case
    from paper_1105_4002_gb300 import TVRError
    pd, gd, bd = dev_f32(torch, p), dev_f32(torch, g), dev_f32(torch, prob.b)
    with pytest.raises(TVRError):
        s.trial_sums(pd, gd, bd, -1.0, cfg.tau)
    with pytest.raises(TVRError):
        s.trial_sums(pd, gd, bd, 1e-3, 0.0)
    with pytest.raises(TVRError):                 # host vectors: the probe takes device memory
        s.trial_sums(p, g, prob.b.astype(F), 1e-3, cfg.tau)

"""GB300-native TV-regularised CT reconstruction with GP, GPBB and UPN.

Python face of libtvr.so (C ABI in include/tvr.h).  Every step of the path
runs in the library's CUDA kernels; this module only marshals arguments:
torch CUDA tensors (device memory, current stream) or host arrays (numpy /
CPU tensors, staged by the library).

    sys = System(geometry)                  # A from the scan geometry (Siddon, FP32 CSR + CSC)
    phi = sys.phi_and_grad(x, b, alpha, tau, grad=g)
    info = sys.solve("upn", b, alpha, tau, eps, x)   # x: x0 in, x* out
"""
from __future__ import annotations

import ctypes
import dataclasses

import numpy as np

from . import _capi
from ._capi import (TVR_CONE, TVR_NOT_CONVERGED, TVR_OK, TVR_PARALLEL, TVR_STOP_PER_N, TVR_STOP_REL,
                    TVRError, check, lib)

__all__ = ["System", "SolveOptions", "SolveResult", "project_Q", "solve_batch", "TVRError", "lib",
           "TVR_STOP_REL", "TVR_STOP_PER_N"]


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a, n: int, name: str, dtype=np.float32):
    """(pointer, is_cuda) for a float32 vector of n entries (torch tensor or numpy)."""
    if a is None:
        return None, False
    if _is_torch(a):
        import torch
        if a.dtype != torch.float32:
            raise TypeError(f"{name}: expected float32, got {a.dtype}")
        if not a.is_contiguous():
            raise ValueError(f"{name}: tensor must be contiguous")
        if a.numel() != n:
            raise ValueError(f"{name}: expected {n} entries, got {a.numel()}")
        return ctypes.c_void_p(a.data_ptr()), a.is_cuda
    if isinstance(a, np.ndarray):
        if a.dtype != dtype:
            raise TypeError(f"{name}: expected {np.dtype(dtype)}, got {a.dtype}")
        if not a.flags.c_contiguous:
            raise ValueError(f"{name}: array must be C-contiguous")
        if a.size != n:
            raise ValueError(f"{name}: expected {n} entries, got {a.size}")
        return a.ctypes.data_as(ctypes.c_void_p), False
    raise TypeError(f"{name}: expected a torch tensor or numpy array")


def _stream(stream, *arrays):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    if any(a is not None and _is_torch(a) and a.is_cuda for a in arrays):
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(0)


@dataclasses.dataclass
class SolveOptions:
    k_max: int = 20000
    stop_mode: int = TVR_STOP_REL
    gpbb_K: int = 2
    gpbb_max_trials: int = 12
    bt_max: int = 60
    use_graph: bool = True
    batch: int = 32
    gpbb_points: int = 2  # GPBB trial points per forward pass (1 or 2; same iterates)
    sweep_lanes: int = 0  # solve_sweep row split: 0 = autotuned, or 2, 4, 8 lanes per row
    gpbb_sigma: float = 0.1
    gpbb_beta0: float = 0.95
    rho_L: float = 2.0
    L_bar: float = 1.0
    mu_bar: float = 0.1
    history: int = 0  # records to keep (0 = none)


@dataclasses.dataclass
class SolveResult:
    status: int
    iters: int
    f_evals: int
    g_evals: int
    trials: int
    passes: int
    phi: float
    gnorm: float
    gnorm0: float
    stop_value: float
    L: float
    theta: float
    mu: float
    history: np.ndarray | None = None
    lanes: tuple[int, int] = (0, 0)  # solve_sweep: lanes per (row, column) of its projections

    @property
    def ok(self) -> bool:
        return self.status == TVR_OK


class System:
    """A built system matrix (owns A and all device workspace)."""

    STORAGE = {"fp32": _capi.TVR_STORAGE_FP32, "bf16": _capi.TVR_STORAGE_BF16_ROWSCALE,
               "u16": _capi.TVR_STORAGE_U16_ROWSCALE, "mf": _capi.TVR_STORAGE_MATRIX_FREE}

    def __init__(self, geometry, stream=None, storage: str = "fp32"):
        views = np.ascontiguousarray(geometry.views, dtype=np.float64)
        self._views = views
        g = _capi.Geometry(int(geometry.n), int(views.shape[0]), int(geometry.det_cols),
                           int(geometry.det_rows), int(getattr(geometry, "kind", TVR_CONE)), 0,
                           views.ctypes.data)
        h = ctypes.c_void_p()
        check(lib().tvr_build_system(ctypes.byref(g), self.STORAGE[storage], _stream(stream),
                                     ctypes.byref(h)), "tvr_build_system")
        self.storage = storage
        self._h = h
        m, N, nnz = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        check(lib().tvr_system_shape(h, ctypes.byref(m), ctypes.byref(N), ctypes.byref(nnz)),
              "tvr_system_shape")
        self.m, self.N, self.nnz = m.value, N.value, nnz.value
        self.n = int(geometry.n)

    def close(self):
        if getattr(self, "_h", None):
            lib().tvr_system_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # ---- A ----
    def export_csr(self):
        rp = np.zeros(self.m + 1, np.int64)
        col = np.zeros(max(self.nnz, 1), np.int32)
        val = np.zeros(max(self.nnz, 1), np.float32)
        check(lib().tvr_system_export_csr(self._h, rp.ctypes.data, col.ctypes.data, val.ctypes.data),
              "tvr_system_export_csr")
        return rp, col[:self.nnz], val[:self.nnz]

    def export_csc(self):
        cp = np.zeros(self.N + 1, np.int64)
        row = np.zeros(max(self.nnz, 1), np.int32)
        val = np.zeros(max(self.nnz, 1), np.float32)
        check(lib().tvr_system_export_csc(self._h, cp.ctypes.data, row.ctypes.data, val.ctypes.data),
              "tvr_system_export_csc")
        return cp, row[:self.nnz], val[:self.nnz]

    def forward(self, x, y, stream=None):
        """y = A x."""
        px, _ = _ptr(x, self.N, "x")
        py, _ = _ptr(y, self.m, "y")
        check(lib().tvr_forward(self._h, px, py, _stream(stream, x, y)), "tvr_forward")
        return y

    def adjoint(self, r, z, stream=None):
        """z = A^T r."""
        pr, _ = _ptr(r, self.m, "r")
        pz, _ = _ptr(z, self.N, "z")
        check(lib().tvr_adjoint(self._h, pr, pz, _stream(stream, r, z)), "tvr_adjoint")
        return z

    def phi_and_grad(self, x, b, alpha: float, tau: float, grad=None, resid=None, phi_dev=None,
                     sync: bool = True, stream=None):
        """phi (and its parts) at x; fills grad / resid when given.

        Returns (phi, 1/2||Ax-b||^2, TV_tau(x)) as floats when sync, else None
        (then phi_dev, a float64 CUDA tensor of >= 3 entries, receives them).
        """
        px, _ = _ptr(x, self.N, "x")
        pb, _ = _ptr(b, self.m, "b")
        pg, _ = _ptr(grad, self.N, "grad")
        pr, _ = _ptr(resid, self.m, "resid")
        pdev = None
        if phi_dev is not None:
            import torch
            if phi_dev.dtype != torch.float64 or not phi_dev.is_cuda or phi_dev.numel() < 3:
                raise ValueError("phi_dev: need a float64 CUDA tensor with >= 3 entries")
            pdev = ctypes.c_void_p(phi_dev.data_ptr())
        out = (ctypes.c_double * 3)()
        check(lib().tvr_phi_and_grad(self._h, px, pb, float(alpha), float(tau), pdev,
                                     ctypes.cast(out, ctypes.c_void_p) if sync else None, pg, pr,
                                     _stream(stream, x, b, grad, resid)), "tvr_phi_and_grad")
        return (out[0], out[1], out[2]) if sync else None

    def gradient_map_norm(self, x, grad, nu: float, stream=None) -> float:
        px, _ = _ptr(x, self.N, "x")
        pg, _ = _ptr(grad, self.N, "grad")
        out = ctypes.c_double()
        check(lib().tvr_gradient_map_norm(self._h, px, pg, float(nu), ctypes.byref(out),
                                          _stream(stream, x, grad)), "tvr_gradient_map_norm")
        return out.value

    def trial_sums(self, p, g, b, step: float, tau: float, xbar=None, resid=None,
                   stream=None):
        """The FP64 sums of one projected trial step from p along g (Alg. 1 and
        Alg. 2's tests): {||A xbar - b||^2, ||A d||^2, g^T d, ||d||^2,
        sum_j B_h(D_j xbar; D_j p), TV_tau(xbar)}; device vectors only."""
        pp, _ = _ptr(p, self.N, "p")
        pgr, _ = _ptr(g, self.N, "g")
        pb, _ = _ptr(b, self.m, "b")
        px = _ptr(xbar, self.N, "xbar")[0] if xbar is not None else None
        pr = _ptr(resid, self.m, "resid")[0] if resid is not None else None
        out = (ctypes.c_double * 6)()
        check(lib().tvr_trial_sums(self._h, pp, pgr, pb, float(step), float(tau),
                                   ctypes.cast(out, ctypes.c_void_p), px, pr,
                                   _stream(stream, p, g, b)), "tvr_trial_sums")
        return list(out)

    # ---- solvers ----
    def solve(self, method: str, b, alpha: float, tau: float, eps: float, x,
              opts: SolveOptions | None = None, stream=None,
              raise_on_error: bool = True) -> SolveResult:
        """Run GP / GPBB / UPN from x (x0 in, x* out: the last accepted iterate).
        With raise_on_error=False a line-search or non-finite stop is returned
        in the result's status instead of raised."""
        fn = {"gp": lib().tvr_solve_gp, "gpbb": lib().tvr_solve_gpbb,
              "upn": lib().tvr_solve_upn}[method]
        o = opts or SolveOptions()
        co = _capi.SolveOpts()
        lib().tvr_solve_opts_default(ctypes.byref(co))
        for f in ("k_max", "stop_mode", "gpbb_K", "gpbb_max_trials", "bt_max", "batch",
                  "gpbb_points", "sweep_lanes", "gpbb_sigma", "gpbb_beta0", "rho_L", "L_bar",
                  "mu_bar"):
            setattr(co, f, getattr(o, f))
        co.use_graph = 1 if o.use_graph else 0
        hist = None
        if o.history > 0:
            hist = np.zeros((o.history, _capi.TVR_HIST_FIELDS), np.float64)
            co.history = hist.ctypes.data
            co.history_len = o.history
        pb, _ = _ptr(b, self.m, "b")
        px, _ = _ptr(x, self.N, "x")
        info = _capi.SolveInfo()
        st = fn(self._h, pb, float(alpha), float(tau), float(eps), ctypes.byref(co), px,
                ctypes.byref(info), _stream(stream, b, x))
        if raise_on_error or st not in (_capi.TVR_ERR_LINESEARCH, _capi.TVR_ERR_NONFINITE):
            check(st, f"tvr_solve_{method}", allow=(TVR_OK, TVR_NOT_CONVERGED))
        return SolveResult(status=info.status, iters=info.iters, f_evals=info.f_evals,
                           g_evals=info.g_evals, trials=info.trials, passes=info.passes,
                           phi=info.phi, gnorm=info.gnorm, gnorm0=info.gnorm0,
                           stop_value=info.stop_value, L=info.L, theta=info.theta, mu=info.mu,
                           history=hist[:info.history_used].copy() if hist is not None else None)

    def solve_sweep(self, method: str, b, alphas, tau: float, eps: float, X,
                    opts: SolveOptions | None = None, stream=None):
        """Solve for up to 8 alphas at once (columns of X: x0 in, x* out); list of results."""
        code = {"gp": 1, "gpbb": 2, "upn": 3}[method]
        k = len(alphas)
        al = (ctypes.c_double * k)(*[float(a) for a in alphas])
        co = self._opts(opts)
        pb, _ = _ptr(b, self.m, "b")
        px, _ = _ptr(X, k * self.N, "X")
        infos = (_capi.SolveInfo * k)()
        st = lib().tvr_solve_sweep(self._h, code, pb, ctypes.cast(al, ctypes.c_void_p), k,
                                   float(tau), float(eps), ctypes.byref(co), px, infos,
                                   _stream(stream, b, X))
        check(st, "tvr_solve_sweep", allow=(TVR_OK, TVR_NOT_CONVERGED))
        return [SolveResult(status=i.status, iters=i.iters, f_evals=i.f_evals, g_evals=i.g_evals,
                            trials=i.trials, passes=i.passes, phi=i.phi, gnorm=i.gnorm,
                            gnorm0=i.gnorm0, stop_value=i.stop_value, L=i.L, theta=i.theta,
                            mu=i.mu, lanes=(i.lanes & 0xff, (i.lanes >> 8) & 0xff))
                for i in infos]

    def _opts(self, opts):
        o = opts or SolveOptions()
        co = _capi.SolveOpts()
        lib().tvr_solve_opts_default(ctypes.byref(co))
        for f in ("k_max", "stop_mode", "gpbb_K", "gpbb_max_trials", "bt_max", "batch",
                  "gpbb_points", "sweep_lanes", "gpbb_sigma", "gpbb_beta0", "rho_L", "L_bar",
                  "mu_bar"):
            setattr(co, f, getattr(o, f))
        co.use_graph = 1 if o.use_graph else 0
        return co

    # ---- measurement ----
    def profile(self, enable, kinds=("forward", "backward", "step", "extrapolation"),
                sample_stride: int = 1):
        """Time launches of the given kernel kinds (enable=False: stop timing);
        solves in graph mode time every sample_stride-th pass."""
        names = ["forward", "backward", "step", "extrapolation"]
        mask = sum(1 << names.index(k) for k in kinds) if enable else 0
        if enable:
            mask |= (int(sample_stride) & 0xff) << 8
        check(lib().tvr_profile_enable(self._h, mask), "tvr_profile_enable")

    def profile_read(self):
        counts = (ctypes.c_int64 * 4)()
        ms = (ctypes.c_double * 4)()
        check(lib().tvr_profile_read(self._h, ctypes.cast(counts, ctypes.c_void_p),
                                     ctypes.cast(ms, ctypes.c_void_p)), "tvr_profile_read")
        return {"forward": (counts[0], ms[0]), "backward": (counts[1], ms[1]),
                "step": (counts[2], ms[2]), "extrapolation": (counts[3], ms[3])}


def solve_batch(method: str, systems, bs, alphas, tau: float, eps: float, xs,
                opts: SolveOptions | None = None, stream=None):
    """Solve independent problems concurrently (one stream per system); list of results."""
    code = {"gp": 1, "gpbb": 2, "upn": 3}[method]
    n = len(systems)
    if not (len(bs) == len(xs) == len(alphas) == n):
        raise ValueError("systems, bs, alphas and xs must have the same length")
    hs = (ctypes.c_void_p * n)(*[s.handle.value for s in systems])
    pb = (ctypes.c_void_p * n)(*[_ptr(b, s.m, "b")[0].value for b, s in zip(bs, systems)])
    px = (ctypes.c_void_p * n)(*[_ptr(x, s.N, "x")[0].value for x, s in zip(xs, systems)])
    al = (ctypes.c_double * n)(*[float(a) for a in alphas])
    co = systems[0]._opts(opts)
    infos = (_capi.SolveInfo * n)()
    st = lib().tvr_solve_batch(ctypes.cast(hs, ctypes.c_void_p), n, code,
                               ctypes.cast(pb, ctypes.c_void_p), ctypes.cast(al, ctypes.c_void_p),
                               float(tau), float(eps), ctypes.byref(co),
                               ctypes.cast(px, ctypes.c_void_p), infos,
                               _stream(stream, *bs, *xs))
    check(st, "tvr_solve_batch", allow=(TVR_OK, TVR_NOT_CONVERGED))
    return [SolveResult(status=i.status, iters=i.iters, f_evals=i.f_evals, g_evals=i.g_evals,
                        trials=i.trials, passes=i.passes, phi=i.phi, gnorm=i.gnorm,
                        gnorm0=i.gnorm0, stop_value=i.stop_value, L=i.L, theta=i.theta, mu=i.mu)
            for i in infos]


def project_Q(x, stream=None):
    """In-place P_Q(x) = max(x, 0) on a float32 CUDA tensor."""
    px, is_cuda = _ptr(x, x.numel(), "x")
    if not is_cuda:
        raise ValueError("project_Q: x must be a CUDA tensor")
    check(lib().tvr_project_Q(px, int(x.numel()), _stream(stream, x)), "tvr_project_Q")
    return x

#!/usr/bin/env python
"""Benchmark of the TV-CT gradient-method path on GB300.

One step = one GPBB solve and one UPN solve to the relative gradient-map
norm eps, from x0 = 0, on the 64^3 few-view cone-beam problem (25 views,
96 x 96 detector, 10 seeded ellipsoids, 1% noise, alpha 1e-2, tau 1e-4).
Every part of the hot path runs inside a step: forward projection, back
projection fused with the TV stencil, projected steps, the FP64 control
reductions, BB / BT / mu-estimate control and the UPN extrapolation.

value  = gradient evaluations (grad phi) per second inside the solves,
         summed over ranks (independent problems per rank: weak scaling);
e2e    = the same through the public call with host (pinned) b and x, the
         copies inside the timed region;
roofline = the dominant kernel (CSC back projection + TV, or CSR forward
         projection) timed with CUDA events on its launch stream during the
         timed region, algorithmic bytes per launch / mean duration.
--impl reference times the FP64 CPU oracle on the same workload instead.
"""
from __future__ import annotations

import os

# The CPU legs (the oracle) run on one host thread: numpy's BLAS would
# otherwise spread vector products over all cores.  Set before numpy loads.
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import json
import math
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grad-phi evals/s and time-to-eps (GPBB/UPN) at 64^3, % of HBM roofline, vs plain FP32"
UNIT = "grad-phi evals/s"
L2_BYTES = 129e6


def _e(v: float) -> str:
    m, e = f"{v:.0e}".split("e")
    return f"{m}e{int(e)}"


def workload(cfg, eps) -> str:
    """The bench workload of a configuration, in words."""
    return (f"TV-CT {cfg.n}^3, cone beam {cfg.views} views x {cfg.det}^2 px (Dso {cfg.dso:g}, "
            f"Dod {cfg.dod:g}), {cfg.ellipsoids} seeded ellipsoids, {cfg.noise * 100:g}% noise, "
            f"alpha {_e(cfg.alpha)}, tau {_e(cfg.tau)}; one GPBB + one UPN solve to relative "
            f"gradient-map norm {_e(eps)} from x0 = 0")


def l2_note(nnz: int) -> str:
    """Whether the stored matrix outgrows L2 (then no flush is needed between steps)."""
    mb = 8 * nnz / 1e6
    if 2 * 8 * nnz > L2_BYTES:
        return f"inputs larger than L2: A stored as CSR + CSC (2 x {mb:.0f} MB) > 129 MB L2"
    return (f"A stored as CSR + CSC (2 x {mb:.0f} MB) fits in the 129 MB L2: L2-resident between "
            f"steps, not flushed")


HBM_FALLBACK_GBS = 6800.0


def dtype_of(storage: str) -> str:
    """The arithmetic type of the path with A stored as `storage`."""
    return {"fp32": "f32", "bf16": "bf16 values, f32 arithmetic",
            "u16": "u16 fixed-point values, f32 arithmetic",
            "mf": "f32 (matrix-free entries)"}[storage]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c64")
    ap.add_argument("--eps", type=float, default=None)
    ap.add_argument("--graph", type=int, default=1,
                    help="1: replay passes as CUDA graphs (kernel timing by event nodes); "
                         "0: launch every pass directly")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-other-configs", action="store_true",
                    help="skip the short runs of the autograd (128^3) and batch (48 problems) "
                         "configurations that the default line reports under other_configs")
    ap.add_argument("--phi-loop", type=int, default=200)
    ap.add_argument("--storage", default="fp32", choices=["fp32", "bf16", "u16", "mf"],
                    help="A as float32, as bfloat16 codes with per-row float32 scale, as 16-bit "
                         "unsigned fixed-point codes with per-row float32 step, or matrix-free "
                         "(entries computed on the fly)")
    ap.add_argument("--pattern", default="solve",
                    choices=["solve", "autograd", "batch", "paper", "grid", "precision", "sweep",
                             "projectors"],
                    help="autograd: phi forward + backward through torch.autograd at 128^3; "
                         "grid: GP, GPBB and UPN over alpha x tau x eps at 64^3; "
                         "precision: GPBB and UPN at 256^3 with A stored three ways; "
                         "sweep: one 8-alpha sweep at 128^3 (--sweep-kmax iterations); "
                         "projectors: forward and adjoint projection times of --storage at --config")
    ap.add_argument("--sweep-kmax", type=int, default=20000,
                    help="iteration cap of the sweep pattern (a short run for profiling)")
    ap.add_argument("--roofline-steps", type=int, default=3,
                    help="extra steps after the timed region in which the dominant kernels "
                         "are timed with CUDA events")
    ap.add_argument("--cpu-baseline-b", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-baseline-kmax", type=int, default=20000, help=argparse.SUPPRESS)
    return ap.parse_args()


# ---------------------------------------------------------------- helpers
def measured_peak_gbs():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sms.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sms.sort()
        med = sms[len(sms) // 2] if sms else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sms)}


def kernel_source_digest(paths) -> str:
    """sha256 of the given C++/CUDA sources with comments and whitespace
    removed: it changes with the code, not with its comments."""
    import hashlib
    import re
    h = hashlib.sha256()
    for name in paths:
        with open(os.path.join(ROOT, name)) as f:
            src = f.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update("".join(src.split()).encode())
    return h.hexdigest()


def captured_traffic(kernel: str, storage: str = "fp32", config: str = "c64"):
    """DRAM bytes per launch from the last ncu capture, if it was taken on this
    configuration and storage and the kernel code is unchanged since."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic_64cubed.json")) as f:
            rec = json.load(f)
        if kernel_source_digest(rec["kernel_sources"]) != rec["kernel_code_sha256"]:
            return None
        if storage != rec["storage"] or config != rec["config"]:
            return None
        return rec.get(kernel)
    except Exception:
        return None


def aggregate(dist, count: float, ms: float, device):
    """Whole-job figures over the ranks: (sum of the work counts, max of the
    times).  dist is torch.distributed (any backend) or None for one process."""
    if dist is None:
        return float(count), float(ms)
    import torch
    c = torch.tensor([float(count)], dtype=torch.float64, device=device)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(c.item()), float(t.item())


def gpu_id_for(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(dev)


def make_problem(cfg, rank):
    """Geometry, phantom and noise draw of this rank's problem (seeded inputs)."""
    import synth
    geom = cfg.geometry()
    x_true = synth.ellipsoid_phantom(cfg.n, cfg.ellipsoids, cfg.semi_axes, cfg.values,
                                     cfg.seed + 100 * rank)
    z = synth.standard_normal(geom.m, cfg.seed + 1000 + 100 * rank)
    return geom, x_true, z


def bench_config(cfg, eps, nnz, storage, graph, world):
    """The `config` of the bench line; both arms print the same dict."""
    return {"workload": workload(cfg, eps), "n": cfg.n, "views": cfg.views, "det": cfg.det,
            "m": cfg.views * cfg.det * cfg.det, "N": cfg.n ** 3, "nnz": int(nnz),
            "alpha": cfg.alpha, "tau": cfg.tau, "eps": eps, "stop": "relative gradient-map norm",
            "methods": ["gpbb", "upn"], "l2": l2_note(nnz), "passes_as_graphs": bool(graph),
            "storage": storage, "parallelism": f"{world} independent problems (one per GPU)"}


DATA_NOTE = ("b = A x_true + e, e = 0.01 ||A x_true|| / sqrt(m) z (z seeded standard normal), "
             "rounded to float32; each arm forms A x_true with its own projector (the GPU arm "
             "in float32 on the device, the CPU oracle in float64), so the two b agree to float32 "
             "rounding")


# ------------------------------------------------------------ reference arm
def run_reference(args, cfg, eps):
    """FP64 CPU oracle on the same workload; each step a bounded sample."""
    import numpy as np
    import oracle
    geom, x_true, z = make_problem(cfg, 0)
    A = oracle.system_matrix(geom)
    b = oracle.make_data(A, x_true, z, cfg.noise)
    prob = oracle.Problem(A=A, b=b, n=cfg.n, alpha=cfg.alpha, tau=cfg.tau)
    x0 = np.zeros(prob.N)
    k_sample = 3

    def step():
        g = 0
        for fn in (oracle.solve_gpbb, oracle.solve_upn):
            r = fn(prob, x0, eps, oracle.Options(k_max=k_sample))
            g += r.g_evals
        return g

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    evals = sum(step() for _ in range(args.steps))
    dt = time.perf_counter() - t0
    v = evals / dt
    world = int(os.environ.get("WORLD_SIZE", "1"))
    sample = (f"GPBB and UPN, first {k_sample} iterations each from x0 = 0 on the full "
              f"{cfg.n}^3 problem, per step ({evals} gradient evaluations in {dt:.1f} s, FP64 "
              f"numpy/scipy, one thread of {os.cpu_count()})")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "data_note": DATA_NOTE,
        "config": bench_config(cfg, eps, A.nnz, args.storage, args.graph, world),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "nproc": os.cpu_count(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def cpu_baseline_leg(args, cfg, eps):
    """Run in a child process (no CUDA): the oracle as it stands solving the
    bench problem to eps with GPBB and with UPN from x0 = 0, with the b the GPU
    arm used (read from --cpu-baseline-b).  Prints one JSON object."""
    import numpy as np
    import oracle
    geom, _, _ = make_problem(cfg, 0)
    b = np.load(args.cpu_baseline_b).astype(np.float64)
    A = oracle.system_matrix(geom)
    prob = oracle.Problem(A=A, b=b, n=cfg.n, alpha=cfg.alpha, tau=cfg.tau)
    x0 = np.zeros(prob.N)
    out = {}
    g_total, t_total = 0, 0.0
    for name, fn in (("gpbb", oracle.solve_gpbb), ("upn", oracle.solve_upn)):
        t0 = time.perf_counter()
        r = fn(prob, x0, eps, oracle.Options(k_max=args.cpu_baseline_kmax))
        dt = time.perf_counter() - t0
        out[name] = {"status": r.status, "iters": r.iters, "g_evals": r.g_evals,
                     "f_evals": r.f_evals, "s": dt}
        g_total += r.g_evals
        t_total += dt
    print(json.dumps({"evals": g_total, "s": t_total, "solves": out, "nproc": os.cpu_count()}),
          flush=True)


def cpu_baseline(cfg, eps, b_host, storage):
    """The oracle as it stands, timed in a child process on the host cores:
    one GPBB and one UPN solve of the bench problem to eps (time-to-eps, FP64
    numpy/scipy, one thread)."""
    import tempfile
    import numpy as np
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "b.npy")
        np.save(path, b_host)
        cmd = [sys.executable, os.path.abspath(__file__), "--config", cfg.name, "--eps", repr(eps),
               "--storage", storage, "--cpu-baseline-b", path]
        env = dict(os.environ)
        for v in ("RANK", "WORLD_SIZE", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT"):
            env.pop(v, None)
        env["CUDA_VISIBLE_DEVICES"] = ""
        p = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=900)
    if p.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"failed: {p.stderr.strip()[-300:]}"}
    rec = json.loads(p.stdout.strip().splitlines()[-1])
    sv = rec["solves"]
    return {"value": rec["evals"] / rec["s"], "unit": UNIT, "cores": 1, "nproc": rec["nproc"],
            "kind": "oracle",
            "time_to_eps": {"gpbb_s": sv["gpbb"]["s"], "upn_s": sv["upn"]["s"],
                            "gpbb_iters": sv["gpbb"]["iters"], "upn_iters": sv["upn"]["iters"],
                            "status": [sv["gpbb"]["status"], sv["upn"]["status"]]},
            "sample": f"one GPBB and one UPN solve of the same {cfg.n}^3 problem to eps from "
                      f"x0 = 0 with the GPU arm's b ({rec['evals']} gradient evaluations in "
                      f"{rec['s']:.1f} s; FP64 numpy/scipy, one thread of {rec['nproc']}; child "
                      f"process)"}


# ------------------------------------------------------------- autograd
def run_autograd(args, emit=True):
    """phi(x; b) forward + backward (torch.autograd) on the 128^3 / 60-view / 192^2 problem;
    returns the record (and prints it with emit)."""
    import numpy as np
    import torch
    import synth
    import __graft_entry__
    __graft_entry__.build()
    import paper_1105_4002_gb300 as tvr
    from paper_1105_4002_gb300.autograd import phi
    cfg = synth.get_config("c128")
    geom = cfg.geometry()
    dev = torch.device("cuda", 0)
    t0 = time.perf_counter()
    sysm = tvr.System(geom)
    torch.cuda.synchronize()
    build_ms = 1e3 * (time.perf_counter() - t0)
    xt = torch.tensor(cfg.phantom(), dtype=torch.float32, device=dev)
    ax = torch.empty(geom.m, dtype=torch.float32, device=dev)
    sysm.forward(xt, ax)
    axh = ax.cpu().numpy().astype(np.float64)
    z = synth.standard_normal(geom.m, cfg.seed + 1000)
    b = torch.tensor((axh + cfg.noise * np.linalg.norm(axh) / math.sqrt(geom.m) * z)
                     .astype(np.float32), device=dev, requires_grad=True)
    x = torch.rand(geom.N, device=dev, requires_grad=True)

    def step():
        x.grad = None
        b.grad = None
        phi(x, b, sysm, cfg.alpha, cfg.tau).backward()

    for _ in range(args.warmup):
        step()
    sysm.profile(True)
    sysm.profile_read()
    sampler = ClockSampler(gpu_id_for(torch, dev))
    torch.cuda.synchronize()
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    prof = sysm.profile_read()
    sysm.profile(False)
    ms = e0.elapsed_time(e1) / args.steps
    m, N, nnz = geom.m, geom.N, sysm.nnz
    bytes_f = 8 * nnz + 8 * (m + 1) + 4 * N + 8 * m
    bytes_b = 8 * nnz + 8 * (N + 1) + 8 * N + 8 * m
    (nf, msf), (nb, msb) = prof["forward"], prof["backward"]
    peak, src = measured_peak_gbs()
    name, mst, cnt, by = max([("fwd_csr", msf, nf, bytes_f), ("vjp_csc_tv", msb, nb, bytes_b)],
                             key=lambda c: c[1])
    ach = by / (mst / cnt / 1e3) / 1e9
    rec = {
        "metric": "phi forward+backward (autograd) evals/s at 128^3", "value": 1e3 / ms,
        "unit": "fwd+bwd/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "TV-CT 128^3, cone beam 60 views x 192^2 px, 20 ellipsoids, 0.5% noise; "
                               "phi(x; b) forward and backward through torch.autograd",
                   "nnz": nnz, "build_system_ms": build_ms,
                   "l2": "inputs larger than L2: A = 2 x 3.0 GB"},
        "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                     "frac": ach / peak, "traffic": None, "kernel": name,
                     "avg_us": 1e3 * mst / cnt, "peak_source": src,
                     "fwd_us": 1e3 * msf / max(nf, 1), "bwd_us": 1e3 * msb / max(nb, 1)},
        "gpu_launches": 3 * args.steps,
        "clocks": clocks}
    if emit:
        print(json.dumps(rec), flush=True)
    return rec


# ------------------------------------------------------ paper experiment
# The experiment of the paper's Sec. IV as printed there (tests/golden/paper_printed_values.txt);
# tau is this implementation's smoothing (the paper does not print one).
PAPER_EXPERIMENT = {"n": 64, "views": (55, 19), "det": 91, "noise": 0.01, "alpha": 1e-2,
                    "tau": 1e-4, "eps": 1e-8, "phi_star_eps_factor": 1e-2,
                    "checkpoints": (10, 30, 100, 300, 1000, 2000)}


def run_paper(args):
    """The convergence comparison of the paper's Sec. IV on its scan shape: a
    64^3 volume, parallel beam with view directions spread evenly over the
    unit sphere, a many-view (55) and a few-view (19) scan of 91^2 pixels,
    Gaussian noise of relative magnitude exactly 0.01, alpha = 0.01, and the
    per-voxel gradient-map stop ||G||/N <= eps = 1e-8.  phi* comes from UPN at
    eps/100 (below the float32 floor of ||G||, so capped at 20000
    iterations).  The phantom is the seeded ellipsoid stand-in (the paper's
    head phantom is not available).  Reported per scan and method: iterations
    and time to eps, and (phi_k - phi*)/phi* after k = 10 ... 2000 iterations
    (phi_k from the solver's history) with the first k below 1e-2, 1e-4, 1e-6."""
    import numpy as np
    import torch
    import synth
    import __graft_entry__
    __graft_entry__.build()
    import paper_1105_4002_gb300 as tvr
    from paper_1105_4002_gb300 import SolveOptions
    from paper_1105_4002_gb300._capi import TVR_STOP_PER_N
    dev = torch.device("cuda", 0)
    P = PAPER_EXPERIMENT
    n, det, alpha, tau, eps = P["n"], P["det"], P["alpha"], P["tau"], P["eps"]
    checkpoints = list(P["checkpoints"])
    x_true = synth.ellipsoid_phantom(n, 10, (4.0, 20.0), (0.0, 1.0), 6)
    results = {}
    sampler = ClockSampler(gpu_id_for(torch, dev))
    sampler.start()
    t_all = time.perf_counter()
    for label, views in ((f"many_view_{P['views'][0]}", P["views"][0]),
                         (f"few_view_{P['views'][1]}", P["views"][1])):
        geom = synth.sphere_parallel_geometry(n, views, det)
        s = tvr.System(geom)
        xt = torch.tensor(x_true, dtype=torch.float32, device=dev)
        ax = torch.empty(geom.m, dtype=torch.float32, device=dev)
        s.forward(xt, ax)
        axh = ax.cpu().numpy().astype(np.float64)
        e = synth.noise_exact(axh, synth.standard_normal(geom.m, 600 + views), P["noise"])
        b = torch.tensor((axh + e).astype(np.float32), device=dev)

        def phi_of(x):
            return s.phi_and_grad(x, b, alpha, tau)[0]

        def solve(method, e_stop, k_max, history=0):
            x = torch.zeros(geom.N, device=dev)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = s.solve(method, b, alpha, tau, e_stop, x,
                        SolveOptions(stop_mode=TVR_STOP_PER_N, k_max=k_max, history=history),
                        raise_on_error=False)
            torch.cuda.synchronize()
            return r, x, 1e3 * (time.perf_counter() - t0)

        r_star, x_star, _ = solve("upn", eps * P["phi_star_eps_factor"], 20000)
        phi_star = phi_of(x_star)
        per = {"rows_m": geom.m, "unknowns_N": geom.N, "rows_below_unknowns": geom.m < geom.N,
               "phi_star": phi_star, "phi_star_upn_iters": r_star.iters,
               "phi_star_stop_per_voxel": r_star.stop_value}
        for method in ("gp", "gpbb", "upn"):
            r, x, ms = solve(method, eps, 20000)
            # phi(x^(k)) of every iteration from the solver's history (one 2000-iteration run)
            rh, _, _ = solve(method, 1e-30, 2000, history=2000)
            rel = (rh.history[:, 6] - phi_star) / phi_star
            curve = {str(k): float(rel[k - 1]) for k in checkpoints if k <= len(rel)}
            first = {f"{t:.0e}": (int(np.argmax(rel <= t)) + 1 if np.any(rel <= t) else None)
                     for t in (1e-2, 1e-4, 1e-6)}
            per[method] = {"iters_to_eps": r.iters, "status": r.status, "ms_to_eps": ms,
                           "f_evals": r.f_evals, "g_evals": r.g_evals,
                           "rel_phi_at_stop": (phi_of(x) - phi_star) / phi_star,
                           "rel_phi_after_k": curve, "first_k_with_rel_phi_below": first}
        results[label] = per
        del s
        torch.cuda.empty_cache()
    clocks = sampler.stop()
    value = results["few_view_19"]["upn"]["first_k_with_rel_phi_below"]["1e-06"]
    print(json.dumps({
        "metric": "iterations until (phi_k - phi*)/phi* <= 1e-6, UPN, few-view 64^3 "
                  "(paper Sec. IV comparison)",
        "value": value, "unit": "iterations", "n_gpus": 1, "steps": 1, "warmup": 0,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "64^3, parallel beam, view directions on a golden-angle spiral over "
                               "the unit sphere, 55 and 19 views of 91^2 px, 10 seeded ellipsoids, "
                               "noise 0.01 relative, alpha 1e-2, tau 1e-4, eps 1e-8 per voxel",
                   "wall_s": time.perf_counter() - t_all},
        "results": results, "clocks": clocks}), flush=True)


# ------------------------------------------------------------- batching
def solver_launch_bytes(m: int, N: int, nnz: int, storage: str, method: str):
    """Algorithmic bytes of one working launch of the solver's two kernels,
    (back projection, trial), each stream counted once: int32 indices, int64
    pointers, float32 values (or bfloat16 plus a float32 scale per row and a
    scaled residual)."""
    vb = 4 if storage == "fp32" else 2
    extra_m = 0 if storage == "fp32" else 8
    # back projection: A^T (values + indices), column pointers, r gather, the
    # four Huber weight planes, x read and g and (p, g) written; GPBB also
    # reads x and g of the previous iterate for the BB dots
    bwd = (4 + vb) * nnz + 8 * (N + 1) + 4 * m + 16 * N + 4 * N + 4 * N + 8 * N
    if method == "gpbb":
        bwd += 8 * N
    # trial: A (values + indices), row pointers, the (p, g) pairs read and xbar
    # written, b read and r written; GPBB (two points per pass) writes the four
    # Huber weight planes at both points and the second point's xbar and
    # residual; UPN reads u and x and writes u, A y - b, y and the planes at y
    # (the extrapolation for the case of acceptance); GP writes the planes at xbar
    fwd = (4 + vb) * nnz + 8 * (m + 1) + 8 * N + 4 * N + 2 * 4 * m + extra_m * m
    fwd += {"gpbb": 16 * N + 4 * m + 20 * N, "upn": 12 * m + 24 * N, "gp": 16 * N}[method]
    return bwd, fwd


def trial_bytes(m: int, N: int, nnz: int, storage: str, method: str) -> float:
    """Algorithmic bytes of one working trial launch, per unit as the scope
    table's measurement row counts them: the f-only trial 8 nnz + 12 m + 8 N
    (values and indices of A, b read and r written and gathered, the gathered
    point), 12 B per voxel for the projected step (A5) and, in UPN, 12 B per
    voxel for the extrapolation (A8).  BF16 storage: 6 B per entry."""
    per_entry = 8 if storage == "fp32" else 6
    b = per_entry * nnz + 12 * m + 8 * N + 12 * N
    if method == "upn":
        b += 12 * N
    return float(b)


def backprojection_bytes(m: int, N: int, nnz: int, storage: str) -> float:
    """Algorithmic bytes of one working back projection: A^T (8 B per entry,
    6 with BF16 values), r read, x read and g written."""
    per_entry = 8 if storage == "fp32" else 6
    return float(per_entry * nnz + 4 * m + 8 * N)


def plain_launch_bytes(m: int, N: int, nnz: int, storage: str):
    """Algorithmic bytes of the plain phi + grad phi kernels, (forward, back
    projection): r = A x - b with x gathered and b read, r written; g = A^T r +
    alpha grad TV with r gathered, x read (TV stencil) and g written."""
    vb = 4 if storage == "fp32" else 2
    extra_m = 0 if storage == "fp32" else 8
    fwd = (4 + vb) * nnz + 8 * (m + 1) + 4 * N + 8 * m + extra_m * m
    bwd = (4 + vb) * nnz + 8 * (N + 1) + 4 * m + 8 * N
    return fwd, bwd


def batch_problems(count=48, seed=5):
    """Uneven problems: edge U{24..96}, views U{8..40}, detector 1.5 x edge (seeded)."""
    import numpy as np
    import synth
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(24, 97))
        v = int(rng.integers(8, 41))
        p = int(round(1.5 * n))
        g = synth.cone_geometry(n, v, p, 3.0 * n, 2.0 * n)
        x_true = synth.ellipsoid_phantom(n, 10, (n / 16, n / 3.2), (0.0, 1.0), 5000 + i)
        z = synth.standard_normal(g.m, 6000 + i)
        out.append((g, x_true, z))
    return out


def run_batch(args, emit=True, storages=("fp32", "bf16", "u16"), sweep=True):
    """solves/s to eps: 48 uneven problems batched vs one by one; 8-alpha sweep at 128^3;
    returns the record (and prints it with emit)."""
    import numpy as np
    import torch
    import synth
    import __graft_entry__
    __graft_entry__.build()
    import paper_1105_4002_gb300 as tvr
    dev = torch.device("cuda", 0)
    eps, alpha, tau = 1e-4, 1e-2, 1e-4
    res = {}

    def make_b(sysm, x_true, z, level):
        xt = torch.tensor(x_true, dtype=torch.float32, device=dev)
        ax = torch.empty(sysm.m, dtype=torch.float32, device=dev)
        sysm.forward(xt, ax)
        axh = ax.cpu().numpy().astype(np.float64)
        return torch.tensor((axh + level * np.linalg.norm(axh) / math.sqrt(sysm.m) * z)
                            .astype(np.float32), device=dev)

    probs = batch_problems()
    for storage in storages:
        systems = [tvr.System(g, storage=storage) for g, _, _ in probs]
        bs = [make_b(s_, xt, z, 0.01) for s_, (g, xt, z) in zip(systems, probs)]
        xs = [torch.zeros(s_.N, device=dev) for s_ in systems]
        al = [alpha] * len(systems)
        tvr.solve_batch("upn", systems, bs, al, tau, eps, xs)          # warm-up (graphs, buffers)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            for x in xs:
                x.zero_()
            rb = tvr.solve_batch("upn", systems, bs, al, tau, eps, xs)
        torch.cuda.synchronize()
        t_batch = (time.perf_counter() - t0) / args.steps
        t0 = time.perf_counter()
        alone = []  # each problem solved alone, with the whole GPU (the call synchronises)
        for s_, b, x in zip(systems, bs, xs):
            t1 = time.perf_counter()
            s_.solve("upn", b, alpha, tau, eps, x.zero_())
            alone.append(time.perf_counter() - t1)
        torch.cuda.synchronize()
        t_seq = time.perf_counter() - t0
        moved = 0.0  # algorithmic bytes of the launches that did work (a trial per f-eval)
        per_bytes = []
        for s_, r in zip(systems, rb):
            bb, bf = solver_launch_bytes(s_.m, s_.N, s_.nnz, storage, "upn")
            per_bytes.append(r.g_evals * bb + r.f_evals * bf)
            moved += per_bytes[-1]
        peak, _ = measured_peak_gbs()
        # Lower bound of any schedule of these solves on these kernels: no
        # problem finishes before it does alone (its passes are a chain), and
        # the bytes cannot move faster than the best rate any problem reaches
        # alone.
        best_rate = max(w / t for w, t in zip(per_bytes, alone))
        bound = max(max(alone), moved / best_rate)
        order = sorted(range(len(systems)), key=lambda i: -alone[i])
        schedule_bound = {
            "sum_alone_s": sum(alone), "max_alone_s": max(alone),
            "best_alone_rate_gbs": best_rate / 1e9, "bytes_over_best_rate_s": moved / best_rate,
            "lower_bound_s": bound, "batch_over_lower_bound": t_batch / bound,
            "largest_alone": [{"n": systems[i].n,
                               "m": systems[i].m, "nnz": systems[i].nnz, "alone_s": alone[i],
                               "gbs_alone": per_bytes[i] / alone[i] / 1e9} for i in order[:6]]}
        res[f"batch48_{storage}"] = {
            "solves_per_s": len(systems) / t_batch, "ms": 1e3 * t_batch,
            "algorithmic_gb": moved / 1e9, "achieved_gbs": moved / t_batch / 1e9,
            "frac_of_measured_hbm": moved / t_batch / 1e9 / peak,
            "one_by_one_solves_per_s": len(systems) / t_seq,
            "converged": sum(r.status == 0 for r in rb), "iters_total": sum(r.iters for r in rb),
            "schedule_bound": schedule_bound}
        del systems, bs, xs
        torch.cuda.empty_cache()

    cfg = synth.get_config("c128")
    alphas = list(np.logspace(-4, -1, 8))
    for storage in (storages if sweep else ()):
        sysm = tvr.System(cfg.geometry(), storage=storage)
        b = make_b(sysm, cfg.phantom(), synth.standard_normal(sysm.m, cfg.seed + 1000), cfg.noise)
        X = torch.zeros(8 * sysm.N, device=dev)
        sysm.solve_sweep("upn", b, alphas, tau, eps, X)                # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rs = sysm.solve_sweep("upn", b, alphas, tau, eps, X.zero_())
        torch.cuda.synchronize()
        t_sw = time.perf_counter() - t0
        x1 = torch.zeros(sysm.N, device=dev)
        sysm.solve("upn", b, alphas[0], tau, eps, x1)                    # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        its = []
        for a in alphas:
            its.append(sysm.solve("upn", b, a, tau, eps, x1.zero_()).iters)
        torch.cuda.synchronize()
        t_single = time.perf_counter() - t0
        res[f"sweep8_128cubed_{storage}"] = {
            "solves_per_s": 8 / t_sw, "ms": 1e3 * t_sw, "single_solves_per_s": 8 / t_single,
            "converged": sum(r.status == 0 for r in rs), "iters": [r.iters for r in rs],
            "lanes_rows_cols": list(rs[0].lanes),
            "single_iters": its}
        del sysm, X
        torch.cuda.empty_cache()
    rec = {
        "metric": "solves/s to eps=1e-4 (UPN): 48 uneven problems batched; 8-alpha sweep at 128^3",
        "value": res["batch48_fp32"]["solves_per_s"], "unit": "solves/s", "n_gpus": 1,
        "steps": args.steps, "warmup": 1, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "48 problems: edge U{24..96}, views U{8..40}, detector 1.5 edge, "
                               "10 ellipsoids, 1% noise; sweep: 128^3 / 60 views / 192^2, "
                               "alphas 1e-4..1e-1 log-spaced", "alpha": alpha, "tau": tau,
                   "eps": eps},
        "results": res}
    if emit:
        print(json.dumps(rec), flush=True)
    return rec


def run_grid(args):
    """The 64^3 problem solved by GP, GPBB and UPN for every alpha in {1e-3,
    1e-2, 1e-1}, tau in {1e-2, 1e-4} and eps in {1e-4, 1e-6} (relative
    gradient-map stop), from x0 = 0 on the same data.  Reported per case:
    status, iterations, gradient and objective evaluations, time to eps and
    gradient evaluations per second."""
    import math
    import numpy as np
    import torch
    import synth
    import __graft_entry__
    __graft_entry__.build()
    import paper_1105_4002_gb300 as tvr
    cfg = synth.get_config(args.config)
    dev = torch.device("cuda", 0)
    geom, x_true, z = make_problem(cfg, 0)
    sysm = tvr.System(geom, storage=args.storage)
    xt = torch.tensor(x_true, dtype=torch.float32, device=dev)
    ax = torch.empty(sysm.m, device=dev)
    sysm.forward(xt, ax)
    axh = ax.cpu().numpy().astype(np.float64)
    b = torch.tensor((axh + cfg.noise * np.linalg.norm(axh) / math.sqrt(sysm.m) * z)
                     .astype(np.float32), device=dev)
    x = torch.zeros(sysm.N, device=dev)
    sysm.solve("upn", b, cfg.alpha, cfg.tau, 1e-4, x)          # warm-up (graphs, buffers)
    cases = []
    total_evals, total_ms = 0, 0.0
    for method in ("gp", "gpbb", "upn"):
        for alpha in (1e-3, 1e-2, 1e-1):
            for tau in (1e-2, 1e-4):
                for eps in (1e-4, 1e-6):
                    x.zero_()
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    r = sysm.solve(method, b, alpha, tau, eps, x)
                    torch.cuda.synchronize()
                    ms = 1e3 * (time.perf_counter() - t0)
                    cases.append({"method": method, "alpha": alpha, "tau": tau, "eps": eps,
                                  "status": r.status, "iters": r.iters, "g_evals": r.g_evals,
                                  "f_evals": r.f_evals, "ms": ms,
                                  "grad_evals_per_s": r.g_evals / (ms / 1e3)})
                    total_evals += r.g_evals
                    total_ms += ms
    print(json.dumps({
        "metric": "gradient evaluations/s and time to eps over the GP/GPBB/UPN x alpha x tau x eps "
                  "grid at 64^3", "value": total_evals / (total_ms / 1e3),
        "unit": "grad-phi evals/s", "n_gpus": 1, "steps": 1, "warmup": 1,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": dtype_of(args.storage),
        "data": "synthetic",
        "config": {"workload": workload(cfg, cfg.eps), "n": cfg.n, "views": cfg.views,
                   "det": cfg.det, "storage": args.storage, "k_max": 20000},
        "converged": sum(c["status"] == 0 for c in cases), "cases": cases}), flush=True)


def run_precision(args):
    """The storage-precision configuration: 256^3, 90 cone-beam views, 384^2
    detector, 40 ellipsoids, 1% noise, alpha 1e-2, tau 1e-4; GPBB and UPN to
    eps = 1e-5 (relative gradient-map stop) with A stored as FP32, as BF16
    codes with per-row FP32 scales, and matrix-free.  The data b comes from the
    FP32 system.  Reported per storage: build time, and per method the
    iterations, time to eps, gradient evaluations/s and the relative L2
    distance of x* from the FP32 storage's x*.  (Errors against the FP64
    oracle per stage at this size: tests/test_gpu_precision.py with
    TVR_PRECISION_FULL=1; the oracle cannot solve at this size.)"""
    import numpy as np
    import torch
    import synth
    import __graft_entry__
    __graft_entry__.build()
    import paper_1105_4002_gb300 as tvr
    cfg = synth.get_config("c256" if args.config == "c64" else args.config)
    dev = torch.device("cuda", 0)
    geom, x_true, z = make_problem(cfg, 0)
    b = None
    ref = {}
    out = {}
    opts = tvr.SolveOptions(k_max=5000)
    for storage in ("fp32", "bf16", "u16", "mf"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sysm = tvr.System(geom, storage=storage)
        torch.cuda.synchronize()
        rec = {"build_ms": 1e3 * (time.perf_counter() - t0), "nnz": sysm.nnz}
        if b is None:
            xt = torch.tensor(x_true, dtype=torch.float32, device=dev)
            ax = torch.empty(sysm.m, device=dev)
            sysm.forward(xt, ax)
            axh = ax.cpu().numpy().astype(np.float64)
            b = torch.tensor((axh + cfg.noise * np.linalg.norm(axh) / math.sqrt(sysm.m) * z)
                             .astype(np.float32), device=dev)
            del xt, ax
        x = torch.zeros(sysm.N, device=dev)
        for method in ("gpbb", "upn"):
            x.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = sysm.solve(method, b, cfg.alpha, cfg.tau, cfg.eps, x, opts)
            torch.cuda.synchronize()
            ms = 1e3 * (time.perf_counter() - t0)
            xs = x.cpu().numpy().astype(np.float64)
            m_rec = {"status": r.status, "iters": r.iters, "g_evals": r.g_evals, "ms": ms,
                     "grad_evals_per_s": r.g_evals / (ms / 1e3), "phi": r.phi}
            if storage == "fp32":
                ref[method] = xs
            else:
                m_rec["rel_l2_to_fp32_xstar"] = float(np.linalg.norm(xs - ref[method])
                                                      / np.linalg.norm(ref[method]))
            rec[method] = m_rec
        out[storage] = rec
        del sysm, x
        torch.cuda.empty_cache()
    print(json.dumps({
        "metric": "time to eps = 1e-5 (GPBB, UPN) at 256^3 with A stored as FP32, BF16 and "
                  "matrix-free", "value": out["fp32"]["upn"]["ms"], "unit": "ms (UPN, FP32)",
        "n_gpus": 1, "steps": 1, "warmup": 0, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"TV-CT {cfg.n}^3, cone beam {cfg.views} views x {cfg.det}^2 px, "
                               f"{cfg.ellipsoids} seeded ellipsoids, 1% noise, alpha {cfg.alpha}, "
                               f"tau {cfg.tau}, eps {cfg.eps}", "k_max": 5000},
        "results": out}), flush=True)


def run_sweep(args):
    """One 8-alpha UPN sweep (1e-4 .. 1e-1, log-spaced) sharing A at 128^3 /
    60 views / 192^2, FP32 storage, to eps = 1e-4 or --sweep-kmax iterations
    (a short run to profile the sweep's kernels); passes per second."""
    import numpy as np
    import torch
    import synth
    import __graft_entry__
    __graft_entry__.build()
    import paper_1105_4002_gb300 as tvr
    cfg = synth.get_config("c128")
    dev = torch.device("cuda", 0)
    sysm = tvr.System(cfg.geometry(), storage=args.storage)
    xt = torch.tensor(cfg.phantom(), dtype=torch.float32, device=dev)
    ax = torch.empty(sysm.m, device=dev)
    sysm.forward(xt, ax)
    axh = ax.cpu().numpy().astype(np.float64)
    z = synth.standard_normal(sysm.m, cfg.seed + 1000)
    b = torch.tensor((axh + cfg.noise * np.linalg.norm(axh) / math.sqrt(sysm.m) * z)
                     .astype(np.float32), device=dev)
    X = torch.zeros(8 * sysm.N, device=dev)
    opts = tvr.SolveOptions(k_max=args.sweep_kmax)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rs = sysm.solve_sweep("upn", b, list(np.logspace(-4, -1, 8)), cfg.tau, 1e-4, X, opts)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    print(json.dumps({
        "metric": "passes/s of an 8-alpha UPN sweep at 128^3", "value": rs[0].passes / dt,
        "unit": "passes/s", "n_gpus": 1, "steps": 1, "warmup": 0, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "TV-CT 128^3, cone beam 60 views x 192^2 px, 20 ellipsoids, 0.5% "
                               "noise, alpha 1e-4 .. 1e-1 (8, log-spaced), tau 1e-4, eps 1e-4",
                   "k_max": args.sweep_kmax, "storage": args.storage, "nnz": sysm.nnz},
        "iters": [r.iters for r in rs], "passes": rs[0].passes, "ms": 1e3 * dt,
        "lanes_rows_cols": list(rs[0].lanes)}), flush=True)


def run_projectors(args):
    """Forward projection y = A x and adjoint z = A^T r alone (tvr_forward,
    tvr_adjoint) for the storage of --storage on the scan of --config, each
    timed with CUDA events over --steps launches after --warmup; FP32 storage
    is timed beside it for comparison."""
    import numpy as np
    import torch
    import synth
    import __graft_entry__
    __graft_entry__.build()
    import paper_1105_4002_gb300 as tvr
    cfg = synth.get_config(args.config)
    geom = cfg.geometry()
    out = {}
    for storage in dict.fromkeys([args.storage, "fp32"]):
        s = tvr.System(geom, storage=storage)
        x = torch.tensor(np.random.default_rng(1).uniform(0, 1, s.N), dtype=torch.float32,
                         device="cuda")
        r = torch.tensor(np.random.default_rng(2).standard_normal(s.m), dtype=torch.float32,
                         device="cuda")
        y = torch.empty(s.m, device="cuda")
        z = torch.empty(s.N, device="cuda")

        def timed(fn):
            for _ in range(max(args.warmup, 1)):
                fn()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.steps):
                fn()
            e1.record()
            torch.cuda.synchronize()
            return 1e3 * e0.elapsed_time(e1) / args.steps

        fwd = timed(lambda: s.forward(x, y))
        adj = timed(lambda: s.adjoint(r, z))
        out[storage] = {"forward_us": fwd, "adjoint_us": adj, "rays_per_s": s.m / (fwd / 1e6),
                        "voxel_views_per_s": s.N * cfg.views / (adj / 1e6)}
        del s
        torch.cuda.empty_cache()
    print(json.dumps({
        "metric": f"forward and adjoint projection time, {args.storage} storage",
        "value": out[args.storage]["forward_us"] + out[args.storage]["adjoint_us"],
        "unit": "us (forward + adjoint)", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": {"workload": workload(cfg, cfg.eps), "storage": args.storage},
        "results": out}), flush=True)


def storage_comparison(args, cfg, eps, geom, b, sys_fp32, value_fp32):
    """The same step (one GPBB and one UPN solve to eps on the same b) with A
    stored as 16-bit codes, after the FP32 timing: gradient evaluations per
    second, their ratio to the FP32 value, and the relative L2 distance of each
    x* from the FP32 solve's."""
    import numpy as np
    import torch
    import paper_1105_4002_gb300 as tvr
    out = {}
    ref = {}
    for m in ("gpbb", "upn"):  # the FP32 solutions, solved again here
        x = torch.zeros(geom.N, dtype=torch.float32, device=b.device)
        sys_fp32.solve(m, b, cfg.alpha, cfg.tau, eps, x,
                       tvr.SolveOptions(use_graph=bool(args.graph)))
        ref[m] = x.cpu().numpy()
    for storage in ("bf16", "u16"):
        try:
            s16 = tvr.System(geom, storage=storage)
            xg = torch.zeros(geom.N, dtype=torch.float32, device=b.device)
            xu = torch.zeros(geom.N, dtype=torch.float32, device=b.device)
            opts = tvr.SolveOptions(use_graph=bool(args.graph))
            for _ in range(2):
                s16.solve("gpbb", b, cfg.alpha, cfg.tau, eps, xg.zero_(), opts)
                s16.solve("upn", b, cfg.alpha, cfg.tau, eps, xu.zero_(), opts)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            steps = max(min(args.steps, 10), 1)
            evals = 0
            e0.record()
            for _ in range(steps):
                r1 = s16.solve("gpbb", b, cfg.alpha, cfg.tau, eps, xg.zero_(), opts)
                r2 = s16.solve("upn", b, cfg.alpha, cfg.tau, eps, xu.zero_(), opts)
                evals += r1.g_evals + r2.g_evals
            e1.record()
            torch.cuda.synchronize()
            v = evals / (e0.elapsed_time(e1) / 1e3)
            d = {m: float(np.linalg.norm(x.cpu().numpy() - ref[m]) / np.linalg.norm(ref[m]))
                 for m, x in (("gpbb", xg), ("upn", xu))}
            out[storage] = {"value": v, "unit": UNIT, "ratio_to_fp32": v / value_fp32,
                            "steps": steps, "gpbb_iters": r1.iters, "upn_iters": r2.iters,
                            "xstar_rel_l2_to_fp32": d, "dtype": dtype_of(storage)}
            del s16
        except Exception as e:  # noqa: BLE001 -- reported, not raised
            out[storage] = {"error": f"{type(e).__name__}: {e}"[:300]}
    return out


def other_configs():
    """Short runs of two other configurations, after the main line's timing,
    so that one default run records them too: phi forward + backward through
    torch.autograd at 128^3 (10 timed steps) and the 48-problem FP32 batch
    (one batched solve, then every problem alone, with the schedule bound).
    A failure is recorded in place of the numbers."""
    import types
    out = {}
    try:
        r = run_autograd(types.SimpleNamespace(steps=10, warmup=3), emit=False)
        out["autograd_128cubed"] = {
            "value": r["value"], "unit": r["unit"], "ms_per_step": r["ms_per_step"],
            "roofline_frac": r["roofline"]["frac"], "roofline_kernel": r["roofline"]["kernel"],
            "workload": r["config"]["workload"]}
    except Exception as e:  # noqa: BLE001 -- reported, not raised
        out["autograd_128cubed"] = {"error": f"{type(e).__name__}: {e}"[:300]}
    try:
        r = run_batch(types.SimpleNamespace(steps=1), emit=False, storages=("fp32",), sweep=False)
        b = r["results"]["batch48_fp32"]
        out["batch48_fp32"] = {
            "value": b["solves_per_s"], "unit": "solves/s to eps = 1e-4 (UPN)",
            "one_by_one_solves_per_s": b["one_by_one_solves_per_s"],
            "converged": b["converged"],
            "batch_over_schedule_lower_bound": b["schedule_bound"]["batch_over_lower_bound"],
            "workload": r["config"]["workload"]}
    except Exception as e:  # noqa: BLE001 -- reported, not raised
        out["batch48_fp32"] = {"error": f"{type(e).__name__}: {e}"[:300]}
    return out


# ------------------------------------------------------------------ our arm
def main():
    args = parse()
    import synth
    cfg = synth.get_config(args.config)
    eps = args.eps if args.eps is not None else cfg.eps
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.cpu_baseline_b:
        cpu_baseline_leg(args, cfg, eps)
        return
    if args.impl == "reference":
        if rank == 0:
            run_reference(args, cfg, eps)
        return
    if args.pattern == "autograd":
        if rank == 0:
            run_autograd(args)
        return
    if args.pattern == "batch":
        if rank == 0:
            run_batch(args)
        return
    if args.pattern == "paper":
        if rank == 0:
            run_paper(args)
        return
    if args.pattern == "grid":
        if rank == 0:
            run_grid(args)
        return
    if args.pattern == "precision":
        if rank == 0:
            run_precision(args)
        return
    if args.pattern == "sweep":
        if rank == 0:
            run_sweep(args)
        return
    if args.pattern == "projectors":
        if rank == 0:
            run_projectors(args)
        return

    import numpy as np
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if dist:
        dist.barrier()
    import paper_1105_4002_gb300 as tvr

    geom, x_true, z = make_problem(cfg, rank)
    t0 = time.perf_counter()
    sysm = tvr.System(geom, storage=args.storage)
    torch.cuda.synchronize()
    build_ms = 1e3 * (time.perf_counter() - t0)

    # data b = A x_true + e (forward projection on the GPU; noise from synth)
    xt = torch.tensor(x_true, dtype=torch.float32, device=dev)
    ax = torch.empty(geom.m, dtype=torch.float32, device=dev)
    sysm.forward(xt, ax)
    axh = ax.cpu().numpy().astype(np.float64)
    sigma = cfg.noise * np.linalg.norm(axh) / math.sqrt(geom.m)
    b_host = (axh + sigma * z).astype(np.float32)
    b = torch.tensor(b_host, device=dev)
    opts = tvr.SolveOptions(use_graph=bool(args.graph))

    def step(bb, x_gp, x_up):
        x_gp.zero_() if hasattr(x_gp, "zero_") else x_gp.fill(0)
        x_up.zero_() if hasattr(x_up, "zero_") else x_up.fill(0)
        r1 = sysm.solve("gpbb", bb, cfg.alpha, cfg.tau, eps, x_gp, opts)
        r2 = sysm.solve("upn", bb, cfg.alpha, cfg.tau, eps, x_up, opts)
        return r1, r2

    xg = torch.zeros(geom.N, dtype=torch.float32, device=dev)
    xu = torch.zeros(geom.N, dtype=torch.float32, device=dev)
    for _ in range(max(args.warmup, 0)):
        step(b, xg, xu)
    torch.cuda.synchronize()

    # ---- timed region (no kernel timing inside: the graphs replay as they are) ----
    sampler = ClockSampler(gpu_id_for(torch, dev))
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    evals = 0
    launches = 0
    passes_gpbb = passes_upn = 0
    t_gpbb, t_upn, it_gpbb, it_upn = [], [], [], []
    for _ in range(args.steps):
        s0 = time.perf_counter()
        r1 = sysm.solve("gpbb", b, cfg.alpha, cfg.tau, eps, xg.zero_(), opts)
        s1 = time.perf_counter()
        r2 = sysm.solve("upn", b, cfg.alpha, cfg.tau, eps, xu.zero_(), opts)
        s2 = time.perf_counter()
        t_gpbb.append(1e3 * (s1 - s0))
        t_upn.append(1e3 * (s2 - s1))
        it_gpbb.append(r1.iters)
        it_upn.append(r2.iters)
        evals += r1.g_evals + r2.g_evals
        passes_gpbb += r1.passes
        passes_upn += r2.passes
        # per solve: the initial phi and gradient (2), two kernels per pass
        # (back projection, trial), phi at x* (forward + TV value, 2)
        launches += (2 + 2 * r1.passes + 2) + (2 + 2 * r2.passes + 2)
    ev1.record()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    elapsed_ms = ev0.elapsed_time(ev1)

    # ---- roofline pass: the same solves again, after the timed region, with
    # CUDA event nodes around the trial and back-projection kernels of every
    # 4th pass (launches that did work only) ----
    sysm.profile(True, kinds=("forward", "backward"), sample_stride=4)
    sysm.profile_read()
    rp_gpbb = rp_upn = 0
    for _ in range(max(args.roofline_steps, 1)):
        rp_gpbb += sysm.solve("gpbb", b, cfg.alpha, cfg.tau, eps, xg.zero_(), opts).passes
        rp_upn += sysm.solve("upn", b, cfg.alpha, cfg.tau, eps, xu.zero_(), opts).passes
    prof = sysm.profile_read()
    sysm.profile(False)
    # per-kernel breakdown: one more step with every kernel timed
    sysm.profile(True)
    sysm.profile_read()
    sysm.solve("gpbb", b, cfg.alpha, cfg.tau, eps, xg.zero_(), opts)
    sysm.solve("upn", b, cfg.alpha, cfg.tau, eps, xu.zero_(), opts)
    breakdown = sysm.profile_read()
    sysm.profile(False)

    evals_all, elapsed_max = aggregate(dist, evals, elapsed_ms, dev)
    value = evals_all / (elapsed_max / 1e3)

    # ---- end-to-end through the public call with host buffers ----
    b_pin = torch.tensor(b_host).pin_memory()
    xg_h = torch.zeros(geom.N, dtype=torch.float32).pin_memory()
    xu_h = torch.zeros(geom.N, dtype=torch.float32).pin_memory()
    if dist:
        dist.barrier()
    e_evals = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r1 = sysm.solve("gpbb", b_pin, cfg.alpha, cfg.tau, eps, xg_h.zero_(), opts)
        r2 = sysm.solve("upn", b_pin, cfg.alpha, cfg.tau, eps, xu_h.zero_(), opts)
        e_evals += r1.g_evals + r2.g_evals
    e_ms = 1e3 * (time.perf_counter() - t0)
    e_all, e_max = aggregate(dist, e_evals, e_ms, dev)
    e2e_value = e_all / (e_max / 1e3)

    # ---- standalone phi_and_grad rate (same kernels, plain mode) ----
    xr = torch.tensor(np.random.default_rng(rank).uniform(0, 1, geom.N), dtype=torch.float32,
                      device=dev)
    g = torch.empty(geom.N, dtype=torch.float32, device=dev)
    phi_dev = torch.empty(4, dtype=torch.float64, device=dev)
    for _ in range(5):
        sysm.phi_and_grad(xr, b, cfg.alpha, cfg.tau, grad=g, phi_dev=phi_dev, sync=False)
    sysm.profile(True)
    sysm.profile_read()
    torch.cuda.synchronize()
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record()
    for _ in range(args.phi_loop):
        sysm.phi_and_grad(xr, b, cfg.alpha, cfg.tau, grad=g, phi_dev=phi_dev, sync=False)
    p1.record()
    torch.cuda.synchronize()
    phi_prof = sysm.profile_read()
    sysm.profile(False)
    phi_ms = p0.elapsed_time(p1) / args.phi_loop

    # ---- cost of a pass whose kernels return at once (after a rejected trial
    # no gradient is due; after the stop nothing is): UPN solves that stop at
    # their first iteration (eps = 1e30), in batches of 512 passes (511 of them
    # do nothing) against batches of 1 ----
    def noop_probe(batch, reps=20):
        o = tvr.SolveOptions(use_graph=bool(args.graph), batch=batch)
        sysm.solve("upn", b, cfg.alpha, cfg.tau, 1e30, xu.zero_(), o)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            sysm.solve("upn", b, cfg.alpha, cfg.tau, 1e30, xu.zero_(), o)
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps
    noop_pass_us = 1e6 * (noop_probe(512, 5) - noop_probe(1, 5)) / 511

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    m, N, nnz = geom.m, geom.N, sysm.nnz
    w_share = rp_gpbb / max(rp_gpbb + rp_upn, 1)
    bytes_fwd = w_share * trial_bytes(m, N, nnz, args.storage, "gpbb") + \
        (1 - w_share) * trial_bytes(m, N, nnz, args.storage, "upn")
    bytes_bwd = backprojection_bytes(m, N, nnz, args.storage)
    # DRAM bytes of the captured GPBB and UPN trial launches, mixed like bytes_fwd
    t_g = captured_traffic("fwd_csr_trial_gpbb", args.storage, args.config)
    t_u = captured_traffic("fwd_csr_trial_upn", args.storage, args.config)
    trial_traffic = (w_share * t_g + (1 - w_share) * t_u) if (t_g and t_u) else None
    bwd_traffic = captured_traffic("bwd_csc_tv", args.storage, args.config)
    peak, peak_kind = measured_peak_gbs()
    roof = None
    nf, msf = prof["forward"]
    nb, msb = prof["backward"]
    if nf and args.storage != "mf":  # matrix-free: ALU-bound, no matrix bytes to count
        avg_s = msf / nf / 1e3
        ach = bytes_fwd / avg_s / 1e9
        bk = {k: 1e3 * v[1] / v[0] for k, v in breakdown.items() if v[0]}
        roof = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "traffic": trial_traffic, "kernel": "fwd_csr_trial",
                "launches": nf, "avg_us": 1e6 * avg_s, "algorithmic_bytes_per_launch": bytes_fwd,
                "bytes_rule": "per unit as in the scope table's measurement row: f-only trial "
                              "8 nnz + 12 m + 8 N, plus 12 B per voxel for the projected step "
                              "and, in UPN, 12 B per voxel for the extrapolation",
                "peak_source": peak_kind,
                "timing": f"separate pass after the timed region ({max(args.roofline_steps, 1)} "
                          "steps): CUDA event nodes around the kernel in every 4th pass, "
                          "launches that did work only",
                "backprojection": ({"avg_us": 1e3 * msb / nb, "launches": nb,
                                    "algorithmic_bytes_per_launch": bytes_bwd,
                                    "achieved": bytes_bwd / (msb / nb / 1e3) / 1e9,
                                    "frac": bytes_bwd / (msb / nb / 1e3) / 1e9 / peak,
                                    "traffic": bwd_traffic} if nb else None),
                "breakdown_us": bk,
                "breakdown_note": "per-launch means of one extra step with every kernel timed "
                                  "(event nodes around each kernel slow the small ones); the "
                                  "projected step runs inside the trial forward kernel"}
    pf, pb = phi_prof["forward"], phi_prof["backward"]
    plain_f, plain_b = plain_launch_bytes(m, N, nnz, args.storage)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": dtype_of(args.storage), "data": "synthetic",
        "data_note": DATA_NOTE,
        "config": bench_config(cfg, eps, nnz, args.storage, args.graph, world),
        "time_to_eps": {"gpbb_ms": sorted(t_gpbb)[len(t_gpbb) // 2],
                        "upn_ms": sorted(t_upn)[len(t_upn) // 2],
                        "gpbb_iters": it_gpbb[-1], "upn_iters": it_upn[-1],
                        "build_system_ms": build_ms},
        "phi_and_grad": {"evals_per_s": 1e3 / phi_ms, "us_per_eval": 1e3 * phi_ms,
                         "fwd_us": 1e3 * pf[1] / max(pf[0], 1), "bwd_us": 1e3 * pb[1] / max(pb[0], 1),
                         "fwd_frac": plain_f / (pf[1] / max(pf[0], 1) / 1e3) / 1e9 / peak if pf[0] else None,
                         "bwd_frac": plain_b / (pb[1] / max(pb[0], 1) / 1e3) / 1e9 / peak if pb[0] else None},
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": 2 * 4 * (m + N), "d2h_bytes_per_step": 2 * 4 * N},
        "gpu_launches": launches,
        "noop_pass_us": noop_pass_us,
        "passes_per_step": (passes_gpbb + passes_upn) / args.steps,
        "iterations_per_step": (sum(it_gpbb) + sum(it_upn)) / args.steps,
        "clocks": clocks,
    }
    if world == 1 and not args.no_other_configs and args.storage == "fp32":
        line["vs_plain_fp32"] = storage_comparison(args, cfg, eps, geom, b, sysm, value)
    if world == 1 and not args.no_other_configs:
        line["other_configs"] = other_configs()
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg, eps, b_host, args.storage)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

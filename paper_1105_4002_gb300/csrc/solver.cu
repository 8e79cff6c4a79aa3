// GP / GPBB / UPN drivers.
//
// A solve is a sequence of identical "passes" (kernels.cu, launch_solver_pass):
//   gradient at the newly accepted point (back projection)
//   -> trial kernel (projected step, forward projection, acceptance test;
//      UPN's extrapolation for the case of acceptance, or GPBB's second
//      trial point).
// Kernels whose work is not due (no new point yet, or the solve has stopped)
// return at once after reading the device state, so the host never needs to
// know the outcome of a line-search trial: it launches passes in batches --
// replayed as one CUDA graph -- and reads a single "done" flag per batch.
// Every data-dependent loop of the method is bounded on the device (k_max,
// the trial caps), and the number of batches is bounded on the host.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "system.cuh"

namespace {

int ensure_solver(tvr_system *sys, int64_t hist_records) {
  for (auto &p : sys->vN)
    if (int rc = ensure_vec(&p, sys->N)) return rc;
  const int nm = coded16(sys->A.storage) ? RM_COUNT : RM_RS;
  for (int k = 0; k < nm; ++k)
    if (int rc = ensure_vec(&sys->vM[k], sys->m)) return rc;
  if (!sys->pg) TVR_CUDA(cudaMalloc(&sys->pg, sizeof(float2) * (sys->N > 0 ? sys->N : 1)));
  for (auto &w : sys->wplanes)
    if (!w) TVR_CUDA(cudaMalloc(&w, sizeof(float) * 4 * (sys->N > 0 ? sys->N : 1)));
  if (!sys->st) TVR_CUDA(cudaMalloc(&sys->st, sizeof(DevState)));
  if (!sys->pinned_flag) TVR_CUDA(cudaMallocHost(&sys->pinned_flag, 64));
  if (!sys->cap_stream) TVR_CUDA(cudaStreamCreateWithFlags(&sys->cap_stream, cudaStreamNonBlocking));
  if (hist_records > sys->hist_cap) {
    if (sys->hist_dev) cudaFree(sys->hist_dev);
    sys->hist_dev = nullptr;
    sys->hist_cap = 0;
    TVR_CUDA(cudaMalloc(&sys->hist_dev, sizeof(double) * TVR_HIST_FIELDS * hist_records));
    sys->hist_cap = (int)hist_records;
  }
  return TVR_OK;
}

// Kernel kinds a solver pass launches: back projection and the trial kernel
// (forward projection with the step and UPN's extrapolation fused).
bool pass_kind(int k, int solver) {
  (void)solver;
  return k == 0 || k == 1;
}

// A batch of passes captured once per (system, method, batch size) and
// replayed.  With kernel timing on, the graph also holds an event node pair
// around every kernel and gives each pass its slot for the "did work" flags.
// `solver` is the pass kind (a solver, or PASS_GPBB2).
int pass_graph(tvr_system *sys, int solver, int batch, bool timed, cudaGraphExec_t *out) {
  cudaGraphExec_t &cache = timed ? sys->pass_graph_prof[solver] : sys->pass_graph[solver];
  int &cache_batch = timed ? sys->pass_graph_prof_batch[solver] : sys->pass_graph_batch[solver];
  const int key = sys->profile | (sys->prof_stride << 8);
  if (cache && cache_batch == batch && (!timed || sys->pass_graph_prof_mask[solver] == key)) {
    *out = cache;
    return TVR_OK;
  }
  if (cache) {
    cudaGraphExecDestroy(cache);
    cache = nullptr;
  }
  if (timed && sys->gprof_batch < batch) {
    if (sys->gprof_ev) {
      for (int i = 0; i < sys->gprof_batch * TVR_PROF_KINDS * 2; ++i)
        cudaEventDestroy(sys->gprof_ev[i]);
      delete[] sys->gprof_ev;
      sys->gprof_ev = nullptr;
      sys->gprof_batch = 0;
      // graphs recorded with the old events are stale
      for (auto &g : sys->pass_graph_prof)
        if (g) {
          cudaGraphExecDestroy(g);
          g = nullptr;
        }
    }
    sys->gprof_ev = new cudaEvent_t[(size_t)batch * TVR_PROF_KINDS * 2]();
    for (int i = 0; i < batch * TVR_PROF_KINDS * 2; ++i)
      TVR_CUDA(cudaEventCreate(&sys->gprof_ev[i]));
    sys->gprof_batch = batch;
  }
  const MatDev A = sys->mat();
  TVR_CUDA(cudaStreamBeginCapture(sys->cap_stream, cudaStreamCaptureModeThreadLocal));
  for (int i = 0; i < batch; ++i) {
    if (timed) {
      PassTiming tm;
      tm.graph_nodes = true;
      for (int k = 0; k < TVR_PROF_KINDS; ++k) {
        tm.slot[k] = (pass_kind(k, solver) && ((sys->profile >> k) & 1) &&
                      i % sys->prof_stride == 0)
                         ? i
                         : -1;
        for (int w = 0; w < 2; ++w) tm.ev[k][w] = sys->gprof_ev[(i * TVR_PROF_KINDS + k) * 2 + w];
      }
      launch_solver_pass(A, sys->st, solver, sys->ws, sys->cap_stream, &tm);
    } else {
      launch_solver_pass(A, sys->st, solver, sys->ws, sys->cap_stream);
    }
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(sys->cap_stream, &g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture(pass batch)");
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate(pass batch)");
  cache = exec;
  cache_batch = batch;
  if (timed) sys->pass_graph_prof_mask[solver] = key;
  *out = exec;
  return TVR_OK;
}

// After a replay of a timed pass graph has completed: add the durations of
// the launches that did work, then clear their flags.
int graph_prof_harvest(tvr_system *sys, int batch) {
  const size_t bytes = sizeof(int) * TVR_PROF_KINDS * kProfPairs;
  TVR_CUDA(cudaMemcpy(sys->prof_flags_host, sys->prof_flags_dev, bytes, cudaMemcpyDeviceToHost));
  TVR_CUDA(cudaMemset(sys->prof_flags_dev, 0, bytes));
  for (int i = 0; i < batch; ++i)
    for (int k = 0; k < TVR_PROF_KINDS; ++k) {
      if (!sys->prof_flags_host[k * kProfPairs + i]) continue;
      float ms = 0.f;
      TVR_CUDA(cudaEventElapsedTime(&ms, sys->gprof_ev[(i * TVR_PROF_KINDS + k) * 2],
                                    sys->gprof_ev[(i * TVR_PROF_KINDS + k) * 2 + 1]));
      sys->prof_ms[k] += ms;
      sys->prof_cnt[k] += 1;
    }
  return TVR_OK;
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

// One solve, split into phases so that several solves can interleave on
// their own streams (tvr_solve_batch).
struct Job {
  tvr_system *sys = nullptr;
  int solver = 0;
  int pass = 0;  // solver, or PASS_GPBB2
  double alpha = 0, tau = 0, eps = 0;
  tvr_solve_opts o{};
  float *x = nullptr;
  bool xdev = false;
  const float *bd = nullptr;
  int64_t hist_n = 0;
  cudaStream_t s = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool timed_graph = false;
  int64_t passes = 0, max_passes = 0;
  bool done = false;
};

int check_opts(const tvr_solve_opts &o) {
  if (o.k_max < 1 || o.gpbb_K < 0 || o.gpbb_K > 8 || o.gpbb_max_trials < 0 || o.bt_max < 0 ||
      o.batch < 1 || o.batch > 1024 || !(o.rho_L > 1.0) || !std::isfinite(o.rho_L) ||
      !finite_pos(o.L_bar) || !(o.mu_bar >= 0.0) || !std::isfinite(o.mu_bar) ||
      !(o.gpbb_sigma > 0.0 && o.gpbb_sigma < 1.0) || !(o.gpbb_beta0 > 0.0 && o.gpbb_beta0 < 1.0) ||
      (o.stop_mode != TVR_STOP_REL && o.stop_mode != TVR_STOP_PER_N) || o.history_len < 0 ||
      (o.history_len > 0 && !o.history) || o.gpbb_points < 0 || o.gpbb_points > 2)
    return fail(TVR_ERR_ARG, "tvr_solve: invalid options");
  return TVR_OK;
}

// Validate, upload x0 and the state, launch the initial phi and gradient.
int job_begin(Job &j, tvr_system *sys, int solver, const float *b, double alpha, double tau,
              double eps, const tvr_solve_opts *uo, float *x, cudaStream_t s) {
  if (!sys || !b || !x) return fail(TVR_ERR_ARG, "tvr_solve: null argument");
  if (!(alpha >= 0.0) || !std::isfinite(alpha) || !finite_pos(tau) || !finite_pos(eps))
    return fail(TVR_ERR_ARG, "tvr_solve: need alpha >= 0, tau > 0, eps > 0 (finite)");
  j.sys = sys;
  j.solver = solver;
  j.alpha = alpha;
  j.tau = tau;
  j.eps = eps;
  j.s = s;
  j.x = x;
  tvr_solve_opts_default(&j.o);
  if (uo) j.o = *uo;
  if (int rc = check_opts(j.o)) return rc;
  const tvr_solve_opts &o = j.o;
  j.pass = solver == SOLVER_GPBB && o.gpbb_points != 1 ? PASS_GPBB2 : solver;
  j.hist_n = o.history ? (o.history_len < (1 << 30) ? o.history_len : (1 << 30)) : 0;
  if (int rc = ensure_solver(sys, j.hist_n)) return rc;
  if (int rc = stage_in(b, sys->m, &sys->stage_bM, s, &j.bd)) return rc;
  j.xdev = is_device_ptr(x);
  const cudaMemcpyKind kin = j.xdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  TVR_CUDA(cudaMemcpyAsync(sys->vN[0], x, sizeof(float) * sys->N, kin, s));
  if (solver == SOLVER_UPN) {
    TVR_CUDA(cudaMemcpyAsync(sys->vN[RN_Y], sys->vN[RN_X], sizeof(float) * sys->N,
                             cudaMemcpyDeviceToDevice, s));
    TVR_CUDA(cudaMemsetAsync(sys->vM[RM_U], 0, sizeof(float) * sys->m, s));
  }
  DevState h;
  std::memset(&h, 0, sizeof(h));
  h.alpha = alpha;
  h.tau = tau;
  h.eps = eps;
  h.rho = o.rho_L;
  h.sigma = o.gpbb_sigma;
  h.beta0 = o.gpbb_beta0;
  h.Lbar = o.L_bar;
  h.mubar = o.mu_bar;
  h.kmax = o.k_max;
  h.K = o.gpbb_K;
  h.max_trials = o.gpbb_max_trials;
  h.bt_max = o.bt_max;
  h.stop_mode = o.stop_mode;
  h.solver = solver;
  h.spec_upn = solver == SOLVER_UPN;
  h.N = sys->N;
  h.b = j.bd;
  for (int k = 0; k < RN_COUNT; ++k) h.vN[k] = sys->vN[k];
  for (int k = 0; k < RM_COUNT; ++k) h.vM[k] = sys->vM[k];
  h.pg = sys->pg;
  h.w = sys->wplanes[0];
  h.wt = sys->wplanes[1];
  h.wt2 = sys->wplanes[2];
  h.hist = j.hist_n > 0 ? sys->hist_dev : nullptr;
  h.prof_flags = sys->prof_flags_dev;
  h.hist_cap = (int)j.hist_n;
  TVR_CUDA(cudaMemcpyAsync(sys->st, &h, sizeof(h), cudaMemcpyHostToDevice, s));
  launch_solver_init(sys->mat(), sys->st, sys->ws, s);
  TVR_CUDA(cudaGetLastError());
  j.exec = nullptr;
  j.timed_graph = o.use_graph && sys->profile && o.batch <= kProfPairs;
  if (o.use_graph && (!sys->profile || j.timed_graph))
    if (int rc = pass_graph(sys, j.pass, o.batch, j.timed_graph, &j.exec)) return rc;
  const int64_t trials = (o.bt_max > o.gpbb_max_trials ? o.bt_max : o.gpbb_max_trials) + 2;
  j.max_passes = ((int64_t)o.k_max + 1) * trials + o.batch;
  j.passes = 0;
  j.done = false;
  return TVR_OK;
}

// One batch of passes and an asynchronous copy of the "done" word.
int job_launch(Job &j) {
  tvr_system *sys = j.sys;
  const MatDev A = sys->mat();
  if (j.exec) {
    TVR_CUDA(cudaGraphLaunch(j.exec, j.s));
  } else {
    for (int i = 0; i < j.o.batch; ++i) {
      PassTiming tm;
      const PassTiming *tp = nullptr;
      if (sys->profile) {
        bool full = false;
        for (int k = 0; k < TVR_PROF_KINDS; ++k) full = full || sys->prof_n[k] >= kProfPairs;
        if (full)
          if (int rc = prof_harvest(sys)) return rc;
        for (int k = 0; k < TVR_PROF_KINDS; ++k) {
          const bool used = pass_kind(k, j.solver) && ((sys->profile >> k) & 1);
          const int sl = used ? prof_take(sys, k, true) : -1;
          tm.slot[k] = sl;
          if (sl >= 0)
            for (int w = 0; w < 2; ++w) tm.ev[k][w] = sys->prof_ev[k][sl][w];
        }
        tp = &tm;
      }
      launch_solver_pass(A, sys->st, j.pass, sys->ws, j.s, tp);
    }
    TVR_CUDA(cudaGetLastError());
  }
  j.passes += j.o.batch;
  TVR_CUDA(cudaMemcpyAsync(sys->pinned_flag, &sys->st->done, sizeof(int), cudaMemcpyDeviceToHost,
                           j.s));
  return TVR_OK;
}

// After the job's stream has drained: read the flag (and the kernel timings).
int job_poll(Job &j) {
  j.done = *j.sys->pinned_flag != 0 || j.passes >= j.max_passes;
  if (j.timed_graph)
    if (int rc = graph_prof_harvest(j.sys, j.o.batch)) return rc;
  return TVR_OK;
}

// Copy x*, evaluate phi(x*), copy the history, fill info.  Synchronises.
int job_end(Job &j, tvr_solve_info *info) {
  tvr_system *sys = j.sys;
  cudaStream_t s = j.s;
  DevState f;
  TVR_CUDA(cudaMemcpyAsync(&f, sys->st, sizeof(f), cudaMemcpyDeviceToHost, s));
  TVR_CUDA(cudaStreamSynchronize(s));
  const MatDev A = sys->mat();
  const cudaMemcpyKind kout = j.xdev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  TVR_CUDA(cudaMemcpyAsync(j.x, f.vN[RN_X], sizeof(float) * sys->N, kout, s));
  launch_forward(A, f.vN[RN_X], j.bd, f.vM[RM_RT], sys->ws, s);
  launch_tv_value(A, f.vN[RN_X], (float)j.alpha, (float)j.tau, sys->ws, sys->phi_ws, s);
  TVR_CUDA(cudaGetLastError());
  double phi[3] = {0, 0, 0};
  TVR_CUDA(cudaMemcpyAsync(phi, sys->phi_ws, sizeof(phi), cudaMemcpyDeviceToHost, s));
  int hist_used = 0;
  if (j.hist_n > 0 && f.hist_used > 0) {
    hist_used = f.hist_used;
    TVR_CUDA(cudaMemcpyAsync(j.o.history, sys->hist_dev,
                             sizeof(double) * TVR_HIST_FIELDS * hist_used, cudaMemcpyDeviceToHost, s));
  }
  TVR_CUDA(cudaStreamSynchronize(s));
  const int status = f.done ? f.status : TVR_NOT_CONVERGED;
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->status = status;
    info->iters = f.k;
    info->f_evals = f.f_evals;
    info->g_evals = f.g_evals;
    info->trials = f.total_trials;
    info->passes = (int32_t)j.passes;
    info->history_used = hist_used;
    info->phi = phi[0];
    info->gnorm = f.gnorm;
    info->gnorm0 = f.gnorm0;
    info->stop_value = f.stopval;
    info->L = j.solver == SOLVER_GPBB ? 1.0 / f.theta : f.L;
    info->theta = f.theta;
    info->mu = f.mu;
  }
  if (status < 0) {
    const char *what = status == TVR_ERR_LINESEARCH ? "line search hit its trial cap"
                                                    : "non-finite control value";
    fail(status, std::string("tvr_solve: ") + what);
  }
  return status;
}

int solve(const tvr_system *csys, int solver, const float *b, double alpha, double tau, double eps,
          const tvr_solve_opts *uo, float *x, tvr_solve_info *info, void *stream) {
  Job j;
  if (int rc = job_begin(j, const_cast<tvr_system *>(csys), solver, b, alpha, tau, eps, uo, x,
                         (cudaStream_t)stream))
    return rc;
  while (!j.done) {
    if (int rc = job_launch(j)) return rc;
    TVR_CUDA(cudaStreamSynchronize(j.s));
    if (int rc = job_poll(j)) return rc;
  }
  return job_end(j, info);
}

}  // namespace

extern "C" {

int tvr_solve_gp(const tvr_system *sys, const float *b, double alpha, double tau, double eps,
                 const tvr_solve_opts *opts, float *x, tvr_solve_info *info, void *stream) {
  return solve(sys, SOLVER_GP, b, alpha, tau, eps, opts, x, info, stream);
}

int tvr_solve_gpbb(const tvr_system *sys, const float *b, double alpha, double tau, double eps,
                   const tvr_solve_opts *opts, float *x, tvr_solve_info *info, void *stream) {
  return solve(sys, SOLVER_GPBB, b, alpha, tau, eps, opts, x, info, stream);
}

int tvr_solve_upn(const tvr_system *sys, const float *b, double alpha, double tau, double eps,
                  const tvr_solve_opts *opts, float *x, tvr_solve_info *info, void *stream) {
  return solve(sys, SOLVER_UPN, b, alpha, tau, eps, opts, x, info, stream);
}

int tvr_solve_batch(tvr_system *const *systems, int32_t count, int32_t method,
                    const float *const *bs, const double *alphas, double tau, double eps,
                    const tvr_solve_opts *opts, float *const *xs, tvr_solve_info *infos,
                    void *stream) {
  if (!systems || !bs || !alphas || !xs || count < 1)
    return fail(TVR_ERR_ARG, "tvr_solve_batch: null argument or count < 1");
  if (method != SOLVER_GP && method != SOLVER_GPBB && method != SOLVER_UPN)
    return fail(TVR_ERR_ARG, "tvr_solve_batch: method must be 1 (GP), 2 (GPBB) or 3 (UPN)");
  for (int i = 0; i < count; ++i) {
    if (!systems[i]) return fail(TVR_ERR_ARG, "tvr_solve_batch: null system");
    for (int k = 0; k < i; ++k)
      if (systems[k] == systems[i])
        return fail(TVR_ERR_ARG, "tvr_solve_batch: a system appears twice (they share workspace)");
  }
  TVR_CUDA(cudaStreamSynchronize((cudaStream_t)stream));  // inputs written on the caller's stream
  std::vector<Job> jobs(count);
  for (int i = 0; i < count; ++i) {
    tvr_system *sys = systems[i];
    if (!sys->run_stream) TVR_CUDA(cudaStreamCreateWithFlags(&sys->run_stream, cudaStreamNonBlocking));
    if (int rc = job_begin(jobs[i], sys, method, bs[i], alphas[i], tau, eps, opts, xs[i],
                           sys->run_stream))
      return rc;
  }
  // Every problem runs batches of passes on its own stream; the host relaunches
  // each one as soon as its previous batch has drained, so small problems do
  // not wait for the large ones.
  for (auto &j : jobs)
    if (int rc = job_launch(j)) return rc;
  for (int running = count; running > 0;) {
    bool progressed = false;
    for (auto &j : jobs) {
      if (j.done) continue;
      const cudaError_t q = cudaStreamQuery(j.s);
      if (q == cudaErrorNotReady) {
        // not an error: keep it out of the error checks that follow launches
        if (cudaPeekAtLastError() == cudaErrorNotReady) (void)cudaGetLastError();
        continue;
      }
      if (q != cudaSuccess) return cuda_fail(q, "cudaStreamQuery(solve batch)");
      progressed = true;
      if (int rc = job_poll(j)) return rc;
      if (j.done)
        --running;
      else if (int rc = job_launch(j))
        return rc;
    }
    if (!progressed) std::this_thread::yield();
  }
  int worst = TVR_OK;
  for (int i = 0; i < count; ++i) {
    const int st = job_end(jobs[i], infos ? &infos[i] : nullptr);
    if (st < 0 && worst >= 0) worst = st;
    if (st == TVR_NOT_CONVERGED && worst == TVR_OK) worst = st;
  }
  return worst;
}

int tvr_trial_sums(const tvr_system *csys, const float *p, const float *g, const float *b, double s,
                   double tau, double sums[6], float *xbar, float *resid, void *stream) {
  tvr_system *sys = const_cast<tvr_system *>(csys);
  if (!sys || !p || !g || !b || !sums) return fail(TVR_ERR_ARG, "tvr_trial_sums: null argument");
  if (!finite_pos(s) || !finite_pos(tau))
    return fail(TVR_ERR_ARG, "tvr_trial_sums: need s > 0 and tau > 0 (finite)");
  if (!is_device_ptr(p) || !is_device_ptr(g) || !is_device_ptr(b) ||
      (xbar && !is_device_ptr(xbar)) || (resid && !is_device_ptr(resid)))
    return fail(TVR_ERR_ARG, "tvr_trial_sums: vectors must be device memory");
  cudaStream_t st = (cudaStream_t)stream;
  if (int rc = ensure_solver(sys, 0)) return rc;
  // the (p_j, g_j) pairs the trial gathers, interleaved by two strided copies
  TVR_CUDA(cudaMemcpy2DAsync(sys->pg, sizeof(float2), p, sizeof(float), sizeof(float), sys->N,
                             cudaMemcpyDeviceToDevice, st));
  TVR_CUDA(cudaMemcpy2DAsync(reinterpret_cast<float *>(sys->pg) + 1, sizeof(float2), g,
                             sizeof(float), sizeof(float), sys->N, cudaMemcpyDeviceToDevice, st));
  // a GP trial at step s (BT's L = 1/s); its control step then accepts or
  // rejects it in this scratch state, which only moves the roles around
  DevState h;
  std::memset(&h, 0, sizeof(h));
  h.alpha = 0.0;
  h.tau = tau;
  h.eps = 0.0;
  h.rho = 2.0;
  h.Lbar = 1.0 / s;
  h.Lt = 1.0 / s;
  h.L = 1.0 / s;
  h.step = s;
  h.kmax = 1 << 30;
  h.bt_max = 0;
  h.solver = SOLVER_GP;
  h.N = sys->N;
  h.b = b;
  for (int k = 0; k < RN_COUNT; ++k) h.vN[k] = sys->vN[k];
  for (int k = 0; k < RM_COUNT; ++k) h.vM[k] = sys->vM[k];
  h.pg = sys->pg;
  h.w = sys->wplanes[0];
  h.wt = sys->wplanes[1];
  h.wt2 = sys->wplanes[2];
  TVR_CUDA(cudaMemcpyAsync(sys->st, &h, sizeof(h), cudaMemcpyHostToDevice, st));
  launch_trial(sys->mat(), sys->st, sys->ws, st);
  TVR_CUDA(cudaGetLastError());
  DevState f;
  TVR_CUDA(cudaMemcpyAsync(&f, sys->st, sizeof(f), cudaMemcpyDeviceToHost, st));
  TVR_CUDA(cudaStreamSynchronize(st));
  sums[0] = f.r_fwd[0];
  sums[1] = f.r_fwd[1];
  for (int k = 0; k < 3; ++k) sums[2 + k] = f.r_step[k];
  sums[5] = f.r_step[4];
  // the trial's outputs are where the roles point after its control step
  // (an accepted trial swaps x with xbar and r with A xbar - b)
  const bool accepted = f.k == 1;
  const float *xb = accepted ? f.vN[RN_X] : f.vN[RN_T];
  const float *rt = accepted ? f.vM[RM_R] : f.vM[RM_RT];
  if (xbar)
    TVR_CUDA(cudaMemcpyAsync(xbar, xb, sizeof(float) * sys->N, cudaMemcpyDeviceToDevice, st));
  if (resid)
    TVR_CUDA(cudaMemcpyAsync(resid, rt, sizeof(float) * sys->m, cudaMemcpyDeviceToDevice, st));
  TVR_CUDA(cudaStreamSynchronize(st));
  return TVR_OK;
}

}  // extern "C"

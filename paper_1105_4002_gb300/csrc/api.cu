// C ABI of libtvr (declared in include/tvr.h): system ownership, argument
// checks, host/device staging, and the solver pass loop.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "tvr_internal.cuh"

#include "system.cuh"

thread_local std::string g_last_error = "no error";

int tvr_fail(int status, const std::string &msg) {
  g_last_error = msg;
  return status;
}

int tvr_cuda_fail(cudaError_t e, const char *what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? TVR_ERR_OOM : TVR_ERR_CUDA;
}

// Copy a padded compressed layout to host, undo the lane-interleaved stored
// order (lane_stored) and drop the padding entries.
static int export_compact(const int64_t *ptr_d, const int32_t *len_d, const int32_t *idx_d,
                          const float *val_d, int64_t rows, int64_t stored, int64_t *ptr_out,
                          int32_t *idx_out, float *val_out) {
  std::vector<int64_t> ptr(rows + 1);
  std::vector<int32_t> len(rows > 0 ? rows : 1);
  TVR_CUDA(cudaMemcpy(ptr.data(), ptr_d, sizeof(int64_t) * (rows + 1), cudaMemcpyDeviceToHost));
  if (rows > 0)
    TVR_CUDA(cudaMemcpy(len.data(), len_d, sizeof(int32_t) * rows, cudaMemcpyDeviceToHost));
  std::vector<int32_t> idx(idx_out && stored ? stored : 0);
  std::vector<float> val(val_out && stored ? stored : 0);
  if (!idx.empty())
    TVR_CUDA(cudaMemcpy(idx.data(), idx_d, sizeof(int32_t) * stored, cudaMemcpyDeviceToHost));
  if (!val.empty())
    TVR_CUDA(cudaMemcpy(val.data(), val_d, sizeof(float) * stored, cudaMemcpyDeviceToHost));
  int64_t o = 0;
  if (ptr_out) ptr_out[0] = 0;
  for (int64_t i = 0; i < rows; ++i) {
    const int64_t L = ptr[i + 1] - ptr[i];
    for (int32_t k = 0; k < len[i]; ++k) {
      const int64_t e = ptr[i] + lane_stored(k, L);
      if (idx_out) idx_out[o + k] = idx[e];
      if (val_out) val_out[o + k] = val[e];
    }
    o += len[i];
    if (ptr_out) ptr_out[i + 1] = o;
  }
  return TVR_OK;
}

extern "C" {

const char *tvr_status_str(int status) {
  switch (status) {
    case TVR_OK: return "TVR_OK";
    case TVR_NOT_CONVERGED: return "TVR_NOT_CONVERGED";
    case TVR_ERR_ARG: return "TVR_ERR_ARG";
    case TVR_ERR_OOM: return "TVR_ERR_OOM";
    case TVR_ERR_CUDA: return "TVR_ERR_CUDA";
    case TVR_ERR_LINESEARCH: return "TVR_ERR_LINESEARCH";
    case TVR_ERR_NONFINITE: return "TVR_ERR_NONFINITE";
    default: return "TVR_UNKNOWN_STATUS";
  }
}

const char *tvr_last_error(void) { return g_last_error.c_str(); }

int tvr_system_free(tvr_system *sys) {
  if (!sys) return TVR_OK;
  cudaSetDevice(sys->device);
  cudaDeviceSynchronize();
  for (auto &g : sys->pass_graph)
    if (g) cudaGraphExecDestroy(g);
  for (auto &g : sys->pass_graph_prof)
    if (g) cudaGraphExecDestroy(g);
  if (sys->gprof_ev) {
    for (int i = 0; i < sys->gprof_batch * TVR_PROF_KINDS * 2; ++i) cudaEventDestroy(sys->gprof_ev[i]);
    delete[] sys->gprof_ev;
  }
  if (sys->cap_stream) cudaStreamDestroy(sys->cap_stream);
  if (sys->run_stream) cudaStreamDestroy(sys->run_stream);
  for (int k = 0; k < TVR_PROF_KINDS; ++k)
    for (int i = 0; i < kProfPairs; ++i)
      for (int w = 0; w < 2; ++w)
        if (sys->prof_ev[k][i][w]) cudaEventDestroy(sys->prof_ev[k][i][w]);
  free_matrix(sys->A);
  sweep_free(sys->sweep);
  if (sys->stage_sweepX) cudaFree(sys->stage_sweepX);
  void *ptrs[] = {sys->ws_mem, sys->stage_xN, sys->stage_gN, sys->stage_bM, sys->stage_rM,
                  sys->phi_ws, sys->st, sys->hist_dev, sys->prof_flags_dev, sys->pg,
                  sys->wplanes[0], sys->wplanes[1], sys->wplanes[2]};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  for (float *p : sys->vN)
    if (p) cudaFree(p);
  for (float *p : sys->vM)
    if (p) cudaFree(p);
  if (sys->pinned_flag) cudaFreeHost(sys->pinned_flag);
  if (sys->prof_flags_host) cudaFreeHost(sys->prof_flags_host);
  delete sys;
  return TVR_OK;
}

int tvr_build_system(const tvr_geometry *g, int32_t storage, void *stream, tvr_system **out) {
  if (!g || !out) return fail(TVR_ERR_ARG, "tvr_build_system: null argument");
  *out = nullptr;
  if (storage != TVR_STORAGE_FP32 && storage != TVR_STORAGE_BF16_ROWSCALE &&
      storage != TVR_STORAGE_U16_ROWSCALE && storage != TVR_STORAGE_MATRIX_FREE)
    return fail(TVR_ERR_ARG, "tvr_build_system: unknown storage");
  if (g->n < 1 || g->n_views < 1 || g->det_cols < 1 || g->det_rows < 1 || !g->views ||
      (g->kind != TVR_CONE && g->kind != TVR_PARALLEL) || g->reserved != 0)
    return fail(TVR_ERR_ARG, "tvr_build_system: invalid geometry");
  const int64_t N = (int64_t)g->n * g->n * g->n;
  if (N >= (int64_t)1 << 31 || g->n > 1 << 20)
    return fail(TVR_ERR_ARG, "tvr_build_system: n^3 must be < 2^31");
  for (int64_t i = 0; i < (int64_t)g->n_views * TVR_VIEW_FIELDS; ++i)
    if (!std::isfinite(g->views[i])) return fail(TVR_ERR_ARG, "tvr_build_system: non-finite view");
  cudaStream_t s = (cudaStream_t)stream;
  tvr_system *sys = new tvr_system();
  int rc = TVR_OK;
  double *views_dev = nullptr;
  auto cleanup = [&]() {
    if (views_dev) cudaFree(views_dev);
  };
#define BUILD_CUDA(call)                          \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) {                      \
      rc = cuda_fail(e_, #call);                  \
      cleanup();                                  \
      tvr_system_free(sys);                       \
      return rc;                                  \
    }                                             \
  } while (0)
  BUILD_CUDA(cudaGetDevice(&sys->device));
  sys->n = g->n;
  sys->V = g->n_views;
  sys->Pu = g->det_cols;
  sys->Pv = g->det_rows;
  sys->kind = g->kind;
  sys->m = (int64_t)g->n_views * g->det_cols * g->det_rows;
  sys->N = N;
  const int64_t m = sys->m;
  const size_t vbytes = sizeof(double) * TVR_VIEW_FIELDS * g->n_views;
  BUILD_CUDA(cudaMalloc(&views_dev, vbytes));
  BUILD_CUDA(cudaMemcpyAsync(views_dev, g->views, vbytes, cudaMemcpyHostToDevice, s));
  if (storage == TVR_STORAGE_MATRIX_FREE) {
    BUILD_CUDA(build_matrix_free(views_dev, g->n, g->n_views, g->det_cols, g->det_rows, g->kind,
                                 m, N, sys->A, s));
  } else {
    BUILD_CUDA(build_matrix(views_dev, g->n, g->det_cols, g->det_rows, g->kind, m, N, sys->A, s));
    if (storage == TVR_STORAGE_BF16_ROWSCALE) BUILD_CUDA(quantize_bf16(sys->A, s));
    if (storage == TVR_STORAGE_U16_ROWSCALE) BUILD_CUDA(quantize_u16(sys->A, s));
    BUILD_CUDA(interleave_lanes(sys->A, s));
  }
  sys->nnz = sys->A.nnz;
  // reduction workspace: per slot partials + counter + outputs
  const size_t part = sizeof(FF) * TVR_MAX_GRID * TVR_RMAX;
  const size_t slot_bytes = part + 256 + 256;
  BUILD_CUDA(cudaMalloc(&sys->ws_mem, slot_bytes * kSlots));
  BUILD_CUDA(cudaMemsetAsync(sys->ws_mem, 0, slot_bytes * kSlots, s));
  RedSlot *slots[kSlots] = {&sys->ws.fwd, &sys->ws.bwd, &sys->ws.step,
                            &sys->ws.yf,  &sys->ws.tv,  &sys->ws.gmap};
  for (int k = 0; k < kSlots; ++k) {
    char *b = (char *)sys->ws_mem + slot_bytes * k;
    slots[k]->partials = (FF *)b;
    slots[k]->counter = (unsigned *)(b + part);
    slots[k]->out = (double *)(b + part + 256);
  }
  kernel_grids(sys->ws, sys->mat(), sys->device);
  BUILD_CUDA(cudaMalloc(&sys->phi_ws, sizeof(double) * 4));
  BUILD_CUDA(cudaStreamSynchronize(s));
  BUILD_CUDA(cudaGetLastError());
#undef BUILD_CUDA
  cleanup();
  *out = sys;
  return TVR_OK;
}

int tvr_system_shape(const tvr_system *sys, int64_t *m, int64_t *N, int64_t *nnz) {
  if (!sys) return fail(TVR_ERR_ARG, "tvr_system_shape: null system");
  if (m) *m = sys->m;
  if (N) *N = sys->N;
  if (nnz) *nnz = sys->nnz;
  return TVR_OK;
}

int tvr_system_export_csr(const tvr_system *sys, int64_t *row_ptr, int32_t *col, float *val) {
  if (!sys) return fail(TVR_ERR_ARG, "export: null system");
  if (sys->A.storage == TVR_STORAGE_MATRIX_FREE)
    return fail(TVR_ERR_ARG, "export: a matrix-free system stores no matrix");
  TVR_CUDA(cudaSetDevice(sys->device));
  TVR_CUDA(cudaDeviceSynchronize());
  const float *vd = sys->A.val;
  float *tmp = nullptr;
  if (val && coded16(sys->A.storage)) {
    TVR_CUDA(cudaMalloc(&tmp, sizeof(float) * (sys->A.nnz_pad > 0 ? sys->A.nnz_pad : 1)));
    cudaError_t e = effective_values(sys->A, false, tmp, 0);
    if (e != cudaSuccess) {
      cudaFree(tmp);
      return cuda_fail(e, "effective_values");
    }
    vd = tmp;
  }
  int rc = export_compact(sys->A.row_ptr, sys->A.row_len, sys->A.col, vd, sys->m, sys->A.nnz_pad,
                          row_ptr, col, val);
  if (tmp) cudaFree(tmp);
  return rc;
}

int tvr_system_export_csc(const tvr_system *sys, int64_t *col_ptr, int32_t *row, float *val) {
  if (!sys) return fail(TVR_ERR_ARG, "export: null system");
  if (sys->A.storage == TVR_STORAGE_MATRIX_FREE)
    return fail(TVR_ERR_ARG, "export: a matrix-free system stores no matrix");
  TVR_CUDA(cudaSetDevice(sys->device));
  TVR_CUDA(cudaDeviceSynchronize());
  const float *vd = sys->A.cval;
  float *tmp = nullptr;
  if (val && coded16(sys->A.storage)) {
    TVR_CUDA(cudaMalloc(&tmp, sizeof(float) * (sys->A.nnz_cpad > 0 ? sys->A.nnz_cpad : 1)));
    cudaError_t e = effective_values(sys->A, true, tmp, 0);
    if (e != cudaSuccess) {
      cudaFree(tmp);
      return cuda_fail(e, "effective_values");
    }
    vd = tmp;
  }
  int rc = export_compact(sys->A.col_ptr, sys->A.col_len, sys->A.row, vd, sys->N, sys->A.nnz_cpad,
                          col_ptr, row, val);
  if (tmp) cudaFree(tmp);
  return rc;
}

int tvr_forward(const tvr_system *csys, const float *x, float *y, void *stream) {
  tvr_system *sys = const_cast<tvr_system *>(csys);
  if (!sys || !x || !y) return fail(TVR_ERR_ARG, "tvr_forward: null argument");
  cudaStream_t s = (cudaStream_t)stream;
  const float *xd;
  int rc = stage_in(x, sys->N, &sys->stage_xN, s, &xd);
  if (rc) return rc;
  const bool yh = !is_device_ptr(y);
  float *yd = y;
  if (yh) {
    if ((rc = ensure_vec(&sys->stage_rM, sys->m))) return rc;
    yd = sys->stage_rM;
  }
  prof_mark(sys, 0, 0, s);
  launch_forward_plain(sys->mat(), xd, yd, sys->ws, s);
  prof_mark(sys, 0, 1, s);
  TVR_CUDA(cudaGetLastError());
  if (yh) {
    TVR_CUDA(cudaMemcpyAsync(y, yd, sizeof(float) * sys->m, cudaMemcpyDeviceToHost, s));
    TVR_CUDA(cudaStreamSynchronize(s));
  }
  return TVR_OK;
}

int tvr_adjoint(const tvr_system *csys, const float *r, float *z, void *stream) {
  tvr_system *sys = const_cast<tvr_system *>(csys);
  if (!sys || !r || !z) return fail(TVR_ERR_ARG, "tvr_adjoint: null argument");
  cudaStream_t s = (cudaStream_t)stream;
  const float *rd;
  int rc = stage_in(r, sys->m, &sys->stage_bM, s, &rd);
  if (rc) return rc;
  const bool zh = !is_device_ptr(z);
  float *zd = z;
  if (zh) {
    if ((rc = ensure_vec(&sys->stage_gN, sys->N))) return rc;
    zd = sys->stage_gN;
  }
  prof_mark(sys, 1, 0, s);
  launch_adjoint_plain(sys->mat(), rd, zd, sys->ws, s);
  prof_mark(sys, 1, 1, s);
  TVR_CUDA(cudaGetLastError());
  if (zh) {
    TVR_CUDA(cudaMemcpyAsync(z, zd, sizeof(float) * sys->N, cudaMemcpyDeviceToHost, s));
    TVR_CUDA(cudaStreamSynchronize(s));
  }
  return TVR_OK;
}

int tvr_phi_and_grad(const tvr_system *csys, const float *x, const float *b, double alpha, double tau,
                     double *phi_dev, double *phi_host, float *grad, float *resid, void *stream) {
  tvr_system *sys = const_cast<tvr_system *>(csys);
  if (!sys || !x || !b) return fail(TVR_ERR_ARG, "tvr_phi_and_grad: null argument");
  if (!(alpha >= 0.0) || !(tau > 0.0) || !std::isfinite(alpha) || !std::isfinite(tau))
    return fail(TVR_ERR_ARG, "tvr_phi_and_grad: need alpha >= 0 and tau > 0");
  cudaStream_t s = (cudaStream_t)stream;
  int rc;
  const float *xd, *bd;
  if ((rc = stage_in(x, sys->N, &sys->stage_xN, s, &xd))) return rc;
  if ((rc = stage_in(b, sys->m, &sys->stage_bM, s, &bd))) return rc;
  bool sync = phi_host != nullptr;
  float *rd = resid;
  const bool rh = resid && !is_device_ptr(resid);
  if (!resid || rh) {
    if ((rc = ensure_vec(&sys->stage_rM, sys->m))) return rc;
    rd = sys->stage_rM;
  }
  double *pd = phi_dev ? phi_dev : sys->phi_ws;
  const MatDev A = sys->mat();
  float *rsd = nullptr;  // BF16 storage: the back projection gathers s_i r_i
  if (A.bf16 && grad) {
    if ((rc = ensure_vec(&sys->stage_rsM, sys->m))) return rc;
    rsd = sys->stage_rsM;
  }
  prof_mark(sys, 0, 0, s);
  launch_forward(A, xd, bd, rd, sys->ws, s, rsd);
  prof_mark(sys, 0, 1, s);
  if (grad) {
    const bool gh = !is_device_ptr(grad);
    float *gd = grad;
    if (gh) {
      if ((rc = ensure_vec(&sys->stage_gN, sys->N))) return rc;
      gd = sys->stage_gN;
    }
    prof_mark(sys, 1, 0, s);
    launch_backward(A, rsd ? rsd : rd, xd, (float)alpha, (float)tau, gd, sys->ws, pd, s);
    prof_mark(sys, 1, 1, s);
    if (gh) {
      TVR_CUDA(cudaMemcpyAsync(grad, gd, sizeof(float) * sys->N, cudaMemcpyDeviceToHost, s));
      sync = true;
    }
  } else {
    launch_tv_value(A, xd, (float)alpha, (float)tau, sys->ws, pd, s);
  }
  TVR_CUDA(cudaGetLastError());
  if (rh) {
    TVR_CUDA(cudaMemcpyAsync(resid, rd, sizeof(float) * sys->m, cudaMemcpyDeviceToHost, s));
    sync = true;
  }
  if (phi_host) TVR_CUDA(cudaMemcpyAsync(phi_host, pd, sizeof(double) * 3, cudaMemcpyDeviceToHost, s));
  if (sync) TVR_CUDA(cudaStreamSynchronize(s));
  return TVR_OK;
}

int tvr_phi_and_grad_f64(const tvr_system *csys, const double *x, const double *b, double alpha,
                         double tau, double *phi_dev, double *phi_host, double *grad,
                         double *resid, void *stream) {
  tvr_system *sys = const_cast<tvr_system *>(csys);
  if (!sys || !x || !b || !resid) return fail(TVR_ERR_ARG, "tvr_phi_and_grad_f64: null argument");
  if (!(alpha >= 0.0) || !(tau > 0.0) || !std::isfinite(alpha) || !std::isfinite(tau))
    return fail(TVR_ERR_ARG, "tvr_phi_and_grad_f64: need alpha >= 0 and tau > 0");
  if (!is_device_ptr(x) || !is_device_ptr(b) || !is_device_ptr(resid) ||
      (grad && !is_device_ptr(grad)) || (phi_dev && !is_device_ptr(phi_dev)))
    return fail(TVR_ERR_ARG, "tvr_phi_and_grad_f64: vectors must be device memory");
  if (!grad) return fail(TVR_ERR_ARG, "tvr_phi_and_grad_f64: grad is required");
  if (sys->A.storage != TVR_STORAGE_FP32)
    return fail(TVR_ERR_ARG, "tvr_phi_and_grad_f64: needs a system with FP32 storage");
  cudaStream_t s = (cudaStream_t)stream;
  double *pd = phi_dev ? phi_dev : sys->phi_ws;
  const MatDev A = sys->mat();
  launch_forward_f64(A, x, b, resid, sys->ws, s);
  launch_backward_f64(A, resid, x, alpha, tau, grad, sys->ws, pd, s);
  TVR_CUDA(cudaGetLastError());
  if (phi_host) {
    TVR_CUDA(cudaMemcpyAsync(phi_host, pd, sizeof(double) * 3, cudaMemcpyDeviceToHost, s));
    TVR_CUDA(cudaStreamSynchronize(s));
  }
  return TVR_OK;
}

int tvr_phi_vjp(const tvr_system *csys, const float *x, const float *resid, double alpha,
                double tau, const double *scale_dev, float *grad_x, float *grad_b, void *stream) {
  tvr_system *sys = const_cast<tvr_system *>(csys);
  if (!sys || !x || !resid || !scale_dev || !grad_x)
    return fail(TVR_ERR_ARG, "tvr_phi_vjp: null argument");
  if (!(alpha >= 0.0) || !(tau > 0.0) || !std::isfinite(alpha) || !std::isfinite(tau))
    return fail(TVR_ERR_ARG, "tvr_phi_vjp: need alpha >= 0 and tau > 0");
  if (!is_device_ptr(x) || !is_device_ptr(resid) || !is_device_ptr(scale_dev) ||
      !is_device_ptr(grad_x) || (grad_b && !is_device_ptr(grad_b)))
    return fail(TVR_ERR_ARG, "tvr_phi_vjp: vectors must be device memory");
  prof_mark(sys, 1, 0, (cudaStream_t)stream);
  launch_vjp(sys->mat(), resid, x, (float)alpha, (float)tau, scale_dev, grad_x, grad_b, sys->ws,
             (cudaStream_t)stream);
  prof_mark(sys, 1, 1, (cudaStream_t)stream);
  TVR_CUDA(cudaGetLastError());
  return TVR_OK;
}

int tvr_phi_vjp_f64(const tvr_system *csys, const double *x, const double *resid, double alpha,
                    double tau, const double *scale_dev, double *grad_x, double *grad_b,
                    void *stream) {
  tvr_system *sys = const_cast<tvr_system *>(csys);
  if (!sys || !x || !resid || !scale_dev || !grad_x)
    return fail(TVR_ERR_ARG, "tvr_phi_vjp_f64: null argument");
  if (!(alpha >= 0.0) || !(tau > 0.0) || !std::isfinite(alpha) || !std::isfinite(tau))
    return fail(TVR_ERR_ARG, "tvr_phi_vjp_f64: need alpha >= 0 and tau > 0");
  if (!is_device_ptr(x) || !is_device_ptr(resid) || !is_device_ptr(scale_dev) ||
      !is_device_ptr(grad_x) || (grad_b && !is_device_ptr(grad_b)))
    return fail(TVR_ERR_ARG, "tvr_phi_vjp_f64: vectors must be device memory");
  if (sys->A.storage != TVR_STORAGE_FP32)
    return fail(TVR_ERR_ARG, "tvr_phi_vjp_f64: needs a system with FP32 storage");
  launch_vjp_f64(sys->mat(), resid, x, alpha, tau, scale_dev, grad_x, grad_b, sys->ws,
                 (cudaStream_t)stream);
  TVR_CUDA(cudaGetLastError());
  return TVR_OK;
}

int tvr_project_Q(float *x, int64_t n, void *stream) {
  if (n < 0 || (!x && n > 0)) return fail(TVR_ERR_ARG, "tvr_project_Q: bad arguments");
  if (n == 0) return TVR_OK;
  if (!is_device_ptr(x)) return fail(TVR_ERR_ARG, "tvr_project_Q: x must be device memory");
  launch_project(x, n, (cudaStream_t)stream);
  TVR_CUDA(cudaGetLastError());
  return TVR_OK;
}

void tvr_solve_opts_default(tvr_solve_opts *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->k_max = 20000;
  o->stop_mode = TVR_STOP_REL;
  o->gpbb_K = 2;
  o->gpbb_max_trials = 12;
  o->bt_max = 60;
  o->use_graph = 1;
  o->batch = 32;
  o->gpbb_points = 2;
  o->gpbb_sigma = 0.1;
  o->gpbb_beta0 = 0.95;
  o->rho_L = 2.0;
  o->L_bar = 1.0;
  o->mu_bar = 0.1;
}

int tvr_profile_enable(tvr_system *sys, int32_t enable) {
  if (!sys) return fail(TVR_ERR_ARG, "tvr_profile_enable: null system");
  if (enable && !sys->prof_ev[0][0][0]) {
    for (int k = 0; k < TVR_PROF_KINDS; ++k)
      for (int i = 0; i < kProfPairs; ++i)
        for (int w = 0; w < 2; ++w) TVR_CUDA(cudaEventCreate(&sys->prof_ev[k][i][w]));
    TVR_CUDA(cudaMalloc(&sys->prof_flags_dev, sizeof(int) * TVR_PROF_KINDS * kProfPairs));
    TVR_CUDA(cudaMemset(sys->prof_flags_dev, 0, sizeof(int) * TVR_PROF_KINDS * kProfPairs));
    TVR_CUDA(cudaMallocHost(&sys->prof_flags_host, sizeof(int) * TVR_PROF_KINDS * kProfPairs));
  }
  if (sys->profile)
    if (int rc = prof_harvest(sys)) return rc;
  sys->profile = enable & ((1 << TVR_PROF_KINDS) - 1);
  const int stride = (enable >> 8) & 0xff;
  sys->prof_stride = stride > 0 ? stride : 1;
  return TVR_OK;
}

int tvr_profile_read(tvr_system *sys, int64_t counts[4], double total_ms[4]) {
  if (!sys || !counts || !total_ms) return fail(TVR_ERR_ARG, "tvr_profile_read: null argument");
  if (int rc = prof_harvest(sys)) return rc;
  for (int k = 0; k < TVR_PROF_KINDS; ++k) {
    counts[k] = sys->prof_cnt[k];
    total_ms[k] = sys->prof_ms[k];
    sys->prof_cnt[k] = 0;
    sys->prof_ms[k] = 0.0;
  }
  return TVR_OK;
}

}  // extern "C"

extern "C" int tvr_gradient_map_norm(const tvr_system *csys, const float *x, const float *grad,
                                     double nu, double *out, void *stream) {
  tvr_system *sys = const_cast<tvr_system *>(csys);
  if (!sys || !x || !grad || !out || !(nu > 0.0) || !std::isfinite(nu))
    return fail(TVR_ERR_ARG, "tvr_gradient_map_norm: bad arguments");
  if (!is_device_ptr(x) || !is_device_ptr(grad))
    return fail(TVR_ERR_ARG, "tvr_gradient_map_norm: x and grad must be device memory");
  cudaStream_t s = (cudaStream_t)stream;
  launch_gmap_norm(x, grad, sys->N, nu, sys->ws, s);
  TVR_CUDA(cudaGetLastError());
  TVR_CUDA(cudaMemcpyAsync(out, sys->ws.gmap.out + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
  TVR_CUDA(cudaStreamSynchronize(s));
  return TVR_OK;
}

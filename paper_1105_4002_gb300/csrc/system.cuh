// The opaque tvr_system and host helpers shared by api.cu and solver.cu.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "tvr_internal.cuh"

int tvr_fail(int status, const std::string &msg);
int tvr_cuda_fail(cudaError_t e, const char *what);

#define TVR_CUDA(call)                                      \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return tvr_cuda_fail(e_, #call); \
  } while (0)

constexpr int kSlots = 6;

struct tvr_sweep_mem;  // device memory of parameter sweeps (sweep.cu)
void sweep_free(tvr_sweep_mem *m);
constexpr int kProfPairs = TVR_PROF_PAIRS;

struct tvr_system {
  int device = 0;
  int n = 0, V = 0, Pu = 0, Pv = 0, kind = 0;
  int64_t m = 0, N = 0, nnz = 0;
  MatStore A;  // padded CSR + CSC
  void *ws_mem = nullptr;
  Workspace ws{};
  // staging and scratch vectors (allocated on first use)
  float *stage_xN = nullptr, *stage_gN = nullptr, *stage_bM = nullptr, *stage_rM = nullptr;
  float *stage_rsM = nullptr;  // BF16 storage: scaled residual for the back projection
  float *stage_sweepX = nullptr;  // host x0 / x* of a sweep, 8 columns
  tvr_sweep_mem *sweep = nullptr;
  double *phi_ws = nullptr;  // 4 doubles
  // solver workspace (allocated on first solve)
  DevState *st = nullptr;
  float *vN[RN_COUNT] = {};
  float *vM[RM_COUNT] = {};
  float2 *pg = nullptr;
  float *wplanes[3] = {nullptr, nullptr, nullptr};  // Huber weight planes (4 N floats each)
  double *hist_dev = nullptr;
  int hist_cap = 0;
  int *pinned_flag = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaStream_t run_stream = nullptr;  // stream of this system's solve inside a batch
  cudaGraphExec_t pass_graph[PASS_KINDS] = {};
  int pass_graph_batch[PASS_KINDS] = {};
  // the same pass graphs with event nodes around every kernel (kernel timing)
  cudaGraphExec_t pass_graph_prof[PASS_KINDS] = {};
  int pass_graph_prof_batch[PASS_KINDS] = {};
  int pass_graph_prof_mask[PASS_KINDS] = {};  // profile | prof_stride << 8 the graph was captured with
  cudaEvent_t *gprof_ev = nullptr;  // [gprof_batch][TVR_PROF_KINDS][2]
  int gprof_batch = 0;
  // kernel timing: event pairs of launches not yet harvested; a pair counts
  // if it was a plain launch or if its kernel set its device "did work" flag
  int profile = 0;      // bit k set: launches of kind k are timed
  int prof_stride = 1;  // pass graphs: time passes i with i % prof_stride == 0
  cudaEvent_t prof_ev[TVR_PROF_KINDS][kProfPairs][2] = {};
  int prof_n[TVR_PROF_KINDS] = {};
  int prof_slot[TVR_PROF_KINDS][kProfPairs] = {};  // -1: plain launch, else device flag slot
  int *prof_flags_dev = nullptr;                   // [TVR_PROF_KINDS * kProfPairs]
  int *prof_flags_host = nullptr;                  // pinned copy
  double prof_ms[TVR_PROF_KINDS] = {};
  int64_t prof_cnt[TVR_PROF_KINDS] = {};

  MatDev mat() const {
    MatDev d{};
    d.n = n;
    d.div_n = make_fastdiv((uint32_t)n);
    d.div_nn = make_fastdiv((uint32_t)n * (uint32_t)n);
    d.m = m;
    d.N = N;
    d.nnz = A.nnz_pad;
    d.row_ptr = A.row_ptr;
    d.col = A.col;
    d.val = A.val;
    d.col_ptr = A.col_ptr;
    d.row = A.row;
    d.cval = A.cval;
    d.bf16 = coded16(A.storage);
    d.u16 = A.storage == TVR_STORAGE_U16_ROWSCALE;
    d.qval = A.qval;
    d.qcval = A.qcval;
    d.rscale = A.rscale;
    d.mf = A.storage == TVR_STORAGE_MATRIX_FREE;
    d.mfv = A.mfv;
    d.mfr = A.mfr;
    d.mfs = A.mfs;
    d.mfz = A.mfz;
    d.mfy = A.mfy;
    d.V = A.V;
    d.Pu = A.Pu;
    d.Pv = A.Pv;
    d.kind = A.kind;
    return d;
  }
};

inline int fail(int status, const std::string &msg) { return tvr_fail(status, msg); }
inline int cuda_fail(cudaError_t e, const char *what) { return tvr_cuda_fail(e, what); }

inline bool is_device_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

inline int ensure_vec(float **p, int64_t len) {
  if (*p) return TVR_OK;
  TVR_CUDA(cudaMalloc(p, sizeof(float) * (len > 0 ? len : 1)));
  return TVR_OK;
}

// Device pointer for an input vector: itself, or a staged copy of host data.
inline int stage_in(const float *src, int64_t len, float **stage, cudaStream_t s, const float **out) {
  if (is_device_ptr(src)) {
    *out = src;
    return TVR_OK;
  }
  int rc = ensure_vec(stage, len);
  if (rc) return rc;
  TVR_CUDA(cudaMemcpyAsync(*stage, src, sizeof(float) * len, cudaMemcpyHostToDevice, s));
  *out = *stage;
  return TVR_OK;
}

// Add the durations of all recorded launches that did work; synchronises on
// the recorded events.
inline int prof_harvest(tvr_system *sys) {
  bool dev = false;
  for (int k = 0; k < TVR_PROF_KINDS; ++k)
    for (int i = 0; i < sys->prof_n[k]; ++i) dev = dev || sys->prof_slot[k][i] >= 0;
  for (int k = 0; k < TVR_PROF_KINDS; ++k)
    if (sys->prof_n[k] > 0) TVR_CUDA(cudaEventSynchronize(sys->prof_ev[k][sys->prof_n[k] - 1][1]));
  if (dev) {
    TVR_CUDA(cudaMemcpy(sys->prof_flags_host, sys->prof_flags_dev, sizeof(int) * TVR_PROF_KINDS * kProfPairs,
                        cudaMemcpyDeviceToHost));
    TVR_CUDA(cudaMemset(sys->prof_flags_dev, 0, sizeof(int) * TVR_PROF_KINDS * kProfPairs));
  }
  for (int k = 0; k < TVR_PROF_KINDS; ++k) {
    for (int i = 0; i < sys->prof_n[k]; ++i) {
      const int sl = sys->prof_slot[k][i];
      if (sl >= 0 && !sys->prof_flags_host[k * kProfPairs + sl]) continue;
      float ms = 0.f;
      TVR_CUDA(cudaEventElapsedTime(&ms, sys->prof_ev[k][i][0], sys->prof_ev[k][i][1]));
      sys->prof_ms[k] += ms;
      sys->prof_cnt[k] += 1;
    }
    sys->prof_n[k] = 0;
  }
  return TVR_OK;
}

// Next event pair of kind k (-1 when profiling is off or the pool is full;
// callers harvest at points where no taken pair is still unrecorded).
inline int prof_take(tvr_system *sys, int k, bool device_flag) {
  if (!((sys->profile >> k) & 1) || sys->prof_n[k] >= kProfPairs) return -1;
  const int i = sys->prof_n[k]++;
  sys->prof_slot[k][i] = device_flag ? i : -1;
  return i;
}

inline void prof_mark(tvr_system *sys, int kind, int which, cudaStream_t s) {
  if (!((sys->profile >> kind) & 1)) return;
  if (which == 0) {
    if (sys->prof_n[kind] >= kProfPairs) prof_harvest(sys);
    const int i = prof_take(sys, kind, false);
    if (i >= 0) cudaEventRecord(sys->prof_ev[kind][i][0], s);
  } else if (sys->prof_n[kind] > 0) {
    cudaEventRecord(sys->prof_ev[kind][sys->prof_n[kind] - 1][1], s);
  }
}

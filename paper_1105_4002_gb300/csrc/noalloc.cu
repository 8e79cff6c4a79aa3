// phi and grad phi without any device allocation.
//
// Some callers must not allocate device memory at the moment they evaluate
// the objective: code whose device memory is owned by another framework's
// caching allocator under a fixed budget (an allocation outside it can fail
// or fragment what that allocator manages), and latency-bound loops that must
// not enter the driver's allocator (cudaMalloc / cudaFree can synchronise the
// device and take unbounded time).  tvr_phi_and_grad_noalloc serves them.  It
// runs the same kernels as tvr_phi_and_grad, but its scratch -- the residual
// vector and the reduction partials, counters and results -- lives in one
// file-scope device array of fixed size instead of the system's lazily
// allocated workspace.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "system.cuh"

namespace {

// Largest residual (rays) the static scratch holds.
constexpr int64_t kNoallocMaxRows = (int64_t)1 << 22;  // 4,194,304 rays = 16 MiB

constexpr size_t kPartBytes = sizeof(FF) * TVR_MAX_GRID * TVR_RMAX;  // 512 KiB per reduction slot
constexpr size_t kCounterBytes = 256;                                 // per slot, zeroed per call
constexpr size_t kOutBytes = 256;                                     // per slot
constexpr int kNoallocSlots = 3;                                      // forward, backward, TV value
constexpr size_t kPhiBytes = 256;
constexpr size_t kScratchBytes = kNoallocSlots * (kPartBytes + kCounterBytes + kOutBytes) +
                                 kPhiBytes + sizeof(float) * kNoallocMaxRows;
static_assert(kScratchBytes < ((size_t)18 << 20), "the documented size is about 17.5 MiB");

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once
// per device: in host code the symbol itself is only a host-side stand-in).
int scratch_address(int dev, unsigned char **out) {
  if (dev < 0 || dev >= kMaxDevices) return tvr_fail(TVR_ERR_ARG, "noalloc: device id out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return tvr_cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_addr[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_addr[dev];
  return TVR_OK;
}

}  // namespace

extern "C" int tvr_phi_and_grad_noalloc(const tvr_system *sys, const float *x, const float *b,
                                        double alpha, double tau, double *phi_dev,
                                        double *phi_host, float *grad, void *stream) {
  if (!sys || !x || !b) return tvr_fail(TVR_ERR_ARG, "tvr_phi_and_grad_noalloc: null argument");
  if (!(alpha >= 0.0) || !(tau > 0.0) || !std::isfinite(alpha) || !std::isfinite(tau))
    return tvr_fail(TVR_ERR_ARG, "tvr_phi_and_grad_noalloc: need alpha >= 0 and tau > 0");
  // 16-bit coded storage (BF16 or U16 codes with row scales) gathers a second,
  // row-scaled residual in the back projection, which the static scratch does
  // not hold
  if (sys->A.storage != TVR_STORAGE_FP32 && sys->A.storage != TVR_STORAGE_MATRIX_FREE)
    return tvr_fail(TVR_ERR_ARG,
                    "tvr_phi_and_grad_noalloc: needs FP32 or matrix-free storage (BF16 or U16 "
                    "row-scale storage would need a second residual)");
  if (sys->m > kNoallocMaxRows)
    return tvr_fail(TVR_ERR_ARG,
                    "tvr_phi_and_grad_noalloc: the system has more rays than the static scratch "
                    "holds (m > 4194304); use tvr_phi_and_grad");
  if (!is_device_ptr(x) || !is_device_ptr(b) || (grad && !is_device_ptr(grad)) ||
      (phi_dev && !is_device_ptr(phi_dev)))
    return tvr_fail(TVR_ERR_ARG,
                    "tvr_phi_and_grad_noalloc: x, b, grad and phi_dev must be device memory");
  int dev = 0;
  TVR_CUDA(cudaGetDevice(&dev));
  if (dev != sys->device)
    return tvr_fail(TVR_ERR_ARG, "tvr_phi_and_grad_noalloc: the system lives on another device");
  unsigned char *base = nullptr;
  if (int rc = scratch_address(dev, &base)) return rc;
  cudaStream_t s = (cudaStream_t)stream;

  // carve the scratch: [slot partials | counters | outputs] x 3, phi, residual
  Workspace ws = sys->ws;
  RedSlot *slots[kNoallocSlots] = {&ws.fwd, &ws.bwd, &ws.tv};
  unsigned char *p = base;
  for (int k = 0; k < kNoallocSlots; ++k) {
    slots[k]->partials = reinterpret_cast<FF *>(p);
    slots[k]->counter = reinterpret_cast<unsigned *>(p + kPartBytes);
    slots[k]->out = reinterpret_cast<double *>(p + kPartBytes + kCounterBytes);
    p += kPartBytes + kCounterBytes + kOutBytes;
  }
  double *phi_static = reinterpret_cast<double *>(p);
  float *r = reinterpret_cast<float *>(p + kPhiBytes);
  // the arrival counters must start at zero; a previous call's values remain otherwise
  for (int k = 0; k < kNoallocSlots; ++k)
    TVR_CUDA(cudaMemsetAsync(slots[k]->counter, 0, kCounterBytes, s));

  double *pd = phi_dev ? phi_dev : phi_static;
  const MatDev A = sys->mat();
  launch_forward(A, x, b, r, ws, s);
  if (grad)
    launch_backward(A, r, x, (float)alpha, (float)tau, grad, ws, pd, s);
  else
    launch_tv_value(A, x, (float)alpha, (float)tau, ws, pd, s);
  TVR_CUDA(cudaGetLastError());
  if (phi_host) {
    TVR_CUDA(cudaMemcpyAsync(phi_host, pd, sizeof(double) * 3, cudaMemcpyDeviceToHost, s));
    TVR_CUDA(cudaStreamSynchronize(s));
  }
  return TVR_OK;
}

// FP64 variants of phi / grad phi and the vector-Jacobian products of phi.
//
// The FP64 kernels serve verification by finite differences (gradcheck with
// h = 1e-6 needs double precision end to end); they read the same padded
// FP32 matrix as the hot path, promoted to double, so they differentiate the
// same function.  The VJP kernels are the backward of phi(x; b):
//   d phi / d x = A^T (A x - b) + alpha grad TV_tau(x),   d phi / d b = -(A x - b),
// each times the upstream scalar, from the residual saved by the forward.
#include "tvr_internal.cuh"

#define FULL 0xffffffffu

namespace {

constexpr int kLanes = 4;

__device__ __forceinline__ double dgroup_sum(double v) {
#pragma unroll
  for (int o = kLanes / 2; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o, kLanes);
  return v;
}

// Deterministic grid reduction of R doubles (block order), result in thread 0
// of the last block.  The partials buffer of the slot holds 8 bytes per entry.
template <int R>
__device__ bool grid_reduce_d(double (&a)[R], const RedSlot &slot, double (&tot)[R]) {
  __shared__ double sh[TVR_BLOCK / 32][R];
  __shared__ bool am_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double *part = reinterpret_cast<double *>(slot.partials);
  for (int k = 0; k < R; ++k) {
    for (int o = 16; o > 0; o >>= 1) a[k] += __shfl_down_sync(FULL, a[k], o);
    if (lane == 0) sh[warp][k] = a[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < R; ++k) {
      double v = 0.0;
      for (int w = 0; w < TVR_BLOCK / 32; ++w) v += sh[w][k];
      part[blockIdx.x * R + k] = v;
    }
    __threadfence();
    am_last = atomicAdd(slot.counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  if (threadIdx.x == 0) {
    for (int k = 0; k < R; ++k) {
      double v = 0.0;
      for (unsigned b = 0; b < gridDim.x; ++b) v += __ldcg(part + b * R + k);
      tot[k] = v;
      slot.out[k] = v;
    }
    *slot.counter = 0u;
  }
  return true;
}

__device__ __forceinline__ void huber_d(const double *__restrict__ x, int ix, int iy, int iz, int n,
                                        double tau, double w[3], double &h) {
  if (ix < 0 || iy < 0 || iz < 0) {
    w[0] = w[1] = w[2] = 0.0;
    h = 0.0;
    return;
  }
  const int64_t j = (int64_t)ix + (int64_t)n * (iy + (int64_t)n * iz);
  const double c = x[j];
  double z[3];
  z[0] = ix + 1 < n ? x[j + 1] - c : 0.0;
  z[1] = iy + 1 < n ? x[j + n] - c : 0.0;
  z[2] = iz + 1 < n ? x[j + (int64_t)n * n] - c : 0.0;
  const double nrm = sqrt(z[0] * z[0] + z[1] * z[1] + z[2] * z[2]);
  const double den = nrm > tau ? nrm : tau;
  for (int e = 0; e < 3; ++e) w[e] = z[e] / den;
  h = nrm >= tau ? nrm - 0.5 * tau : nrm * nrm / (2.0 * tau);
}

// r = A x - b (b may be null: r = A x); sum r^2.
__global__ void __launch_bounds__(TVR_BLOCK)
    k_forward_f64(MatDev A, const double *__restrict__ x, const double *__restrict__ b,
                  double *__restrict__ r, RedSlot slot) {
  const int lane = threadIdx.x & (kLanes - 1);
  const int sub = (threadIdx.x & 31) / kLanes;
  const int64_t warp = ((int64_t)blockIdx.x * TVR_BLOCK + threadIdx.x) >> 5;
  const int64_t nwarp = (int64_t)gridDim.x * (TVR_BLOCK / 32);
  double acc = 0.0;
  for (int64_t base = warp * (32 / kLanes); base < A.m; base += nwarp * (32 / kLanes)) {
    const int64_t row = base + sub;
    const bool valid = row < A.m;
    const int64_t beg = valid ? A.row_ptr[row] : 0, end = valid ? A.row_ptr[row + 1] : 0;
    double s = 0.0;
    for (int64_t e0 = beg + 4 * lane; e0 < end; e0 += 4 * kLanes) {
      const int4 c4 = *reinterpret_cast<const int4 *>(A.col + e0);
      const float4 v4 = *reinterpret_cast<const float4 *>(A.val + e0);
      s = fma((double)v4.x, x[c4.x], s);
      s = fma((double)v4.y, x[c4.y], s);
      s = fma((double)v4.z, x[c4.z], s);
      s = fma((double)v4.w, x[c4.w], s);
    }
    s = dgroup_sum(s);
    if (valid && lane == 0) {
      const double ri = b ? s - b[row] : s;
      r[row] = ri;
      acc += ri * ri;
    }
  }
  double a[1] = {acc}, tot[1];
  grid_reduce_d<1>(a, slot, tot);
}

// MODE 0: g = A^T r + alpha grad TV(x), TV value, phi from data_in.
// MODE 1: VJP: g = scale (A^T r + alpha grad TV(x)), gb = -scale r.
template <int MODE>
__global__ void __launch_bounds__(TVR_BLOCK)
    k_backward_f64(MatDev A, const double *__restrict__ r, const double *__restrict__ x, double alpha,
                   double tau, const double *__restrict__ scale_p, double *__restrict__ g,
                   double *__restrict__ gb, RedSlot slot, const double *__restrict__ data_in,
                   double *phi_dev) {
  const int n = A.n;
  const int lane = threadIdx.x & (kLanes - 1);
  const int sub = (threadIdx.x & 31) / kLanes;
  const int64_t warp = ((int64_t)blockIdx.x * TVR_BLOCK + threadIdx.x) >> 5;
  const int64_t nwarp = (int64_t)gridDim.x * (TVR_BLOCK / 32);
  const double scale = MODE == 1 ? *scale_p : 1.0;
  double tv = 0.0;
  for (int64_t base = warp * (32 / kLanes); base < A.N; base += nwarp * (32 / kLanes)) {
    const int64_t j = base + sub;
    const bool valid = j < A.N;
    const int64_t beg = valid ? A.col_ptr[j] : 0, end = valid ? A.col_ptr[j + 1] : 0;
    double s = 0.0;
    for (int64_t e0 = beg + 4 * lane; e0 < end; e0 += 4 * kLanes) {
      const int4 i4 = *reinterpret_cast<const int4 *>(A.row + e0);
      const float4 v4 = *reinterpret_cast<const float4 *>(A.cval + e0);
      s = fma((double)v4.x, r[i4.x], s);
      s = fma((double)v4.y, r[i4.y], s);
      s = fma((double)v4.z, r[i4.z], s);
      s = fma((double)v4.w, r[i4.w], s);
    }
    s = dgroup_sum(s);
    int ix, iy, iz;
    voxel_of(A, j, ix, iy, iz);
    double w[3] = {0.0, 0.0, 0.0}, h = 0.0, c = 0.0;
    if (valid) {
      huber_d(x, ix - (lane == 1), iy - (lane == 2), iz - (lane == 3), n, tau, w, h);
      c = lane == 0 ? -(w[0] + w[1] + w[2]) : (lane == 1 ? w[0] : (lane == 2 ? w[1] : w[2]));
    }
    c += __shfl_down_sync(FULL, c, 2, kLanes);
    c += __shfl_down_sync(FULL, c, 1, kLanes);
    if (valid && lane == 0) {
      g[j] = scale * (s + alpha * c);
      tv += h;
    }
  }
  if (MODE == 1) {
    if (gb) {
      const int64_t stride = (int64_t)gridDim.x * TVR_BLOCK;
      for (int64_t i = (int64_t)blockIdx.x * TVR_BLOCK + threadIdx.x; i < A.m; i += stride)
        gb[i] = -scale * r[i];
    }
    return;
  }
  double a[1] = {tv}, tot[1];
  if (grid_reduce_d<1>(a, slot, tot) && threadIdx.x == 0 && phi_dev) {
    const double data = 0.5 * data_in[0];
    phi_dev[0] = data + alpha * tot[0];
    phi_dev[1] = data;
    phi_dev[2] = tot[0];
  }
}

}  // namespace

void launch_forward_f64(const MatDev &A, const double *x, const double *b, double *r,
                        const Workspace &ws, cudaStream_t s) {
  k_forward_f64<<<ws.grid_fwd, TVR_BLOCK, 0, s>>>(A, x, b, r, ws.fwd);
}

void launch_backward_f64(const MatDev &A, const double *r, const double *x, double alpha,
                         double tau, double *g, const Workspace &ws, double *phi_dev,
                         cudaStream_t s) {
  k_backward_f64<0><<<ws.grid_bwd, TVR_BLOCK, 0, s>>>(A, r, x, alpha, tau, nullptr, g, nullptr,
                                                      ws.bwd, ws.fwd.out, phi_dev);
}

void launch_vjp_f64(const MatDev &A, const double *r, const double *x, double alpha, double tau,
                    const double *scale, double *gx, double *gb, const Workspace &ws,
                    cudaStream_t s) {
  k_backward_f64<1><<<ws.grid_bwd, TVR_BLOCK, 0, s>>>(A, r, x, alpha, tau, scale, gx, gb, ws.bwd,
                                                      nullptr, nullptr);
}

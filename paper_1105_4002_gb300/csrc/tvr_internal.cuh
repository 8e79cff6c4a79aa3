// Internal declarations of libtvr: device helpers, solver state, launchers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tvr.h"

#define TVR_BLOCK 256          // threads per block of every streaming kernel
#define TVR_RMAX 16            // reductions carried by one kernel
#define TVR_MAX_GRID 4096      // upper bound on blocks of a reducing kernel
#define TVR_PROF_PAIRS 4096    // timed launches held per kernel kind between harvests
#define TVR_PROF_KINDS 4       // forward, back projection, step, UPN extrapolation

// ---------------------------------------------------------------------------
// Double-single ("float-float") accumulation.
//
// GB300 executes FP64 at about 1/64 of the FP32 rate, so per-element FP64
// arithmetic would cost more than the HBM traffic of the streaming kernels.
// Sums are therefore carried as an unevaluated pair hi + lo of floats:
// TwoSum (Knuth) gives the exact rounding error of each addition and TwoProd
// (via fmaf) the exact error of each product, so a product of two floats is
// accumulated without loss and the pair keeps about 48 significant bits.  The
// pair is turned into a double once per reduction.  Every combination order
// is fixed, so the results are deterministic.
// ---------------------------------------------------------------------------
struct __align__(8) FF {
  float hi, lo;
};

__device__ __forceinline__ FF ff_zero() { return FF{0.f, 0.f}; }

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void ff_add(FF &a, float b) {
  float s, e;
  two_sum(a.hi, b, s, e);
  a.hi = s;
  a.lo = __fadd_rn(a.lo, e);
}

// a += x * y with the product's rounding error kept.
__device__ __forceinline__ void ff_add_prod(FF &a, float x, float y) {
  float p = __fmul_rn(x, y);
  float pe = __fmaf_rn(x, y, -p);
  ff_add(a, p);
  a.lo = __fadd_rn(a.lo, pe);
}

__device__ __forceinline__ FF ff_merge(FF a, FF b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  float hi = __fadd_rn(s, e);
  float lo = __fsub_rn(e, __fsub_rn(hi, s));
  return FF{hi, lo};
}

__device__ __forceinline__ FF ff_shfl_down(FF a, int off) {
  FF b;
  b.hi = __shfl_down_sync(0xffffffffu, a.hi, off);
  b.lo = __shfl_down_sync(0xffffffffu, a.lo, off);
  return b;
}

__device__ __forceinline__ double ff_to_double(FF a) { return (double)a.hi + (double)a.lo; }

// Reduction workspace of one kernel: per-block partials and an arrival counter.
struct RedSlot {
  FF *partials;        // [TVR_MAX_GRID * TVR_RMAX]
  unsigned *counter;   // reset to 0 by the finishing block
  double *out;         // [TVR_RMAX] final sums (FP64)
};

__device__ __forceinline__ FF ff_shfl_xor(FF a, int mask) {
  FF b;
  b.hi = __shfl_xor_sync(0xffffffffu, a.hi, mask);
  b.lo = __shfl_xor_sync(0xffffffffu, a.lo, mask);
  return b;
}

// Warp-wide reduce-scatter of R <= 16 pairs (padded to P, a power of two):
// each exchange step at lane distance 16, 8, ... keeps one half of the values
// a lane carries and merges the partner's copy of that half, so that after
// log2 P steps lane l carries value k = l / (32 / P) alone; the remaining
// steps reduce it within the group of 32 / P lanes.  R values cost
// (P - 1) + 5 - log2 P merges instead of 5 R.  ff_merge is commutative, so
// both partners of an exchange hold the same result.
template <int R>
struct RedShape {
  static_assert(R >= 1 && R <= 16, "R");
  static constexpr int P = R == 1 ? 1 : (R == 2 ? 2 : (R <= 4 ? 4 : (R <= 8 ? 8 : 16)));
};

template <int R>
__device__ __forceinline__ FF warp_reduce_scatter(const FF (&a)[R]) {
  constexpr int P = RedShape<R>::P;
  const int lane = threadIdx.x & 31;
  FF v[P];
#pragma unroll
  for (int k = 0; k < P; ++k) v[k] = k < R ? a[k < R ? k : 0] : ff_zero();
  int off = 16;
#pragma unroll
  for (int cnt = P / 2; cnt >= 1; cnt >>= 1, off >>= 1) {
    const bool hi = lane & off;
#pragma unroll
    for (int i = 0; i < cnt; ++i) {
      const FF keep = hi ? v[cnt + i] : v[i];
      const FF send = hi ? v[i] : v[cnt + i];
      v[i] = ff_merge(keep, ff_shfl_xor(send, off));
    }
  }
#pragma unroll
  for (; off > 0; off >>= 1) v[0] = ff_merge(v[0], ff_shfl_xor(v[0], off));
  return v[0];
}

// Block-wide reduction of R pairs; the result is valid in every thread.
// Warps reduce-scatter; then thread t < P W (W warps) holds value t / W of
// warp t % W and the groups of W lanes reduce.
template <int R>
__device__ __forceinline__ void block_reduce(FF (&a)[R]) {
  constexpr int P = RedShape<R>::P;
  constexpr int W = TVR_BLOCK / 32;
  constexpr int L = 32 / P;
  constexpr int T2 = (P * W + 31) / 32 * 32;  // threads of the second stage (whole warps)
  static_assert((W & (W - 1)) == 0 && T2 <= TVR_BLOCK, "block shape");
  __shared__ FF sh[P][W];
  __shared__ FF res[P];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const FF v = warp_reduce_scatter<R>(a);
  if ((lane & (L - 1)) == 0) sh[lane / L][warp] = v;
  __syncthreads();
  if (threadIdx.x < T2) {
    const int t = threadIdx.x;
    FF u = t < P * W ? sh[t / W][t % W] : ff_zero();
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) u = ff_merge(u, ff_shfl_xor(u, o));
    if (t < P * W && t % W == 0) res[t / W] = u;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < R; ++k) a[k] = res[k];
}

// Grid-wide deterministic reduction.  Every block stores its partial; the last
// block to arrive sums all partials in block order and returns true in all of
// its threads, with the FP64 totals in `tot` (valid in thread 0) and in
// slot.out.  No thread ever waits on another block.
template <int R>
__device__ __forceinline__ bool grid_reduce(FF (&a)[R], const RedSlot &slot, double (&tot)[R]) {
  __shared__ bool am_last;
  block_reduce<R>(a);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < R; ++k) slot.partials[blockIdx.x * R + k] = a[k];
    __threadfence();
    unsigned t = atomicAdd(slot.counter, 1u);
    am_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  FF s[R];
#pragma unroll
  for (int k = 0; k < R; ++k) s[k] = ff_zero();
  for (int i = threadIdx.x; i < (int)gridDim.x; i += TVR_BLOCK) {
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const float2 v = __ldcg(reinterpret_cast<const float2 *>(slot.partials + i * R + k));
      s[k] = ff_merge(s[k], FF{v.x, v.y});
    }
  }
  block_reduce<R>(s);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < R; ++k) {
      tot[k] = ff_to_double(s[k]);
      slot.out[k] = tot[k];
    }
    *slot.counter = 0u;
  }
  return true;
}

// ---------------------------------------------------------------------------
// Huber weight of one voxel: z = D_k x (forward differences, 0 across the
// border), returns w = z / max(tau, |z|), |z| and h_tau(z).  A voxel outside
// the grid yields w = 0.
// ---------------------------------------------------------------------------
struct Huber {
  float z[3];
  float w[3];
  float nrm;
  float h;
};

__device__ __forceinline__ float huber_h(float nrm, float tau) {
  return nrm >= tau ? __fsub_rn(nrm, 0.5f * tau) : __fdiv_rn(__fmul_rn(nrm, nrm), 2.f * tau);
}

__device__ __forceinline__ void diff3(const float *__restrict__ x, int ix, int iy, int iz, int n,
                                      float z[3]) {
  const int64_t j = (int64_t)ix + (int64_t)n * (iy + (int64_t)n * iz);
  const float c = __ldg(x + j);
  z[0] = ix + 1 < n ? __fsub_rn(__ldg(x + j + 1), c) : 0.f;
  z[1] = iy + 1 < n ? __fsub_rn(__ldg(x + j + n), c) : 0.f;
  z[2] = iz + 1 < n ? __fsub_rn(__ldg(x + j + (int64_t)n * n), c) : 0.f;
}

__device__ __forceinline__ float norm3(const float z[3]) {
  return __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(z[0], z[0]), __fmul_rn(z[1], z[1])),
                              __fmul_rn(z[2], z[2])));
}

// Huber weights of a difference vector z with |z| = nrm: w_e = z_e / max(tau, |z|),
// as one correctly rounded reciprocal and three products.
__device__ __forceinline__ void huber_weights(const float z[3], float nrm, float tau, float w[3]) {
  const float r = __frcp_rn(fmaxf(tau, nrm));
#pragma unroll
  for (int e = 0; e < 3; ++e) w[e] = __fmul_rn(z[e], r);
}

__device__ __forceinline__ void huber_at(const float *__restrict__ x, int ix, int iy, int iz,
                                         int n, float tau, Huber &o) {
  if (ix < 0 || iy < 0 || iz < 0) {
    o.z[0] = o.z[1] = o.z[2] = 0.f;
    o.w[0] = o.w[1] = o.w[2] = 0.f;
    o.nrm = 0.f;
    o.h = 0.f;
    return;
  }
  diff3(x, ix, iy, iz, n, o.z);
  o.nrm = norm3(o.z);
  huber_weights(o.z, o.nrm, tau, o.w);
  o.h = huber_h(o.nrm, tau);
}

// Bregman divergence of h_tau at base z evaluated at zb = z + dlt:
//   h(zb) - h(z) - w(z) . dlt  (>= 0),
// in a form without cancellation when both points lie in the same zone:
//   quadratic zone: |dlt|^2 / (2 tau);
//   linear zone:    |z x dlt|^2 / (|z| (|zb||z| + z.zb))  when z.zb > 0.
__device__ __forceinline__ float huber_bregman_n(const float z[3], float nz, const float zb[3],
                                                 float nb, const float dlt[3], float tau) {
  if (nz < tau && nb < tau) {
    const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dlt[0], dlt[0]), __fmul_rn(dlt[1], dlt[1])),
                               __fmul_rn(dlt[2], dlt[2]));
    return __fdiv_rn(d2, 2.f * tau);
  }
  const float dot = __fadd_rn(__fadd_rn(__fmul_rn(z[0], zb[0]), __fmul_rn(z[1], zb[1])),
                              __fmul_rn(z[2], zb[2]));
  if (nz >= tau && nb >= tau && dot > 0.f) {
    const float c0 = __fsub_rn(__fmul_rn(z[1], dlt[2]), __fmul_rn(z[2], dlt[1]));
    const float c1 = __fsub_rn(__fmul_rn(z[2], dlt[0]), __fmul_rn(z[0], dlt[2]));
    const float c2 = __fsub_rn(__fmul_rn(z[0], dlt[1]), __fmul_rn(z[1], dlt[0]));
    const float cc = __fadd_rn(__fadd_rn(__fmul_rn(c0, c0), __fmul_rn(c1, c1)), __fmul_rn(c2, c2));
    return __fdiv_rn(cc, __fmul_rn(nz, __fadd_rn(__fmul_rn(nb, nz), dot)));
  }
  const float den = fmaxf(tau, nz);
  const float wd = __fdiv_rn(__fadd_rn(__fadd_rn(__fmul_rn(z[0], dlt[0]), __fmul_rn(z[1], dlt[1])),
                                       __fmul_rn(z[2], dlt[2])),
                             den);
  const float b = __fsub_rn(__fsub_rn(huber_h(nb, tau), huber_h(nz, tau)), wd);
  return fmaxf(b, 0.f);
}

__device__ __forceinline__ float huber_bregman(const float z[3], float nz, const float zb[3],
                                               const float dlt[3], float tau) {
  return huber_bregman_n(z, nz, zb, norm3(zb), dlt, tau);
}


// ---------------------------------------------------------------------------
// Solver state, resident in device memory.  Control scalars are FP64 and are
// only touched by one thread (the finishing block of a reducing kernel).
// Vector roles are pointers that the control logic swaps on acceptance.
// ---------------------------------------------------------------------------
enum SolverKind { SOLVER_NONE = 0, SOLVER_GP = 1, SOLVER_GPBB = 2, SOLVER_UPN = 3 };
// Kind of solver pass (graph cache slot): the solver, or GPBB with two trial
// points per forward pass.
enum { PASS_GPBB2 = 4, PASS_KINDS = 5 };

// Y2, RY2, U2, RYS2: UPN's extrapolation formed speculatively by each trial
// (the values y, A y - b, u would take if the trial is accepted); they swap
// with Y, RY, U, RYS on acceptance.
// T2, RT2, RTS2: GPBB's second trial point of a pass (step beta^2 theta).
enum RoleN { RN_X = 0, RN_T, RN_Y, RN_G, RN_GN, RN_Y2, RN_T2, RN_COUNT };
// RS, RTS, RYS: the residuals R, RT, RY times the per-row scales (BF16 storage
// only), which the back projection gathers so that it applies the same
// matrix s_i q_ij as the forward projection.
enum RoleM { RM_R = 0, RM_RT, RM_RY, RM_U, RM_AD, RM_RY2, RM_U2, RM_RT2, RM_RS, RM_RTS, RM_RYS,
             RM_RYS2, RM_RTS2, RM_COUNT };

#define TVR_FHIST 16

struct DevState {
  // configuration
  double alpha, tau, eps, rho, sigma, beta0, Lbar, mubar;
  int kmax, K, max_trials, bt_max, stop_mode, solver;
  int64_t N;
  const float *b;  // data vector (device)
  // control scalars
  double L, Lt, theta, beta, beta_prev, mu, M;
  int M_valid;
  double step, step2;           // step size of the trial's projected step; GPBB: theta for G
  double f_cur, fhist[TVR_FHIST];
  int nhist;
  double gnorm, gnorm0, stopval, gnorm_trial;
  int k, trial, need_grad, done, status;
  int total_trials, f_evals, g_evals;
  // reduction results
  double r_init[TVR_RMAX], r_fwd[TVR_RMAX], r_bwd[TVR_RMAX], r_step[TVR_RMAX], r_yf[TVR_RMAX];
  // UPN with the extrapolation fused into the trial kernel: the trial also
  // forms y, u, A y - b and the Huber weights of y for the case of acceptance
  // (roles Y2, U2, RY2, RYS2 and the planes wt) with the reductions r_spec =
  // {||x+ - x||^2, ||u||^2, sum_j B_h(D_j x+; D_j y)}; ctrl_trial adopts them
  // on acceptance.
  int spec_upn;
  double r_spec[3];
  // GPBB with two trial points per pass: the second point's sums
  // {||A xbar2 - b||^2, ||A d2||^2} and {g^T d2, ||d2||^2, sum B_h, TV_tau(xbar2)}
  double r_fwd2[2], r_step2[4];
  // vector roles
  float *vN[RN_COUNT];
  float *vM[RM_COUNT];
  float2 *pg;  // (p_j, g_j): base point of the next trial and the gradient there,
               // written by the back projection (solver and init modes)
  // Huber weights w_e(D_j v) of the point v where the next gradient is taken,
  // as 4 planes of N floats: w_0, w_1, w_2 and (w_0 + w_1) + w_2.  `w` holds
  // them for the current gradient point; each trial writes `wt` for the point
  // its acceptance would make the next gradient point (xbar for GP / GPBB, y
  // for UPN), and the two swap on acceptance.  The back projection then reads
  // the TV gradient instead of re-evaluating the stencil.
  float *w, *wt, *wt2;  // wt2: planes at GPBB's second trial point
  // history (device buffer of hist_cap records)
  double *hist;
  int hist_cap, hist_used;
  // kernel-timing flags: prof_flags[kind * TVR_PROF_PAIRS + slot] = 1 when a
  // timed launch did work (kind 0 forward, 1 back projection, 2 step, 3 extrapolation)
  int *prof_flags;
};

// ---------------------------------------------------------------------------
// Device views of A and launch shapes.
// ---------------------------------------------------------------------------
// Unsigned division by an invariant divisor d >= 1 with a multiply-high, an
// add and a shift (Granlund and Montgomery, "Division by invariant integers
// using multiplication", 1994, Sec. 4): l = ceil(log2 d),
// m = floor(2^32 (2^l - d) / d) + 1, q = (mulhi(u, m) + u) >> l, exact for
// every u < 2^31 (the sum cannot overflow).  Voxel indices are below 2^31
// because the stored indices are int32.
struct FastDiv {
  uint32_t d, m, l;
};

inline FastDiv make_fastdiv(uint32_t d) {
  uint32_t l = 0;
  while (l < 32 && (uint64_t(1) << l) < d) ++l;
  const uint64_t m = ((uint64_t(1) << 32) * ((uint64_t(1) << l) - d)) / d + 1;
  return FastDiv{d, (uint32_t)m, l};
}

__device__ __forceinline__ uint32_t fast_div(uint32_t u, const FastDiv &f) {
  return (__umulhi(u, f.m) + u) >> f.l;
}

struct MfView;  // matrix-free view constants (mf.cuh)

struct MatDev {
  int n;
  FastDiv div_n, div_nn;   // divisors n and n^2 of the voxel index
  int64_t m, N, nnz;
  const int64_t *row_ptr;  // CSR [m+1], every row padded to a multiple of 4 entries
  const int32_t *col;      // [stored]
  const float *val;        // [stored]
  const int64_t *col_ptr;  // CSC [N+1], every column padded to a multiple of 4 entries
  const int32_t *row;      // [stored]
  const float *cval;       // [stored]
  // 16-bit coded storage (BF16 or U16): a_ij = rscale[i] * q_ij, the same
  // codes q in CSR and CSC; u16 selects the code format (decode16)
  int bf16;
  int u16;
  const __nv_bfloat16 *qval;   // CSR codes [stored]
  const __nv_bfloat16 *qcval;  // CSC codes [stored]
  const float *rscale;         // [m]
  // matrix-free storage: no arrays above; view constants and scan shape
  int mf;
  const MfView *mfv;
  // per-ray constants of the matrix-free projector (mf.cuh, mf_ray_table):
  // {1/d_x, 1/d_y, 1/d_z, |d|} per ray, and the ray start for parallel beam
  const float4 *mfr, *mfs;
  // all views separable (MfView::sep): k_mf_adjoint_sep writes A^T r here
  // and the back projection reads it instead of enumerating pixels; else null
  float *mfz;
  // all views separable: k_mf_forward_sep writes up to 4 blocks of m row sums
  // here and the forward projection reads them instead of walking its rays
  float *mfy;
  int V, Pu, Pv, kind;
};

// Loads of the streamed matrix arrays (indices, values): read once per
// projection, so they bypass L1 allocation and leave L1 to the gathered
// vector, which neighbouring rows and columns reuse.
__device__ __forceinline__ int4 ld_stream(const int32_t *p) {
  int4 v;
  asm("ld.global.nc.L1::no_allocate.v4.s32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}
__device__ __forceinline__ float4 ld_stream(const float *p) {
  float4 v;
  asm("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}
__device__ __forceinline__ uint2 ld_stream2(const void *p) {
  uint2 v;
  asm("ld.global.nc.L1::no_allocate.v2.u32 {%0,%1}, [%2];"
               : "=r"(v.x), "=r"(v.y)
               : "l"(p));
  return v;
}

// Four stored 16-bit codes (two 32-bit words, the first code in the low half)
// widened to float32: bfloat16 codes (the upper half of a float32's bits), or
// 16-bit unsigned fixed-point codes (the integer itself, exact in float32; the
// row scale carries the step).  The format is a compile-time choice of each
// kernel instance.
template <bool U16>
__device__ __forceinline__ float4 decode16(uint2 raw) {
  if (U16)
    return make_float4(__uint2float_rn(raw.x & 0xffffu), __uint2float_rn(raw.x >> 16),
                       __uint2float_rn(raw.y & 0xffffu), __uint2float_rn(raw.y >> 16));
  return make_float4(__uint_as_float(raw.x << 16), __uint_as_float(raw.x & 0xffff0000u),
                     __uint_as_float(raw.y << 16), __uint_as_float(raw.y & 0xffff0000u));
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may be scheduled while its predecessor on the stream is still
// running.  It lets its own successor do the same, then waits until the
// predecessor has completed and its writes are visible; nothing before the
// wait touches memory.  Without a programmatic dependency both are no-ops.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// (ix, iy, iz) of voxel j = ix + n (iy + n iz).
__device__ __forceinline__ void voxel_of(const MatDev &A, int64_t j, int &ix, int &iy, int &iz) {
  const uint32_t u = (uint32_t)j;
  const uint32_t z = fast_div(u, A.div_nn);
  const uint32_t rem = u - z * A.div_nn.d;
  const uint32_t y = fast_div(rem, A.div_n);
  iz = (int)z;
  iy = (int)y;
  ix = (int)(rem - y * A.div_n.d);
}

struct Workspace {
  RedSlot fwd, bwd, step, yf, tv, gmap;
  int grid_fwd, grid_bwd, grid_elem, grid_trial, grid_trial_x, grid_trial_2;
  int grid_mfsep;  // k_mf_adjoint_sep (0: not used by this system)
  int grid_mfsep_fwd[3];  // k_mf_forward_sep with 1, 2, 4 sums
};

// Launchers (kernels.cu).  `st` selects solver mode (pointers and scalars from
// the device state); st == nullptr is the plain mode with explicit pointers.
void launch_forward(const MatDev &A, const float *x, const float *b, float *r, const Workspace &ws,
                    cudaStream_t s, float *rs = nullptr);
void launch_forward_plain(const MatDev &A, const float *x, float *y, const Workspace &ws,
                          cudaStream_t s);
void launch_backward(const MatDev &A, const float *r, const float *x, float alpha, float tau,
                     float *g, const Workspace &ws, double *phi_dev, cudaStream_t s);
void launch_adjoint_plain(const MatDev &A, const float *r, float *z, const Workspace &ws,
                          cudaStream_t s);
void launch_vjp(const MatDev &A, const float *r, const float *x, float alpha, float tau,
                const double *scale, float *gx, float *gb, const Workspace &ws, cudaStream_t s);
void launch_forward_f64(const MatDev &A, const double *x, const double *b, double *r,
                        const Workspace &ws, cudaStream_t s);
void launch_backward_f64(const MatDev &A, const double *r, const double *x, double alpha,
                         double tau, double *g, const Workspace &ws, double *phi_dev,
                         cudaStream_t s);
void launch_vjp_f64(const MatDev &A, const double *r, const double *x, double alpha, double tau,
                    const double *scale, double *gx, double *gb, const Workspace &ws,
                    cudaStream_t s);
void launch_tv_value(const MatDev &A, const float *x, float alpha, float tau, const Workspace &ws,
                     double *phi_dev, cudaStream_t s);
void launch_project(float *x, int64_t n, cudaStream_t s);
void launch_gmap_norm(const float *x, const float *g, int64_t n, double nu, const Workspace &ws,
                      cudaStream_t s);

// Solver-mode launchers (pointers and scalars come from the device state).
void launch_solver_init(const MatDev &A, DevState *st, const Workspace &ws, cudaStream_t s);
// Optional CUDA-event timing of the launches of one pass (kinds: 0 forward,
// 1 back projection, 2 step, 3 extrapolation): events recorded around each
// launch, and the launch's slot for its "did work" flag (-1: not timed).
struct PassTiming {
  cudaEvent_t ev[TVR_PROF_KINDS][2];
  int slot[TVR_PROF_KINDS];
  bool graph_nodes = false;  // record as event nodes of a graph being captured
};
void launch_solver_pass(const MatDev &A, DevState *st, int solver, const Workspace &ws,
                        cudaStream_t s, const PassTiming *timing = nullptr);
// The single-point trial kernel alone (GP mode), for tvr_trial_sums.
void launch_trial(const MatDev &A, DevState *st, const Workspace &ws, cudaStream_t s);

// Construction of A (build_system.cu).  Rows of the CSR and columns of the
// CSC are padded to multiples of 4 entries (padding: the last real index with
// value 0) so that every lane reads 4 entries with one 16-byte load; row_len /
// col_len keep the real counts.
// Stored order of a padded row or column of length L (a multiple of 4).  In
// each block of 16 entries (the last block may hold 4, 8 or 12), the 4-entry
// group that lane l of a 4-lane group loads holds the entries l, l + g,
// l + 2g, l + 3g of the block (g = groups in the block).  The k-th elements of
// the four lanes' groups are then four consecutive entries, so one gather
// instruction touches neighbouring voxels of a ray (CSR) or neighbouring
// detector pixels of a view (CSC).  Sums over a row are unchanged up to the
// order of the additions.
__host__ __device__ inline int64_t lane_logical(int64_t p, int64_t L) {  // stored -> logical
  const int64_t q = p & ~int64_t(15);
  const int64_t g4 = (L - q) >> 2;
  const int g = g4 < 4 ? (int)g4 : 4;
  return q + (int64_t)g * (p & 3) + ((p & 15) >> 2);
}
__host__ __device__ inline int64_t lane_stored(int64_t p, int64_t L) {  // logical -> stored
  const int64_t q = p & ~int64_t(15);
  const int64_t g4 = (L - q) >> 2;
  const int g = g4 < 4 ? (int)g4 : 4;
  const int r = (int)(p & 15);
  return q + 4 * (r % g) + r / g;
}

struct MatStore {
  int64_t m = 0, N = 0;
  int64_t nnz = 0;       // real entries
  int64_t nnz_pad = 0;   // stored CSR entries
  int64_t nnz_cpad = 0;  // stored CSC entries
  int64_t *row_ptr = nullptr, *col_ptr = nullptr;  // padded offsets [m+1], [N+1]
  int32_t *row_len = nullptr, *col_len = nullptr;  // real counts [m], [N]
  int32_t *col = nullptr, *row = nullptr;
  float *val = nullptr, *cval = nullptr;  // FP32 storage (null for BF16)
  int storage = TVR_STORAGE_FP32;
  __nv_bfloat16 *qval = nullptr, *qcval = nullptr;  // BF16 codes (null for FP32)
  float *rscale = nullptr;                          // BF16 per-row scales [m]
  MfView *mfv = nullptr;                            // matrix-free view constants [V]
  float4 *mfr = nullptr, *mfs = nullptr;            // matrix-free ray table [m] (mfs: parallel)
  float *mfz = nullptr;  // matrix-free, all views separable: A^T r of the last back projection [N]
  float *mfy = nullptr;  // matrix-free, all views separable: row sums of the last forward [4 m]
  int V = 0, Pu = 0, Pv = 0, kind = 0;
};
cudaError_t scan_exclusive_i64(const int64_t *in, int64_t n, int64_t *out, int64_t *tmp,
                               cudaStream_t s);
int64_t scan_tmp_len(int64_t n);
cudaError_t build_matrix(const double *views_dev, int n, int Pu, int Pv, int kind, int64_t m,
                         int64_t N, MatStore &A, cudaStream_t s);
cudaError_t quantize_bf16(MatStore &A, cudaStream_t s);
cudaError_t quantize_u16(MatStore &A, cudaStream_t s);
inline bool coded16(int storage) {
  return storage == TVR_STORAGE_BF16_ROWSCALE || storage == TVR_STORAGE_U16_ROWSCALE;
}
cudaError_t build_matrix_free(const double *views_dev, int n, int V, int Pu, int Pv, int kind,
                              int64_t m, int64_t N, MatStore &A, cudaStream_t s);
cudaError_t interleave_lanes(MatStore &A, cudaStream_t s);
cudaError_t effective_values(const MatStore &A, bool csc, float *out, cudaStream_t s);
void free_matrix(MatStore &A);

int occupancy_grid(const void *kernel, int block, int device);
void kernel_grids(Workspace &ws, const MatDev &A, int device);

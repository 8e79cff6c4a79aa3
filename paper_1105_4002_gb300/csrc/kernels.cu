// Hot-path kernels of the TV-CT gradient methods (sm_103a).
//
//   k_forward   r = A x - b (CSR, row-parallel), 1/2||r||^2.  Trial modes (the
//               second kernel of a solver pass) gather (p, g) pairs, form
//               xbar = P_Q(p - s g) per entry for A xbar and A(xbar - p), fuse
//               the projected step over the voxels (g^T d, ||d||^2, sum_j B_h,
//               TV_tau(xbar), the Huber weights of the next gradient point) and,
//               in UPN, the extrapolation y = x+ + beta (x+ - x) with its residual
//               A y - b for the case of acceptance; GPBB forms two trial points
//               (the second at the step a rejection leads to); the last block
//               runs the test.  Rows and voxels are independent phases: odd
//               warps run the voxels first
//   k_backward  g = A^T r + alpha grad TV_tau(x) (CSC gather, atomic-free); plain
//               modes fuse the TV_tau stencil and its value, the solver mode
//               reads the TV gradient from the Huber weight planes and adds the
//               BB dots (GPBB); it also writes the (p, g) pairs of the next trial
//   k_tv_value  TV_tau(x) alone (phi without a gradient)
//   k_project   P_Q in place; k_gmap gradient-map norm
// Matrix-free storage (template flag MF) replaces the CSR / CSC loops by the
// on-the-fly entries of mf.cuh.
//
// All reductions: double-single per thread / warp / block, deterministic
// block-ordered finish in the last block (tvr_internal.cuh).
#include <utility>

#include "ctrl.cuh"
#include "mf.cuh"
#include "tvr_internal.cuh"

#define FULL 0xffffffffu

namespace {

#ifndef TVR_ROW_LANES
#define TVR_ROW_LANES 4
#endif
#ifndef TVR_COL_LANES
#define TVR_COL_LANES 4
#endif
#ifndef TVR_FWD_MIN_BLOCKS
#define TVR_FWD_MIN_BLOCKS 5
#endif
#ifndef TVR_TRIAL_MIN_BLOCKS
#define TVR_TRIAL_MIN_BLOCKS 4
#endif
#ifndef TVR_BWD_MIN_BLOCKS
#define TVR_BWD_MIN_BLOCKS 5
#endif
#ifndef TVR_MF_MIN_BLOCKS
#define TVR_MF_MIN_BLOCKS 4
#endif
#ifndef TVR_MF_SEP_LANES
#define TVR_MF_SEP_LANES 2
#endif
#ifndef TVR_MF_SEP_K
#define TVR_MF_SEP_K 4
#endif
#ifndef TVR_MF_FSEP_LANES
#define TVR_MF_FSEP_LANES 8
#endif
#ifndef TVR_MF_FSEP_K
#define TVR_MF_FSEP_K 4
#endif
#ifndef TVR_MF_SEP_MIN_BLOCKS
#define TVR_MF_SEP_MIN_BLOCKS 3
#endif
#ifndef TVR_MF_ROW_LANES
#define TVR_MF_ROW_LANES 4
#endif
#ifndef TVR_MF_COL_LANES
#define TVR_MF_COL_LANES 4
#endif
constexpr int kRowLanes = TVR_ROW_LANES;  // lanes per CSR row
constexpr int kColLanes = TVR_COL_LANES;  // lanes per CSC column (>= 4: TV uses lanes 0..3)
constexpr int kMfRowLanes = TVR_MF_ROW_LANES;  // matrix-free: lanes per ray (slabs split among them)
constexpr int kMfColLanes = TVR_MF_COL_LANES;  // matrix-free: lanes per voxel (views split among them)
constexpr int kMfSepLanes = TVR_MF_SEP_LANES;  // separable matrix-free: lanes per voxel stack
constexpr int kMfSepK = TVR_MF_SEP_K;          // separable matrix-free: voxels per stack (along z)
constexpr int kMfFsepLanes = TVR_MF_FSEP_LANES;  // separable matrix-free forward: lanes per ray stack
constexpr int kMfFsepK = TVR_MF_FSEP_K;          // separable matrix-free forward: rays per stack
static_assert(kMfSepLanes >= 1 && kMfSepLanes <= 32 && (kMfSepLanes & (kMfSepLanes - 1)) == 0,
              "lanes");
static_assert(kColLanes >= 4 && kColLanes <= 32 && (kColLanes & (kColLanes - 1)) == 0, "lanes");
static_assert(kRowLanes >= 1 && kRowLanes <= 32 && (kRowLanes & (kRowLanes - 1)) == 0, "lanes");
static_assert(kMfColLanes >= 4 && kMfColLanes <= 32 && (kMfColLanes & (kMfColLanes - 1)) == 0,
              "lanes");
static_assert(kMfRowLanes >= 1 && kMfRowLanes <= 32 && (kMfRowLanes & (kMfRowLanes - 1)) == 0,
              "lanes");

template <int G>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_down_sync(FULL, v, o, G));
  return v;
}

__device__ __forceinline__ float proj(float v) { return v < 0.f ? 0.f : v; }

// Four stored values at a 4-aligned position: float32, or 16-bit codes
// widened to float32 (decode16: bfloat16, or unsigned fixed point with U16).
template <bool BF, bool U16>
__device__ __forceinline__ float4 load4(const float *__restrict__ v32,
                                        const __nv_bfloat16 *__restrict__ v16, int64_t e) {
  if (BF) return decode16<U16>(ld_stream2(v16 + e));
  return ld_stream(v32 + e);
}

__device__ __forceinline__ float xbar_of(float p, float g, float s) {
  return proj(__fsub_rn(p, __fmul_rn(s, g)));
}

// Per-voxel part of the step: d = xbar_j - p_j, the terms of g^T d, ||d||^2,
// the GPBB ||x - P(x - theta g)||^2, the TV Bregman sum and h_tau(D_j xbar)
// (for phi(xbar)), and (W) the Huber weights at xbar.  pk / xk: p and xbar at
// the forward neighbours (in[e]).
template <bool W = true>
__device__ __forceinline__ float step_voxel(float pj, float gj, float xb, const float pk[3],
                                            const float xk[3], const bool in[3], float s2,
                                            bool want_g2, float tau, FF &a0, FF &a1, FF &a2,
                                            FF &a3, FF &ah, float w[3]) {
  const float d = __fsub_rn(xb, pj);
  ff_add_prod(a0, gj, d);
  ff_add_prod(a1, d, d);
  if (want_g2) {
    const float e = __fsub_rn(pj, proj(__fsub_rn(pj, __fmul_rn(s2, gj))));
    ff_add_prod(a3, e, e);
  }
  float z[3], zb[3], dl[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    if (in[e]) {
      z[e] = __fsub_rn(pk[e], pj);
      zb[e] = __fsub_rn(xk[e], xb);
      dl[e] = __fsub_rn(__fsub_rn(xk[e], pk[e]), d);
    } else {
      z[e] = zb[e] = dl[e] = 0.f;
    }
  }
  const float nb = norm3(zb);
  ff_add(a2, huber_bregman_n(z, norm3(z), zb, nb, dl, tau));
  ff_add(ah, huber_h(nb, tau));
  if (W) huber_weights(zb, nb, tau, w);
  return d;
}

// UPN extrapolation (Alg. 3): y = x+ + beta (x+ - x).
__device__ __forceinline__ float y_of(float xn, float xo, float beta) {
  return __fmaf_rn(beta, __fsub_rn(xn, xo), xn);
}

// Per-voxel part: Huber weights of D y and the Bregman term at voxel j.
// xk / yk: x+ and y at the forward neighbours (in[e]).
__device__ __forceinline__ void yform_voxel(float xn, float yj, const float xk[3],
                                            const float yk[3], const bool in[3], float tau,
                                            FF &a2, float w[3]) {
  const float dq0 = __fsub_rn(xn, yj);
  float z[3], zq[3], dl[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    if (in[e]) {
      z[e] = __fsub_rn(yk[e], yj);
      zq[e] = __fsub_rn(xk[e], xn);
      dl[e] = __fsub_rn(__fsub_rn(xk[e], yk[e]), dq0);
    } else {
      z[e] = zq[e] = dl[e] = 0.f;
    }
  }
  const float nz = norm3(z);
  huber_weights(z, nz, tau, w);
  ff_add(a2, huber_bregman(z, nz, zq, dl, tau));
}

// FWD_TRIAL_X: the UPN trial, which also forms the extrapolation for the
// case of acceptance; FWD_TRIAL_2: the GPBB trial with two points (steps
// beta theta and beta^2 theta).  Separate instances, so that the GP / GPBB
// single-point trial keeps its register budget.
enum FwdMode { FWD_RESID = 0, FWD_Y = 1, FWD_INIT = 2, FWD_TRIAL = 3, FWD_TRIAL_X = 4,
               FWD_TRIAL_2 = 5 };
enum BwdMode { BWD_GRAD = 0, BWD_ADJ = 1, BWD_INIT = 2, BWD_SOLVER = 3, BWD_VJP = 4 };

// ---------------------------------------------------------------------------
// Forward projection.  G lanes per row, rows of a warp are consecutive (rays
// of neighbouring detector pixels, which share voxels: x gathers hit in L1).
// ---------------------------------------------------------------------------
template <int G, int MODE, bool BF, bool MF = false, bool U16 = false>
__global__ void __launch_bounds__(TVR_BLOCK, MF ? TVR_MF_MIN_BLOCKS
                                            : (MODE == FWD_TRIAL || MODE == FWD_TRIAL_X ||
                                                       MODE == FWD_TRIAL_2
                                                   ? TVR_TRIAL_MIN_BLOCKS
                                                   : TVR_FWD_MIN_BLOCKS))
    k_forward(MatDev A, const float *__restrict__ xin, const float *__restrict__ b,
              float *__restrict__ rout, RedSlot slot, DevState *st, int prof_slot = -1,
              float *__restrict__ rsout = nullptr) {
  constexpr bool TRIAL = MODE == FWD_TRIAL || MODE == FWD_TRIAL_X || MODE == FWD_TRIAL_2;
  constexpr bool SPEC = MODE == FWD_TRIAL_X;
  constexpr bool TWO = MODE == FWD_TRIAL_2;
  pdl_enter();
  const float *x = xin;
  const float2 *pg = nullptr;  // trial mode: (p_j, g_j) per voxel
  float s = 0.f;               // trial mode: step size
  float sq = 0.f;              // two-point trial: step of the second point
  float *r = rout;
  float *rs = rsout;           // BF16 storage: r times the row scale
  // UPN: the extrapolation for the case of acceptance (see DevState::spec_upn)
  const float *u_old = nullptr;
  float *u2 = nullptr, *ry2 = nullptr, *rys2 = nullptr;
  float bcur = 0.f, bnew = 0.f;
  if (MODE == FWD_INIT) {
    const bool upn = st->solver == SOLVER_UPN;
    b = st->b;
    x = upn ? st->vN[RN_Y] : st->vN[RN_X];
    r = upn ? st->vM[RM_RY] : st->vM[RM_R];
    rs = upn ? st->vM[RM_RYS] : st->vM[RM_RS];
  } else if (TRIAL) {
    if (st->done) return;
    if (prof_slot >= 0 && blockIdx.x == 0 && threadIdx.x == 0) st->prof_flags[prof_slot] = 1;
    b = st->b;
    pg = st->pg;
    s = (float)st->step;
    r = st->vM[RM_RT];
    rs = st->vM[RM_RTS];
    if (TWO) sq = (float)((st->beta * st->beta) * st->theta);  // the step after a rejection
    if (SPEC) {
      __shared__ float sh_bnew;
      u_old = st->vM[RM_U];
      u2 = st->vM[RM_U2];
      ry2 = st->vM[RM_RY2];
      rys2 = BF ? st->vM[RM_RYS2] : nullptr;
      bcur = (float)st->beta;  // beta_{k-1}: u = A(x+ - y) + beta_{k-1} u_{k-1}
      if (threadIdx.x == 0) {
        double tn, mun;
        sh_bnew = (float)upn_next(st, st->Lt, tn, mun);  // beta_k if this trial is accepted
      }
      __syncthreads();
      bnew = sh_bnew;
    }
  }
  constexpr int RPW = 32 / G;
  const int lane = threadIdx.x & (G - 1);
  const int sub = (threadIdx.x & 31) / G;
  const int64_t warp = ((int64_t)blockIdx.x * TVR_BLOCK + threadIdx.x) >> 5;
  const int64_t nwarp = (int64_t)gridDim.x * (TVR_BLOCK / 32);
  FF a0 = ff_zero(), a1 = ff_zero(), au = ff_zero();
  FF c0 = ff_zero(), c1 = ff_zero();  // two-point trial: the second point's residual sums
  auto rows_phase = [&]() {
    for (int64_t base = warp * RPW; base < A.m; base += nwarp * RPW) {
      const int64_t row = base + sub;
      const bool valid = row < A.m;
      int64_t beg = 0, end = 0;
      if (valid && !MF) {
        beg = __ldg(A.row_ptr + row);
        end = __ldg(A.row_ptr + row + 1);
      }
      float sx = 0.f, sd = 0.f, sx2 = 0.f, sd2 = 0.f;
      // plain modes: b_i loaded ahead of the row sum (in the trial modes the
      // extra live register costs more than the latency it hides)
      float bi = 0.f;
      if (!TRIAL && MODE != FWD_Y && valid && lane == 0) bi = __ldg(b + row);
      if (MF && valid && A.mfy) {
        // separable views: the row sums from k_mf_forward_sep, launched just before
        if (lane == 0) {
          sx = __ldg(A.mfy + row);
          if (TRIAL) sd = __ldg(A.mfy + A.m + row);
          if (TWO) {
            sx2 = __ldg(A.mfy + 2 * A.m + row);
            sd2 = __ldg(A.mfy + 3 * A.m + row);
          }
        }
      } else if (MF && valid) {
        // matrix-free: the entries of the row from the ray geometry (mf.cuh)
        const int64_t per = (int64_t)A.Pu * A.Pv;
        const int vi = (int)(row / per);
        const int64_t rem = row - (int64_t)vi * per;
        const int q = (int)(rem / A.Pu), pp = (int)(rem - (int64_t)q * A.Pu);
        MfRay ray;
        mf_pixel_ray(A.mfv[vi], A.kind, A.Pu, A.Pv, pp, q, ray);
        mf_row<G>(ray, A.n, lane, [&](int c, float v) {
          if (TRIAL) {
            const float2 qc = __ldg(pg + c);
            const float bc = xbar_of(qc.x, qc.y, s);
            sx = __fmaf_rn(v, bc, sx);
            sd = __fmaf_rn(v, __fsub_rn(bc, qc.x), sd);
            if (TWO) {
              const float bc2 = xbar_of(qc.x, qc.y, sq);
              sx2 = __fmaf_rn(v, bc2, sx2);
              sd2 = __fmaf_rn(v, __fsub_rn(bc2, qc.x), sd2);
            }
          } else {
            sx = __fmaf_rn(v, __ldg(x + c), sx);
          }
        });
      }
      // Rows are padded to multiples of 4 entries: each lane reads 4 entries
      // with one 16-byte load of indices and one of values, then gathers.  The
      // loads of the lane's next 4 entries are issued before this trip's
      // arithmetic waits on its gathers (a two-stage software pipeline).
      int64_t e0 = beg + 4 * lane;
      int4 cn = make_int4(0, 0, 0, 0);
      float4 vn = make_float4(0.f, 0.f, 0.f, 0.f);
      if (e0 < end) {
        cn = ld_stream(A.col + e0);
        vn = load4<BF, U16>(A.val, A.qval, e0);
      }
      for (; e0 < end; e0 += 4 * G) {
        const int4 c4 = cn;
        const float4 v4 = vn;
        const int64_t e1 = e0 + 4 * G;
        if (TRIAL) {
          // xbar_j = P_Q(p_j - s g_j) and d_j = xbar_j - p_j, as the step phase forms them
          const float2 q0 = __ldg(pg + c4.x), q1 = __ldg(pg + c4.y);
          const float2 q2 = __ldg(pg + c4.z), q3 = __ldg(pg + c4.w);
          if (e1 < end) {
            cn = ld_stream(A.col + e1);
            vn = load4<BF, U16>(A.val, A.qval, e1);
          }
          const float b0 = xbar_of(q0.x, q0.y, s), b1 = xbar_of(q1.x, q1.y, s);
          const float b2 = xbar_of(q2.x, q2.y, s), b3 = xbar_of(q3.x, q3.y, s);
          sx = __fmaf_rn(v4.x, b0, sx);
          sd = __fmaf_rn(v4.x, __fsub_rn(b0, q0.x), sd);
          sx = __fmaf_rn(v4.y, b1, sx);
          sd = __fmaf_rn(v4.y, __fsub_rn(b1, q1.x), sd);
          sx = __fmaf_rn(v4.z, b2, sx);
          sd = __fmaf_rn(v4.z, __fsub_rn(b2, q2.x), sd);
          sx = __fmaf_rn(v4.w, b3, sx);
          sd = __fmaf_rn(v4.w, __fsub_rn(b3, q3.x), sd);
          if (TWO) {  // the second point, from the same gathered pairs
            const float e0_ = xbar_of(q0.x, q0.y, sq), e1_ = xbar_of(q1.x, q1.y, sq);
            const float e2_ = xbar_of(q2.x, q2.y, sq), e3_ = xbar_of(q3.x, q3.y, sq);
            sx2 = __fmaf_rn(v4.x, e0_, sx2);
            sd2 = __fmaf_rn(v4.x, __fsub_rn(e0_, q0.x), sd2);
            sx2 = __fmaf_rn(v4.y, e1_, sx2);
            sd2 = __fmaf_rn(v4.y, __fsub_rn(e1_, q1.x), sd2);
            sx2 = __fmaf_rn(v4.z, e2_, sx2);
            sd2 = __fmaf_rn(v4.z, __fsub_rn(e2_, q2.x), sd2);
            sx2 = __fmaf_rn(v4.w, e3_, sx2);
            sd2 = __fmaf_rn(v4.w, __fsub_rn(e3_, q3.x), sd2);
          }
        } else {
          const float x0 = __ldg(x + c4.x), x1 = __ldg(x + c4.y);
          const float x2 = __ldg(x + c4.z), x3 = __ldg(x + c4.w);
          if (e1 < end) {
            cn = ld_stream(A.col + e1);
            vn = load4<BF, U16>(A.val, A.qval, e1);
          }
          sx = __fmaf_rn(v4.x, x0, sx);
          sx = __fmaf_rn(v4.y, x1, sx);
          sx = __fmaf_rn(v4.z, x2, sx);
          sx = __fmaf_rn(v4.w, x3, sx);
        }
      }
      sx = group_sum<G>(sx);
      if (TRIAL) sd = group_sum<G>(sd);
      if (TWO) {
        sx2 = group_sum<G>(sx2);
        sd2 = group_sum<G>(sd2);
      }
      if (valid && lane == 0) {
        float sc = 1.f;
        if (BF) {
          sc = __ldg(A.rscale + row);
          sx = __fmul_rn(sc, sx);
          sd = __fmul_rn(sc, sd);
          if (TWO) {
            sx2 = __fmul_rn(sc, sx2);
            sd2 = __fmul_rn(sc, sd2);
          }
        }
        if (MODE == FWD_Y) {
          r[row] = sx;
        } else {
          if (TRIAL) bi = __ldg(b + row);
          const float ri = __fsub_rn(sx, bi);
          r[row] = ri;
          if (BF && rs) rs[row] = __fmul_rn(sc, ri);
          ff_add_prod(a0, ri, ri);
          if (TRIAL) {
            ff_add_prod(a1, sd, sd);
            if (TWO) {
              const float ri2 = __fsub_rn(sx2, bi);
              st->vM[RM_RT2][row] = ri2;
              if (BF) st->vM[RM_RTS2][row] = __fmul_rn(sc, ri2);
              ff_add_prod(c0, ri2, ri2);
              ff_add_prod(c1, sd2, sd2);
            }
            if (SPEC) {  // UPN: u and A y - b for the case of acceptance (residual by linearity)
              const float un = __fmaf_rn(bcur, u_old[row], sd);
              u2[row] = un;
              const float ry = __fmaf_rn(bnew, un, ri);
              ry2[row] = ry;
              if (BF && rys2) rys2[row] = __fmul_rn(sc, ry);
              ff_add_prod(au, un, un);
            }
          }
        }
      }
    }
  };
  // Step phase: xbar = P_Q(p - s g) (eq. gradientmethod; Alg. 1, Alg. 2) over
  // the voxels, with the reductions of the acceptance tests.  xbar at the
  // forward neighbours is recomputed with the same expression, so the TV
  // Bregman sum and the Huber weights (written for GP / GPBB, whose next
  // gradient is taken at the accepted xbar) see exactly the stored values.
  // UPN: also y = x+ + beta_k (x+ - x) for the case of acceptance, the
  // Huber weights of D y, ||x+ - x||^2 and sum_j B_h(D_j x+; D_j y) (Alg. 3,
  // eq. mu_k_estimate), recomputing y at the forward neighbours.
  FF s0 = ff_zero(), s1 = ff_zero(), s2 = ff_zero(), s3 = ff_zero(), sb = ff_zero();
  FF sh = ff_zero();  // TV_tau(xbar)
  // two-point trial: the second point's g^T d, ||d||^2, sum B_h, TV_tau
  FF d0 = ff_zero(), d1 = ff_zero(), d2 = ff_zero(), dh = ff_zero();
  auto voxel_phase = [&]() {
    if constexpr (TRIAL) {
      {
        const bool upn = st->solver == SOLVER_UPN;
        constexpr bool spec = SPEC;
        const bool want_g2 = st->solver == SOLVER_GPBB && st->trial == 0;
        const float sg2 = (float)st->step2;
        const float tau = (float)st->tau;
        float *__restrict__ t = st->vN[RN_T];
        float *__restrict__ wt = (!upn || spec) ? st->wt : nullptr;
        const float *__restrict__ xo = st->vN[RN_X];
        float *__restrict__ y2 = st->vN[RN_Y2];
        const int n = A.n;
        const int64_t nn = (int64_t)n * n, N = A.N;
        const int64_t stride = (int64_t)gridDim.x * TVR_BLOCK;
        for (int64_t j = (int64_t)blockIdx.x * TVR_BLOCK + threadIdx.x; j < N; j += stride) {
          const float2 q = pg[j];
          const float xb = xbar_of(q.x, q.y, s);
          int ix, iy, iz;
          voxel_of(A, j, ix, iy, iz);
          const int64_t off[3] = {1, n, nn};
          const bool in[3] = {ix + 1 < n, iy + 1 < n, iz + 1 < n};
          float pk[3], gk[3], xk[3];
    #pragma unroll
          for (int e = 0; e < 3; ++e) {
            const float2 qk = in[e] ? pg[j + off[e]] : make_float2(0.f, 0.f);
            pk[e] = qk.x;
            gk[e] = qk.y;
            xk[e] = in[e] ? xbar_of(qk.x, qk.y, s) : 0.f;
          }
          float w[3];
          step_voxel<!SPEC>(q.x, q.y, xb, pk, xk, in, sg2, want_g2, tau, s0, s1, s2, s3, sh, w);
          t[j] = xb;
          if (TWO) {  // the second point, as a trial at step sq would form it
            const float xq = xbar_of(q.x, q.y, sq);
            float xkq[3], wq[3];
    #pragma unroll
            for (int e = 0; e < 3; ++e) xkq[e] = in[e] ? xbar_of(pk[e], gk[e], sq) : 0.f;
            FF unused = ff_zero();
            step_voxel(q.x, q.y, xq, pk, xkq, in, sg2, false, tau, d0, d1, d2, unused, dh, wq);
            st->vN[RN_T2][j] = xq;
            float *__restrict__ wq_ = st->wt2;
            wq_[j] = wq[0];
            wq_[N + j] = wq[1];
            wq_[2 * N + j] = wq[2];
            wq_[3 * N + j] = __fadd_rn(__fadd_rn(wq[0], wq[1]), wq[2]);
          }
          if (spec) {
            const float xoj = xo[j];
            const float dx = __fsub_rn(xb, xoj);
            const float yj = __fmaf_rn(bnew, dx, xb);
            ff_add_prod(s3, dx, dx);
            float yk[3];
    #pragma unroll
            for (int e = 0; e < 3; ++e) yk[e] = in[e] ? y_of(xk[e], xo[j + off[e]], bnew) : 0.f;
            yform_voxel(xb, yj, xk, yk, in, tau, sb, w);
            y2[j] = yj;
          }
          if (wt) {  // Huber weights at the next gradient point: xbar (GP, GPBB) or y (UPN)
            wt[j] = w[0];
            wt[N + j] = w[1];
            wt[2 * N + j] = w[2];
            wt[3 * N + j] = __fadd_rn(__fadd_rn(w[0], w[1]), w[2]);
          }
        }
      }
    }
  };
  // The two phases of a trial are independent (the rows gather (p, g) and
  // write the residuals; the voxels read (p, g) and x and write xbar, y and
  // the planes).  Odd warps run the voxels first, so that every SM mixes
  // latency-bound voxel work with the row streams instead of ending the
  // kernel on the voxel phase alone.
  const bool voxels_first = TRIAL && (warp & 1);
#pragma unroll 1
  for (int ph = 0; ph < 2; ++ph) {
    if ((ph == 0) != voxels_first)
      rows_phase();
    else
      voxel_phase();
  }
  if (MODE == FWD_Y) return;
  if (!TRIAL) {
    FF acc[1] = {a0};
    double tot[1];
    if (grid_reduce<1>(acc, slot, tot) && threadIdx.x == 0 && MODE == FWD_INIT)
      st->r_init[0] = tot[0];
    return;
  }
  if constexpr (TWO) {
    // {first point: ||r||^2, ||A d||^2, g^T d, ||d||^2, sum B_h, ||x - P(x - theta g)||^2,
    //  TV_tau; second point: ||r||^2, ||A d||^2, g^T d, ||d||^2, sum B_h, TV_tau}
    FF acc[13] = {a0, a1, s0, s1, s2, s3, sh, c0, c1, d0, d1, d2, dh};
    double tot[13];
    if (grid_reduce<13>(acc, slot, tot) && threadIdx.x == 0) {
      st->r_fwd[0] = tot[0];
      st->r_fwd[1] = tot[1];
#pragma unroll
      for (int k = 0; k < 4; ++k) st->r_step[k] = tot[2 + k];
      st->r_step[4] = tot[6];
      st->r_fwd2[0] = tot[7];
      st->r_fwd2[1] = tot[8];
#pragma unroll
      for (int k = 0; k < 4; ++k) st->r_step2[k] = tot[9 + k];
      ctrl_trial2(st, tot);
    }
    return;
  }
  // slot 5: GPBB ||x - P(x - theta g)||^2, or UPN ||x+ - x||^2; slot 8: TV_tau(xbar)
  FF acc[9] = {a0, a1, s0, s1, s2, s3, au, sb, sh};
  double tot[9];
  if (grid_reduce<9>(acc, slot, tot) && threadIdx.x == 0) {
    st->r_fwd[0] = tot[0];
    st->r_fwd[1] = tot[1];
#pragma unroll
    for (int k = 0; k < 4; ++k) st->r_step[k] = tot[2 + k];
    st->r_step[4] = tot[8];
    if (SPEC) {
      st->r_spec[0] = tot[5];
      st->r_spec[1] = tot[6];
      st->r_spec[2] = tot[7];
    }
    ctrl_trial(st, tot);
  }
}

// ---------------------------------------------------------------------------
// Back projection fused with the TV_tau stencil.  G lanes per column (voxel);
// lanes 0..3 of a group evaluate the Huber weights of voxels j, j-ex, j-ey,
// j-ez, whose sum gives [grad TV_tau(x)]_j = -sum_e w_j,e + sum_e w_{j-e},e.
// ---------------------------------------------------------------------------
template <int G, int MODE, bool BF, bool MF = false, bool U16 = false>
__global__ void __launch_bounds__(TVR_BLOCK, MF ? TVR_MF_MIN_BLOCKS : TVR_BWD_MIN_BLOCKS)
    k_backward(MatDev A, const float *__restrict__ rin, const float *__restrict__ xin, float alpha,
               float tau, double alpha_d, float *__restrict__ gout, RedSlot slot,
               const double *__restrict__ data_in, double *phi_dev, DevState *st,
               int prof_slot = -1, const double *__restrict__ scale_p = nullptr,
               float *__restrict__ gb = nullptr) {
  pdl_enter();
  const float *r = rin;
  const float *x = xin;
  float *g = gout;
  const float *xo = nullptr;  // GPBB: x^(k-1)
  const float *go = nullptr;  // GPBB: g^(k-1)
  int kind = SOLVER_NONE;
  if (MODE == BWD_INIT || MODE == BWD_SOLVER) {
    if (MODE == BWD_SOLVER && (st->done || !st->need_grad)) return;
    if (prof_slot >= 0 && blockIdx.x == 0 && threadIdx.x == 0)
      st->prof_flags[TVR_PROF_PAIRS + prof_slot] = 1;
    kind = st->solver;
    alpha = (float)st->alpha;
    tau = (float)st->tau;
    if (kind == SOLVER_UPN) {
      x = st->vN[RN_Y];
      r = BF ? st->vM[RM_RYS] : st->vM[RM_RY];
      g = st->vN[RN_G];
    } else {
      x = st->vN[RN_X];
      r = BF ? st->vM[RM_RS] : st->vM[RM_R];
      g = st->vN[RN_G];
      if (MODE == BWD_SOLVER && kind == SOLVER_GPBB) {
        g = st->vN[RN_GN];
        xo = st->vN[RN_T];
        go = st->vN[RN_G];
      }
    }
  }
  const int n = A.n;
  const int64_t nn = (int64_t)n * n;
  constexpr int RPW = 32 / G;
  const int lane = threadIdx.x & (G - 1);
  const int sub = (threadIdx.x & 31) / G;
  const int64_t warp = ((int64_t)blockIdx.x * TVR_BLOCK + threadIdx.x) >> 5;
  const int64_t nwarp = (int64_t)gridDim.x * (TVR_BLOCK / 32);
  FF a0 = ff_zero(), a1 = ff_zero(), a2 = ff_zero();
  for (int64_t base = warp * RPW; base < A.N; base += nwarp * RPW) {
    const int64_t j = base + sub;
    const bool valid = j < A.N;
    int64_t beg = 0, end = 0;
    if (valid && !MF) {
      beg = __ldg(A.col_ptr + j);
      end = __ldg(A.col_ptr + j + 1);
    }
    int ix = 0, iy = 0, iz = 0;
    if (MODE != BWD_ADJ || MF) voxel_of(A, valid ? j : 0, ix, iy, iz);
    // solver mode: this lane's term of [grad TV_tau]_j from the Huber weight
    // planes (lane 0: -(w_0 + w_1 + w_2) at j; lanes 1..3: w_e at j - e),
    // loaded ahead of the projection loop
    float c = 0.f;
    float hh = 0.f;  // lane 0: h_tau(D_j x), for TV_tau(x)
    if (MODE != BWD_SOLVER && MODE != BWD_ADJ && valid && lane < 4) {
      // plain modes: the lane's Huber weights from x, evaluated ahead of the
      // projection loop (lanes 1..3 at the backward neighbours)
      Huber hw;
      huber_at(x, ix - (lane == 1), iy - (lane == 2), iz - (lane == 3), n, tau, hw);
      c = lane == 0 ? -__fadd_rn(__fadd_rn(hw.w[0], hw.w[1]), hw.w[2])
                    : (lane == 1 ? hw.w[0] : (lane == 2 ? hw.w[1] : hw.w[2]));
      hh = hw.h;
    }
    if (MODE == BWD_SOLVER && valid && lane < 4) {
      const float *__restrict__ W = st->w;
      if (lane == 0)
        c = -__ldg(W + 3 * A.N + j);
      else if (lane == 1)
        c = ix > 0 ? __ldg(W + j - 1) : 0.f;
      else if (lane == 2)
        c = iy > 0 ? __ldg(W + A.N + j - n) : 0.f;
      else
        c = iz > 0 ? __ldg(W + 2 * A.N + j - nn) : 0.f;
    }
    float s = 0.f;
    if (MF && valid) {
      if (A.mfz) {
        // separable views: (A^T r)_j from k_mf_adjoint_sep, launched just before
        if (lane == 0) s = __ldg(A.mfz + j);
      } else {
        // the entries of the column from the view geometry (mf.cuh)
        mf_column<G>(A.mfv, A.mfr, A.mfs, A.V, A.kind, A.Pu, A.Pv, A.n, ix, iy, iz, lane,
                     [&](int64_t i, float v) { s = __fmaf_rn(v, __ldg(r + i), s); });
      }
    }
    // two-stage software pipeline over the lane's 4-entry groups, as in the
    // forward projection
    int64_t e0 = beg + 4 * lane;
    int4 in4 = make_int4(0, 0, 0, 0);
    float4 vn = make_float4(0.f, 0.f, 0.f, 0.f);
    if (e0 < end) {
      in4 = ld_stream(A.row + e0);
      vn = load4<BF, U16>(A.cval, A.qcval, e0);
    }
    for (; e0 < end; e0 += 4 * G) {
      const int4 i4 = in4;
      const float4 v4 = vn;
      float r0 = __ldg(r + i4.x), r1 = __ldg(r + i4.y);
      float r2 = __ldg(r + i4.z), r3 = __ldg(r + i4.w);
      const int64_t e1 = e0 + 4 * G;
      if (e1 < end) {
        in4 = ld_stream(A.row + e1);
        vn = load4<BF, U16>(A.cval, A.qcval, e1);
      }
      if (BF && (MODE == BWD_ADJ || MODE == BWD_VJP)) {  // caller's r: apply the row scales
        r0 = __fmul_rn(r0, __ldg(A.rscale + i4.x));
        r1 = __fmul_rn(r1, __ldg(A.rscale + i4.y));
        r2 = __fmul_rn(r2, __ldg(A.rscale + i4.z));
        r3 = __fmul_rn(r3, __ldg(A.rscale + i4.w));
      }
      s = __fmaf_rn(v4.x, r0, s);
      s = __fmaf_rn(v4.y, r1, s);
      s = __fmaf_rn(v4.z, r2, s);
      s = __fmaf_rn(v4.w, r3, s);
    }
    s = group_sum<G>(s);
    if (MODE == BWD_ADJ) {
      if (valid && lane == 0) g[j] = s;
      continue;
    }
    c = __fadd_rn(c, __shfl_down_sync(FULL, c, 2, G));
    c = __fadd_rn(c, __shfl_down_sync(FULL, c, 1, G));
    if (MODE == BWD_VJP) {
      if (valid && lane == 0) g[j] = __fmul_rn((float)*scale_p, __fmaf_rn(alpha, c, s));
      continue;
    }
    if (valid && lane == 0) {
      const float gj = __fmaf_rn(alpha, c, s);
      g[j] = gj;
      if (MODE == BWD_INIT || MODE == BWD_SOLVER) st->pg[j] = make_float2(x[j], gj);
      if (MODE != BWD_SOLVER) ff_add(a0, hh);
      if (MODE == BWD_SOLVER && kind == SOLVER_GPBB) {
        const float sj = __fsub_rn(x[j], xo[j]);
        ff_add_prod(a1, sj, __fsub_rn(gj, go[j]));
        ff_add_prod(a2, sj, sj);
      }
    }
  }
  if (MODE == BWD_ADJ) return;
  if (MODE == BWD_VJP) {
    if (gb) {
      const float sc = (float)*scale_p;
      const int64_t stride = (int64_t)gridDim.x * TVR_BLOCK;
      for (int64_t i = (int64_t)blockIdx.x * TVR_BLOCK + threadIdx.x; i < A.m; i += stride)
        gb[i] = -__fmul_rn(sc, r[i]);
    }
    return;
  }
  FF acc[3] = {a0, a1, a2};
  double tot[3];
  if (grid_reduce<3>(acc, slot, tot) && threadIdx.x == 0) {
    if (MODE == BWD_GRAD) {
      const double data = 0.5 * data_in[0];
      if (phi_dev) {
        phi_dev[0] = data + alpha_d * tot[0];
        phi_dev[1] = data;
        phi_dev[2] = tot[0];
      }
    } else if (MODE == BWD_INIT) {
      ctrl_init(st, tot);
    } else {
      if (kind == SOLVER_UPN) tot[1] = st->r_yf[2];  // TV Bregman sum from the extrapolation
      st->r_bwd[0] = tot[0];
      st->r_bwd[1] = tot[1];
      st->r_bwd[2] = tot[2];
      ctrl_after_grad(st, tot);
    }
  }
}

// TV_tau(x) alone; finishes phi from the forward kernel's 1/2||r||^2.
__global__ void __launch_bounds__(TVR_BLOCK)
    k_tv_value(MatDev A, const float *__restrict__ x, float tau, double alpha_d, RedSlot slot,
               const double *__restrict__ data_in, double *phi_dev) {
  const int n = A.n;
  FF a0 = ff_zero();
  const int64_t stride = (int64_t)gridDim.x * TVR_BLOCK;
  for (int64_t j = (int64_t)blockIdx.x * TVR_BLOCK + threadIdx.x; j < A.N; j += stride) {
    int ix, iy, iz;
    voxel_of(A, j, ix, iy, iz);
    float z[3];
    diff3(x, ix, iy, iz, n, z);
    ff_add(a0, huber_h(norm3(z), tau));
  }
  FF acc[1] = {a0};
  double tot[1];
  if (grid_reduce<1>(acc, slot, tot) && threadIdx.x == 0) {
    const double data = 0.5 * data_in[0];
    if (phi_dev) {
      phi_dev[0] = data + alpha_d * tot[0];
      phi_dev[1] = data;
      phi_dev[2] = tot[0];
    }
  }
}

__global__ void __launch_bounds__(TVR_BLOCK) k_project(float *__restrict__ x, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * TVR_BLOCK;
  for (int64_t i = (int64_t)blockIdx.x * TVR_BLOCK + threadIdx.x; i < n; i += stride)
    x[i] = proj(x[i]);
}

// ||G_nu(x)|| = nu ||x - P_Q(x - g / nu)||.
__global__ void __launch_bounds__(TVR_BLOCK)
    k_gmap(const float *__restrict__ x, const float *__restrict__ g, int64_t n, float inv_nu,
           double nu, RedSlot slot) {
  FF a0 = ff_zero();
  const int64_t stride = (int64_t)gridDim.x * TVR_BLOCK;
  for (int64_t i = (int64_t)blockIdx.x * TVR_BLOCK + threadIdx.x; i < n; i += stride) {
    const float e = __fsub_rn(x[i], proj(__fsub_rn(x[i], __fmul_rn(g[i], inv_nu))));
    ff_add_prod(a0, e, e);
  }
  FF acc[1] = {a0};
  double tot[1];
  if (grid_reduce<1>(acc, slot, tot) && threadIdx.x == 0) slot.out[1] = nu * sqrt(tot[0]);
}

// Matrix-free back projection z = A^T r for scans whose views are all
// separable (MfView::sep): G lanes per stack of K voxels along z, the views
// split among the lanes (mf_column_sep), summed over the lanes at the end.
// The back projection launched next reads z in place of its own pixel
// enumeration.  With st (solver modes) r is the residual that back projection
// takes from the device state, and with skip_idle the kernel returns at once
// where that back projection returns at once.
template <int G, int K>
__global__ void __launch_bounds__(TVR_BLOCK, TVR_MF_SEP_MIN_BLOCKS)
    k_mf_adjoint_sep(MatDev A, const float *__restrict__ rin, DevState *st, int skip_idle,
                     float *__restrict__ z) {
  pdl_enter();
  const float *r = rin;
  if (st) {
    if (skip_idle && (st->done || !st->need_grad)) return;
    r = st->solver == SOLVER_UPN ? st->vM[RM_RY] : st->vM[RM_R];
  }
  const int n = A.n;
  const int64_t stacks = (int64_t)n * n * ((n + K - 1) / K);
  constexpr int RPW = 32 / G;
  const int lane = threadIdx.x & (G - 1);
  const int sub = (threadIdx.x & 31) / G;
  const int64_t warp = ((int64_t)blockIdx.x * TVR_BLOCK + threadIdx.x) >> 5;
  const int64_t nwarp = (int64_t)gridDim.x * (TVR_BLOCK / 32);
  for (int64_t base = warp * RPW; base < stacks; base += nwarp * RPW) {
    const int64_t gi = base + sub;
    const bool valid = gi < stacks;
    // stack gi = ix + n (iy + n c): x fastest, so a warp's writes of one k
    // are consecutive voxels (gi < n^3 < 2^31: exact for fast_div)
    const uint32_t u = valid ? (uint32_t)gi : 0u;
    const uint32_t c = fast_div(u, A.div_nn);
    const uint32_t rem = u - c * A.div_nn.d;
    const uint32_t iy = fast_div(rem, A.div_n);
    const uint32_t ix = rem - iy * A.div_n.d;
    const int iz0 = (int)c * K;
    float acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.f;
    if (valid)
      for (int vi = lane; vi < A.V; vi += G)
        mf_column_sep<K>(A.mfv[vi], A.mfr, vi, A.Pu, A.Pv, n, (int)ix, (int)iy, iz0, r, acc);
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = group_sum<G>(acc[k]);
    if (valid && lane == 0) {
#pragma unroll
      for (int k = 0; k < K; ++k)
        if (iz0 + k < n) z[(int64_t)ix + (int64_t)n * ((int64_t)iy + (int64_t)n * (iz0 + k))] = acc[k];
    }
  }
}

// Matrix-free forward projection for scans whose views are all separable
// (MfView::sep): G lanes per stack of K rays (rows q of one detector column),
// the x-y slabs of their shared path split among the lanes (mf_row_sep),
// summed over the lanes at the end.  The forward projection launched next
// reads the row sums from y in place of its own walk along each ray:
//   S = 1: y = A x (x = xin, or with st the point FWD_INIT projects);
//   S = 2: the trial's A xbar and A d from the pairs (p_j, g_j) and step s;
//   S = 4: those two and the second trial point's (two-point GPBB pass).
// y holds S blocks of m values.  The trial modes return at once where the
// trial kernel does (the solve has stopped).
template <int G, int K, int S>
__global__ void __launch_bounds__(TVR_BLOCK, S == 4 ? 3 : TVR_MF_MIN_BLOCKS)  // 4 sums: no spills
    k_mf_forward_sep(MatDev A, const float *__restrict__ xin, DevState *st,
                     float *__restrict__ y) {
  static_assert(S == 1 || S == 2 || S == 4, "sums");
  pdl_enter();
  const float *x = xin;
  const float2 *pg = nullptr;
  float s = 0.f, sq = 0.f;
  if (S == 1 && st) x = st->solver == SOLVER_UPN ? st->vN[RN_Y] : st->vN[RN_X];
  if (S > 1) {
    if (st->done) return;
    pg = st->pg;
    s = (float)st->step;  // the trial kernel's steps, formed the same way
    if (S == 4) sq = (float)((st->beta * st->beta) * st->theta);
  }
  const int64_t per = (int64_t)A.Pu * A.Pv;
  const int64_t nch = (A.Pv + K - 1) / K;
  const int64_t stacks = (int64_t)A.V * nch * A.Pu;
  constexpr int RPW = 32 / G;
  const int lane = threadIdx.x & (G - 1);
  const int sub = (threadIdx.x & 31) / G;
  const int64_t warp = ((int64_t)blockIdx.x * TVR_BLOCK + threadIdx.x) >> 5;
  const int64_t nwarp = (int64_t)gridDim.x * (TVR_BLOCK / 32);
  for (int64_t base = warp * RPW; base < stacks; base += nwarp * RPW) {
    const int64_t gi = base + sub;
    const bool valid = gi < stacks;
    // stack gi = p + Pu (c + nch vi): p fastest, so a warp's rays are
    // neighbouring columns
    const int64_t g = valid ? gi : 0;
    const int p = (int)(g % A.Pu);
    const int64_t rest = g / A.Pu;
    const int c = (int)(rest % nch), vi = (int)(rest / nch);
    float acc[K][S];
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int t = 0; t < S; ++t) acc[k][t] = 0.f;
    if (valid) {
      const MfView &v = A.mfv[vi];
      MfRay r0;
      float izv[K], dzv[K], dnv[K];
      bool ok[K];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int q = c * K + k;
        ok[k] = q < A.Pv;
        MfRay rk;
        mf_pixel_ray(v, TVR_CONE, A.Pu, A.Pv, p, ok[k] ? q : 0, rk);
        if (k == 0) r0 = rk;
        izv[k] = rk.inv[2];
        dzv[k] = rk.d[2];
        dnv[k] = rk.dn;
      }
      mf_row_sep<G, K>(r0, izv, dzv, dnv, ok, A.n, lane, [&](int k, int j, float a) {
        if (S == 1) {
          acc[k][0] = __fmaf_rn(a, __ldg(x + j), acc[k][0]);
        } else {
          const float2 qc = __ldg(pg + j);
          const float bc = xbar_of(qc.x, qc.y, s);
          acc[k][0] = __fmaf_rn(a, bc, acc[k][0]);
          acc[k][1] = __fmaf_rn(a, __fsub_rn(bc, qc.x), acc[k][1]);
          if (S == 4) {
            const float bc2 = xbar_of(qc.x, qc.y, sq);
            acc[k][2] = __fmaf_rn(a, bc2, acc[k][2]);
            acc[k][3] = __fmaf_rn(a, __fsub_rn(bc2, qc.x), acc[k][3]);
          }
        }
      });
    }
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int t = 0; t < S; ++t) acc[k][t] = group_sum<G>(acc[k][t]);
    if (valid && lane == 0) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int q = c * K + k;
        if (q >= A.Pv) continue;
        const int64_t row = (int64_t)vi * per + (int64_t)q * A.Pu + p;
#pragma unroll
        for (int t = 0; t < S; ++t) y[(int64_t)t * A.m + row] = acc[k][t];
      }
    }
  }
}

int elem_grid(int64_t n, int cap) {
  int64_t b = (n + TVR_BLOCK - 1) / TVR_BLOCK;
  if (b < 1) b = 1;
  return (int)(b < cap ? b : cap);
}

}  // namespace

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
int occupancy_grid(const void *kernel, int block, int device) {
  int sms = 0, per = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, block, 0);
  if (per < 1) per = 1;
  int g = sms * per;
  return g < TVR_MAX_GRID ? g : TVR_MAX_GRID;
}

// Launch with programmatic stream serialization (the kernel calls pdl_enter
// first), so that its blocks are scheduled while the predecessor drains.
template <typename... P, typename... A>
void launch_pdl(void (*kernel)(P...), int grid, cudaStream_t s, A &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(TVR_BLOCK);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

// Kernel instance for the system's storage (float32 or bfloat16 values).
template <int MODE>
auto fwd_kernel(const MatDev &A) {
  return A.mf ? k_forward<kMfRowLanes, MODE, false, true>
              : (A.bf16 ? (A.u16 ? k_forward<kRowLanes, MODE, true, false, true>
                                 : k_forward<kRowLanes, MODE, true>)
                        : k_forward<kRowLanes, MODE, false>);
}
template <int MODE>
auto bwd_kernel(const MatDev &A) {
  return A.mf ? k_backward<kMfColLanes, MODE, false, true>
              : (A.bf16 ? (A.u16 ? k_backward<kColLanes, MODE, true, false, true>
                                 : k_backward<kColLanes, MODE, true>)
                        : k_backward<kColLanes, MODE, false>);
}

// Grids of the hot kernels, each from the occupancy of the instance that runs
// for this system's storage (FP32, BF16 or matrix-free values differ in
// registers): at most one wave of resident blocks, and no more blocks than the
// work needs (rows or columns in groups of TVR_BLOCK / lanes, voxels in groups
// of TVR_BLOCK), so that the kernels of small systems leave room for others
// running concurrently on other streams.
void kernel_grids(Workspace &ws, const MatDev &A, int device) {
  auto cap = [](int grid, int64_t need) {
    need = need < 1 ? 1 : need;
    return (int)(need < grid ? need : grid);
  };
  auto occ = [&](const void *k) { return occupancy_grid(k, TVR_BLOCK, device); };
  const int rl = A.mf ? kMfRowLanes : kRowLanes, cl = A.mf ? kMfColLanes : kColLanes;
  const int64_t rows = (A.m + TVR_BLOCK / rl - 1) / (TVR_BLOCK / rl);
  const int64_t cols = (A.N + TVR_BLOCK / cl - 1) / (TVR_BLOCK / cl);
  const int64_t vox = (A.N + TVR_BLOCK - 1) / TVR_BLOCK;
  const int64_t fwd_need = rows > vox ? rows : vox;
  ws.grid_fwd = cap(occ((const void *)fwd_kernel<FWD_RESID>(A)), rows);
  ws.grid_trial = cap(occ((const void *)fwd_kernel<FWD_TRIAL>(A)), fwd_need);
  ws.grid_trial_x = cap(occ((const void *)fwd_kernel<FWD_TRIAL_X>(A)), fwd_need);
  ws.grid_trial_2 = cap(occ((const void *)fwd_kernel<FWD_TRIAL_2>(A)), fwd_need);
  ws.grid_bwd = cap(occ((const void *)bwd_kernel<BWD_SOLVER>(A)), cols);
  ws.grid_elem = cap(occ((const void *)k_tv_value), vox);
  const int64_t stacks = (int64_t)A.n * A.n * ((A.n + kMfSepK - 1) / kMfSepK);
  ws.grid_mfsep = A.mfz ? cap(occ((const void *)k_mf_adjoint_sep<kMfSepLanes, kMfSepK>),
                              (stacks + TVR_BLOCK / kMfSepLanes - 1) / (TVR_BLOCK / kMfSepLanes))
                        : 0;
  const int64_t rstacks = (int64_t)A.V * ((A.Pv + kMfFsepK - 1) / kMfFsepK) * A.Pu;
  const int64_t rneed = (rstacks + TVR_BLOCK / kMfFsepLanes - 1) / (TVR_BLOCK / kMfFsepLanes);
  ws.grid_mfsep_fwd[0] = A.mfy ? cap(occ((const void *)k_mf_forward_sep<kMfFsepLanes, kMfFsepK, 1>), rneed) : 0;
  ws.grid_mfsep_fwd[1] = A.mfy ? cap(occ((const void *)k_mf_forward_sep<kMfFsepLanes, kMfFsepK, 2>), rneed) : 0;
  ws.grid_mfsep_fwd[2] = A.mfy ? cap(occ((const void *)k_mf_forward_sep<kMfFsepLanes, kMfFsepK, 4>), rneed) : 0;
}

// Separable matrix-free scans: the row sums (S of them) into A.mfy ahead of
// the forward projection that reads them (no launch for other storage).
template <int S>
static void launch_mf_fsep(const MatDev &A, const float *x, DevState *st, const Workspace &ws,
                           cudaStream_t s) {
  if (!A.mfy) return;
  launch_pdl(k_mf_forward_sep<kMfFsepLanes, kMfFsepK, S>, ws.grid_mfsep_fwd[S == 1 ? 0 : (S == 2 ? 1 : 2)],
             s, A, x, st, A.mfy);
}

// Separable matrix-free scans: A^T r into A.mfz ahead of the back projection
// that reads it (no launch for other storage).
static void launch_mf_sep(const MatDev &A, const float *r, DevState *st, int skip_idle,
                          const Workspace &ws, cudaStream_t s) {
  if (!A.mfz) return;
  launch_pdl(k_mf_adjoint_sep<kMfSepLanes, kMfSepK>, ws.grid_mfsep, s, A, r, st, skip_idle, A.mfz);
}

void launch_forward(const MatDev &A, const float *x, const float *b, float *r, const Workspace &ws,
                    cudaStream_t s, float *rs) {
  launch_mf_fsep<1>(A, x, nullptr, ws, s);
  launch_pdl(fwd_kernel<FWD_RESID>(A), ws.grid_fwd, s, A, x, b, r, ws.fwd, nullptr, -1, rs);
}

void launch_forward_plain(const MatDev &A, const float *x, float *y, const Workspace &ws,
                          cudaStream_t s) {
  launch_mf_fsep<1>(A, x, nullptr, ws, s);
  fwd_kernel<FWD_Y>(A)<<<ws.grid_fwd, TVR_BLOCK, 0, s>>>(A, x, nullptr, y, ws.fwd, nullptr, -1,
                                                          nullptr);
}

void launch_backward(const MatDev &A, const float *r, const float *x, float alpha, float tau,
                     float *g, const Workspace &ws, double *phi_dev, cudaStream_t s) {
  launch_mf_sep(A, r, nullptr, 0, ws, s);
  launch_pdl(bwd_kernel<BWD_GRAD>(A), ws.grid_bwd, s, A, r, x, alpha, tau, (double)alpha, g, ws.bwd,
             ws.fwd.out, phi_dev, nullptr, -1, nullptr, nullptr);
}

void launch_adjoint_plain(const MatDev &A, const float *r, float *z, const Workspace &ws,
                          cudaStream_t s) {
  launch_mf_sep(A, r, nullptr, 0, ws, s);
  bwd_kernel<BWD_ADJ>(A)<<<ws.grid_bwd, TVR_BLOCK, 0, s>>>(
      A, r, nullptr, 0.f, 1.f, 0.0, z, ws.bwd, nullptr, nullptr, nullptr, -1, nullptr, nullptr);
}

void launch_vjp(const MatDev &A, const float *r, const float *x, float alpha, float tau,
                const double *scale, float *gx, float *gb, const Workspace &ws, cudaStream_t s) {
  launch_mf_sep(A, r, nullptr, 0, ws, s);
  launch_pdl(bwd_kernel<BWD_VJP>(A), ws.grid_bwd, s, A, r, x, alpha, tau, (double)alpha, gx, ws.bwd,
             nullptr, nullptr, nullptr, -1, scale, gb);
}

void launch_tv_value(const MatDev &A, const float *x, float alpha, float tau, const Workspace &ws,
                     double *phi_dev, cudaStream_t s) {
  k_tv_value<<<elem_grid(A.N, ws.grid_elem), TVR_BLOCK, 0, s>>>(A, x, tau, (double)alpha, ws.tv,
                                                                 ws.fwd.out, phi_dev);
}

void launch_project(float *x, int64_t n, cudaStream_t s) {
  k_project<<<elem_grid(n, 4 * 152 * 8), TVR_BLOCK, 0, s>>>(x, n);
}

void launch_gmap_norm(const float *x, const float *g, int64_t n, double nu, const Workspace &ws,
                      cudaStream_t s) {
  k_gmap<<<elem_grid(n, ws.grid_elem), TVR_BLOCK, 0, s>>>(x, g, n, (float)(1.0 / nu), nu, ws.gmap);
}

void launch_solver_init(const MatDev &A, DevState *st, const Workspace &ws, cudaStream_t s) {
  launch_mf_fsep<1>(A, nullptr, st, ws, s);
  launch_pdl(fwd_kernel<FWD_INIT>(A), ws.grid_fwd, s, A, nullptr, nullptr, nullptr, ws.fwd, st, -1,
             nullptr);
  launch_mf_sep(A, nullptr, st, 0, ws, s);
  launch_pdl(bwd_kernel<BWD_INIT>(A), ws.grid_bwd, s, A, nullptr, nullptr, 0.f, 1.f, 0.0, nullptr,
             ws.bwd, nullptr, nullptr, st, -1, nullptr, nullptr);
}

// One pass: gradient at the new point (skipped after a rejected trial) ->
// trial kernel (forward projection with the projected step fused, UPN's
// extrapolation for the case of acceptance, the acceptance test).
void launch_solver_pass(const MatDev &A, DevState *st, int solver, const Workspace &ws,
                        cudaStream_t s, const PassTiming *tm) {
  auto mark = [&](int kind, int which) {
    if (!tm || tm->slot[kind] < 0) return;
    if (tm->graph_nodes)
      cudaEventRecordWithFlags(tm->ev[kind][which], s, cudaEventRecordExternal);
    else
      cudaEventRecord(tm->ev[kind][which], s);
  };
  auto slot = [&](int kind) { return tm ? tm->slot[kind] : -1; };
  mark(1, 0);
  launch_mf_sep(A, nullptr, st, 1, ws, s);
  launch_pdl(bwd_kernel<BWD_SOLVER>(A), ws.grid_bwd, s, A, nullptr, nullptr, 0.f, 1.f, 0.0, nullptr,
             ws.bwd, nullptr, nullptr, st, slot(1), nullptr, nullptr);
  mark(1, 1);
  mark(0, 0);
  if (solver == PASS_GPBB2)
    launch_mf_fsep<4>(A, nullptr, st, ws, s);
  else
    launch_mf_fsep<2>(A, nullptr, st, ws, s);
  // `solver` is the pass kind: a solver, or PASS_GPBB2 (two trial points)
  auto trial = solver == SOLVER_UPN   ? fwd_kernel<FWD_TRIAL_X>(A)
               : solver == PASS_GPBB2 ? fwd_kernel<FWD_TRIAL_2>(A)
                                      : fwd_kernel<FWD_TRIAL>(A);
  const int grid = solver == SOLVER_UPN   ? ws.grid_trial_x
                   : solver == PASS_GPBB2 ? ws.grid_trial_2
                                          : ws.grid_trial;
  launch_pdl(trial, grid, s, A, nullptr, nullptr, nullptr, ws.fwd, st, slot(0), nullptr);
  mark(0, 1);
}

void launch_trial(const MatDev &A, DevState *st, const Workspace &ws, cudaStream_t s) {
  launch_mf_fsep<2>(A, nullptr, st, ws, s);
  launch_pdl(fwd_kernel<FWD_TRIAL>(A), ws.grid_trial, s, A, nullptr, nullptr, nullptr, ws.fwd, st,
             -1, nullptr);
}

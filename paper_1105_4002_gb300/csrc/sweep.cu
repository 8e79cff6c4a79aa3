// Parameter sweep: up to 8 solves of the same system and data with different
// alpha, in lockstep, sharing every read of A.
//
// Vectors of the sweep are interleaved [index][8] (column c of entry i at
// i * 8 + c), so one gather of an index in a projection brings the 8 values
// of all columns in one 32-byte sector.  A pass is
//   [UPN: extrapolation] -> A^T gather -> gradient + TV stencil + control
//   -> projected steps -> A gather -> residuals + acceptance tests,
// where the two projections (k_spmm_cols, k_spmm_rows) read A once for all
// columns and every other kernel runs one thread per (index, column).
// Each column keeps its own DevState: its vector pointers address column c
// with stride 8, so the control code of the single solves (ctrl.cuh) runs
// unchanged per column, its pointer swaps acting as per-column parity flips.
// A column that has stopped, or that has no new point, is masked out; a pass
// skips a projection when no column needs it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "ctrl.cuh"
#include "system.cuh"

namespace {

constexpr int KS = 8;               // columns of a sweep
// blocks of a reducing sweep kernel: its partials (grid * KS * 4 values) fill
// at most a reduction slot
constexpr int kSweepMaxGrid = TVR_MAX_GRID * TVR_RMAX / (KS * 4);

struct SweepDev {
  DevState col[KS];
  int k;  // columns in use
};

// Interleaved arrays of one sweep.
struct SweepBufs {
  float *P0, *P1, *Y, *G0, *G1, *XB, *DD, *S;  // N * KS
  float *R0, *R1, *RY, *U, *AD, *RG, *Z, *ZD;  // m * KS
};

// ---- column-layout reduction: thread t always handles column t % KS ----
template <int R>
__device__ bool col_reduce(FF (&a)[R], const RedSlot &slot, double (&tot)[R]) {
  __shared__ FF sh[TVR_BLOCK / 32][KS][R];
  __shared__ FF fin[32][KS][R];
  __shared__ bool am_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < R; ++k) {
    a[k] = ff_merge(a[k], ff_shfl_down(a[k], 16));
    a[k] = ff_merge(a[k], ff_shfl_down(a[k], 8));
  }
  if (lane < KS)
#pragma unroll
    for (int k = 0; k < R; ++k) sh[warp][lane][k] = a[k];
  __syncthreads();
  if (threadIdx.x < KS) {
#pragma unroll
    for (int k = 0; k < R; ++k) {
      FF v = ff_zero();
      for (int w = 0; w < TVR_BLOCK / 32; ++w) v = ff_merge(v, sh[w][threadIdx.x][k]);
      slot.partials[(blockIdx.x * KS + threadIdx.x) * R + k] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    am_last = atomicAdd(slot.counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  const int c = threadIdx.x % KS, grp = threadIdx.x / KS;  // 32 groups of 8
  FF v[R];
#pragma unroll
  for (int k = 0; k < R; ++k) v[k] = ff_zero();
  for (int b = grp; b < (int)gridDim.x; b += TVR_BLOCK / KS) {
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const float2 p = __ldcg(reinterpret_cast<const float2 *>(slot.partials + (b * KS + c) * R + k));
      v[k] = ff_merge(v[k], FF{p.x, p.y});
    }
  }
#pragma unroll
  for (int k = 0; k < R; ++k) fin[grp][c][k] = v[k];
  __syncthreads();
  if (threadIdx.x < KS) {
#pragma unroll
    for (int k = 0; k < R; ++k) {
      FF s = ff_zero();
      for (int g = 0; g < TVR_BLOCK / KS; ++g) s = ff_merge(s, fin[g][threadIdx.x][k]);
      tot[k] = ff_to_double(s);
    }
  }
  if (threadIdx.x == 0) *slot.counter = 0u;
  return true;
}

// ---- strided stencil helpers (column pointer, stride KS) ----
__device__ __forceinline__ float at(const float *p, int64_t j) { return p[j * KS]; }

__device__ __forceinline__ void diff3s(const float *x, int ix, int iy, int iz, int n, float z[3]) {
  const int64_t j = (int64_t)ix + (int64_t)n * (iy + (int64_t)n * iz);
  const float c = at(x, j);
  z[0] = ix + 1 < n ? __fsub_rn(at(x, j + 1), c) : 0.f;
  z[1] = iy + 1 < n ? __fsub_rn(at(x, j + n), c) : 0.f;
  z[2] = iz + 1 < n ? __fsub_rn(at(x, j + (int64_t)n * n), c) : 0.f;
}

__device__ __forceinline__ void huber_s(const float *x, int ix, int iy, int iz, int n, float tau,
                                        Huber &o) {
  if (ix < 0 || iy < 0 || iz < 0) {
    o.z[0] = o.z[1] = o.z[2] = 0.f;
    o.w[0] = o.w[1] = o.w[2] = 0.f;
    o.nrm = o.h = 0.f;
    return;
  }
  diff3s(x, ix, iy, iz, n, o.z);
  o.nrm = norm3(o.z);
  huber_weights(o.z, o.nrm, tau, o.w);
  o.h = huber_h(o.nrm, tau);
}

__device__ __forceinline__ float proj(float v) { return v < 0.f ? 0.f : v; }


// ---- projections shared by all columns ----
// G lanes per row (the row split): each lane reads 4 entries with one 16-byte
// load of indices and one of values, at stride 4 G; any G covers every entry
// of the lane-interleaved storage exactly once, only the order of additions
// changes.
template <int G, bool TWO, bool BF, bool U16 = false>
__global__ void __launch_bounds__(TVR_BLOCK)
    k_spmm_rows(MatDev A, const float *__restrict__ in0, const float *__restrict__ in1,
                float *__restrict__ out0, float *__restrict__ out1, const SweepDev *sd, int init) {
  static_assert(G == 2 || G == 4 || G == 8, "lanes per row");
  if (!init) {
    bool any = false;
    for (int c = 0; c < KS; ++c) any = any || !sd->col[c].done;
    if (!any) return;
  }
  const int lane = threadIdx.x & (G - 1), sub = (threadIdx.x & 31) / G;
  const int64_t warp = ((int64_t)blockIdx.x * TVR_BLOCK + threadIdx.x) >> 5;
  const int64_t nwarp = (int64_t)gridDim.x * (TVR_BLOCK / 32);
  for (int64_t base = warp * (32 / G); base < A.m; base += nwarp * (32 / G)) {
    const int64_t row = base + sub;
    const bool valid = row < A.m;
    const int64_t beg = valid ? __ldg(A.row_ptr + row) : 0, end = valid ? __ldg(A.row_ptr + row + 1) : 0;
    float s0[KS], s1[KS];
#pragma unroll
    for (int c = 0; c < KS; ++c) s0[c] = s1[c] = 0.f;
    for (int64_t e0 = beg + 4 * lane; e0 < end; e0 += 4 * G) {
      const int4 c4 = ld_stream(A.col + e0);
      float4 v4;
      if (BF) {
        v4 = decode16<U16>(ld_stream2(A.qval + e0));
      } else {
        v4 = ld_stream(A.val + e0);
      }
      const int cs[4] = {c4.x, c4.y, c4.z, c4.w};
      const float vs[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float4 *p0 = reinterpret_cast<const float4 *>(in0 + (int64_t)cs[u] * KS);
        const float4 a = __ldg(p0), b = __ldg(p0 + 1);
        s0[0] = __fmaf_rn(vs[u], a.x, s0[0]); s0[1] = __fmaf_rn(vs[u], a.y, s0[1]);
        s0[2] = __fmaf_rn(vs[u], a.z, s0[2]); s0[3] = __fmaf_rn(vs[u], a.w, s0[3]);
        s0[4] = __fmaf_rn(vs[u], b.x, s0[4]); s0[5] = __fmaf_rn(vs[u], b.y, s0[5]);
        s0[6] = __fmaf_rn(vs[u], b.z, s0[6]); s0[7] = __fmaf_rn(vs[u], b.w, s0[7]);
        if (TWO) {
          const float4 *p1 = reinterpret_cast<const float4 *>(in1 + (int64_t)cs[u] * KS);
          const float4 d = __ldg(p1), f = __ldg(p1 + 1);
          s1[0] = __fmaf_rn(vs[u], d.x, s1[0]); s1[1] = __fmaf_rn(vs[u], d.y, s1[1]);
          s1[2] = __fmaf_rn(vs[u], d.z, s1[2]); s1[3] = __fmaf_rn(vs[u], d.w, s1[3]);
          s1[4] = __fmaf_rn(vs[u], f.x, s1[4]); s1[5] = __fmaf_rn(vs[u], f.y, s1[5]);
          s1[6] = __fmaf_rn(vs[u], f.z, s1[6]); s1[7] = __fmaf_rn(vs[u], f.w, s1[7]);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < KS; ++c) {
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) {
        s0[c] = __fadd_rn(s0[c], __shfl_down_sync(0xffffffffu, s0[c], o, G));
        if (TWO) s1[c] = __fadd_rn(s1[c], __shfl_down_sync(0xffffffffu, s1[c], o, G));
      }
    }
    if (valid && lane == 0) {
      const float sc = BF ? __ldg(A.rscale + row) : 1.f;
      float4 *o0 = reinterpret_cast<float4 *>(out0 + row * KS);
      o0[0] = make_float4(__fmul_rn(sc, s0[0]), __fmul_rn(sc, s0[1]), __fmul_rn(sc, s0[2]), __fmul_rn(sc, s0[3]));
      o0[1] = make_float4(__fmul_rn(sc, s0[4]), __fmul_rn(sc, s0[5]), __fmul_rn(sc, s0[6]), __fmul_rn(sc, s0[7]));
      if (TWO) {
        float4 *o1 = reinterpret_cast<float4 *>(out1 + row * KS);
        o1[0] = make_float4(__fmul_rn(sc, s1[0]), __fmul_rn(sc, s1[1]), __fmul_rn(sc, s1[2]), __fmul_rn(sc, s1[3]));
        o1[1] = make_float4(__fmul_rn(sc, s1[4]), __fmul_rn(sc, s1[5]), __fmul_rn(sc, s1[6]), __fmul_rn(sc, s1[7]));
      }
    }
  }
}

template <int G, bool BF, bool U16 = false>
__global__ void __launch_bounds__(TVR_BLOCK)
    k_spmm_cols(MatDev A, const float *__restrict__ in, float *__restrict__ out, const SweepDev *sd,
                int init) {
  static_assert(G == 2 || G == 4 || G == 8, "lanes per column");
  if (!init) {
    bool any = false;
    for (int c = 0; c < KS; ++c) any = any || (!sd->col[c].done && sd->col[c].need_grad);
    if (!any) return;
  }
  const int lane = threadIdx.x & (G - 1), sub = (threadIdx.x & 31) / G;
  const int64_t warp = ((int64_t)blockIdx.x * TVR_BLOCK + threadIdx.x) >> 5;
  const int64_t nwarp = (int64_t)gridDim.x * (TVR_BLOCK / 32);
  for (int64_t base = warp * (32 / G); base < A.N; base += nwarp * (32 / G)) {
    const int64_t j = base + sub;
    const bool valid = j < A.N;
    const int64_t beg = valid ? __ldg(A.col_ptr + j) : 0, end = valid ? __ldg(A.col_ptr + j + 1) : 0;
    float s[KS];
#pragma unroll
    for (int c = 0; c < KS; ++c) s[c] = 0.f;
    for (int64_t e0 = beg + 4 * lane; e0 < end; e0 += 4 * G) {
      const int4 i4 = ld_stream(A.row + e0);
      float4 v4;
      if (BF) {
        v4 = decode16<U16>(ld_stream2(A.qcval + e0));
      } else {
        v4 = ld_stream(A.cval + e0);
      }
      const int is[4] = {i4.x, i4.y, i4.z, i4.w};
      const float vs[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float4 *p = reinterpret_cast<const float4 *>(in + (int64_t)is[u] * KS);
        const float4 a = __ldg(p), b = __ldg(p + 1);
        s[0] = __fmaf_rn(vs[u], a.x, s[0]); s[1] = __fmaf_rn(vs[u], a.y, s[1]);
        s[2] = __fmaf_rn(vs[u], a.z, s[2]); s[3] = __fmaf_rn(vs[u], a.w, s[3]);
        s[4] = __fmaf_rn(vs[u], b.x, s[4]); s[5] = __fmaf_rn(vs[u], b.y, s[5]);
        s[6] = __fmaf_rn(vs[u], b.z, s[6]); s[7] = __fmaf_rn(vs[u], b.w, s[7]);
      }
    }
#pragma unroll
    for (int c = 0; c < KS; ++c)
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) s[c] = __fadd_rn(s[c], __shfl_down_sync(0xffffffffu, s[c], o, G));
    if (valid && lane == 0) {
      float4 *o = reinterpret_cast<float4 *>(out + j * KS);
      o[0] = make_float4(s[0], s[1], s[2], s[3]);
      o[1] = make_float4(s[4], s[5], s[6], s[7]);
    }
  }
}

// Index of (entry, column) thread layout: column c = t % KS fixed per thread.
struct ColIter {
  int c;
  int64_t i, stride;
  __device__ ColIter() {
    const int64_t t = (int64_t)blockIdx.x * TVR_BLOCK + threadIdx.x;
    c = (int)(t % KS);
    i = t / KS;
    stride = (int64_t)gridDim.x * TVR_BLOCK / KS;
  }
};

// ---- residual after the forward projection ----
// init: r = Z - b -> R (or RY for UPN) and RG; sum r^2 -> r_init.
// trial: r = Z - b -> RT, RG (GP / GPBB), AD = ZD (UPN); sums r^2, (A d)^2 -> ctrl_trial.
template <bool INIT, bool BF>
__global__ void __launch_bounds__(TVR_BLOCK)
    k_sw_fwd_post(MatDev A, const float *__restrict__ b, const float *__restrict__ Z,
                  const float *__restrict__ ZD, float *__restrict__ RG, SweepDev *sd, RedSlot slot) {
  ColIter it;
  DevState *st = &sd->col[it.c];
  const bool active = INIT ? it.c < sd->k : !st->done;
  const bool upn = st->solver == SOLVER_UPN;
  float *r = INIT ? (upn ? st->vM[RM_RY] : st->vM[RM_R]) : st->vM[RM_RT];
  float *ad = upn ? st->vM[RM_AD] : nullptr;
  FF a0 = ff_zero(), a1 = ff_zero();
  if (active) {
    for (int64_t i = it.i; i < A.m; i += it.stride) {
      const float ri = __fsub_rn(Z[i * KS + it.c], __ldg(b + i));
      r[i * KS] = ri;
      if (INIT || !upn) RG[i * KS + it.c] = BF ? __fmul_rn(__ldg(A.rscale + i), ri) : ri;
      ff_add_prod(a0, ri, ri);
      if (!INIT) {
        const float d = ZD[i * KS + it.c];
        if (ad) ad[i * KS] = d;
        ff_add_prod(a1, d, d);
      }
    }
  }
  FF acc[2] = {a0, a1};
  double tot[2];
  if (col_reduce<2>(acc, slot, tot) && threadIdx.x < KS) {
    DevState *s = &sd->col[threadIdx.x];
    if (INIT) {
      if ((int)threadIdx.x < sd->k) s->r_init[0] = tot[0];
    } else if (!s->done) {
      s->r_fwd[0] = tot[0];
      s->r_fwd[1] = tot[1];
      ctrl_trial(s, tot);
    }
  }
}

// ---- gradient after the back projection: g = S + alpha grad TV_tau at the base point ----
template <bool INIT>
__global__ void __launch_bounds__(TVR_BLOCK, 4)
    k_sw_bwd_post(MatDev A, const float *__restrict__ S, SweepDev *sd, RedSlot slot) {
  ColIter it;
  DevState *st = &sd->col[it.c];
  const bool active = INIT ? it.c < sd->k : (!st->done && st->need_grad);
  const int kind = st->solver;
  const float alpha = (float)st->alpha, tau = (float)st->tau;
  const float *x = kind == SOLVER_UPN ? st->vN[RN_Y] : st->vN[RN_X];
  float *g = (!INIT && kind == SOLVER_GPBB) ? st->vN[RN_GN] : st->vN[RN_G];
  const float *q = st->vN[RN_X];   // UPN: x^(k) for the Bregman sum at y^(k)
  const float *xo = st->vN[RN_T];  // GPBB: x^(k-1)
  const float *go = st->vN[RN_G];  // GPBB: g^(k-1)
  const int n = A.n;
  FF a0 = ff_zero(), a1 = ff_zero(), a2 = ff_zero();
  if (active) {
    for (int64_t j = it.i; j < A.N; j += it.stride) {
      int ix, iy, iz;
      voxel_of(A, j, ix, iy, iz);
      Huber h0, h1, h2, h3;
      huber_s(x, ix, iy, iz, n, tau, h0);
      huber_s(x, ix - 1, iy, iz, n, tau, h1);
      huber_s(x, ix, iy - 1, iz, n, tau, h2);
      huber_s(x, ix, iy, iz - 1, n, tau, h3);
      // same association as the lane-shuffle sum of the single-solve kernel
      const float own = -__fadd_rn(__fadd_rn(h0.w[0], h0.w[1]), h0.w[2]);
      const float tvg = __fadd_rn(__fadd_rn(own, h2.w[1]), __fadd_rn(h1.w[0], h3.w[2]));
      const float gj = __fmaf_rn(alpha, tvg, S[j * KS + it.c]);
      g[j * KS] = gj;
      ff_add(a0, h0.h);
      if (!INIT && kind == SOLVER_GPBB) {
        const float sj = __fsub_rn(at(x, j), at(xo, j));
        ff_add_prod(a1, sj, __fsub_rn(gj, at(go, j)));
        ff_add_prod(a2, sj, sj);
      }
      if (!INIT && kind == SOLVER_UPN) {
        const int64_t nn = (int64_t)n * n;
        float zb[3], dl[3];
        diff3s(q, ix, iy, iz, n, zb);
        const float d0 = __fsub_rn(at(q, j), at(x, j));
        dl[0] = ix + 1 < n ? __fsub_rn(__fsub_rn(at(q, j + 1), at(x, j + 1)), d0) : 0.f;
        dl[1] = iy + 1 < n ? __fsub_rn(__fsub_rn(at(q, j + n), at(x, j + n)), d0) : 0.f;
        dl[2] = iz + 1 < n ? __fsub_rn(__fsub_rn(at(q, j + nn), at(x, j + nn)), d0) : 0.f;
        ff_add(a1, huber_bregman(h0.z, h0.nrm, zb, dl, tau));
      }
    }
  }
  FF acc[3] = {a0, a1, a2};
  double tot[3];
  if (col_reduce<3>(acc, slot, tot) && threadIdx.x < KS) {
    DevState *s = &sd->col[threadIdx.x];
    if (INIT) {
      if ((int)threadIdx.x < sd->k) ctrl_init(s, tot);
    } else if (!s->done && s->need_grad) {
      s->r_bwd[0] = tot[0];
      s->r_bwd[1] = tot[1];
      s->r_bwd[2] = tot[2];
      ctrl_after_grad(s, tot);
    }
  }
}

// ---- projected steps (one thread per voxel and column) ----
__global__ void __launch_bounds__(TVR_BLOCK)
    k_sw_step(MatDev A, float *__restrict__ XB, float *__restrict__ DD, SweepDev *sd, RedSlot slot) {
  ColIter it;
  DevState *st = &sd->col[it.c];
  const bool active = !st->done;
  const bool upn = st->solver == SOLVER_UPN;
  const float *p = upn ? st->vN[RN_Y] : st->vN[RN_X];
  const float *g = st->vN[RN_G];
  float *t = st->vN[RN_T];
  const float s = (float)st->step, s2 = (float)st->step2, tau = (float)st->tau;
  const bool want_g2 = st->solver == SOLVER_GPBB && st->trial == 0;
  const int n = A.n;
  FF a0 = ff_zero(), a1 = ff_zero(), a2 = ff_zero(), a3 = ff_zero();
  if (active) {
    for (int64_t j = it.i; j < A.N; j += it.stride) {
      const float pj = at(p, j), gj = at(g, j);
      const float xb = proj(__fsub_rn(pj, __fmul_rn(s, gj)));
      const float d = __fsub_rn(xb, pj);
      t[j * KS] = xb;
      XB[j * KS + it.c] = xb;
      DD[j * KS + it.c] = d;
      ff_add_prod(a0, gj, d);
      ff_add_prod(a1, d, d);
      if (want_g2) {
        const float e = __fsub_rn(pj, proj(__fsub_rn(pj, __fmul_rn(s2, gj))));
        ff_add_prod(a3, e, e);
      }
      int ix, iy, iz;
      voxel_of(A, j, ix, iy, iz);
      const int64_t off[3] = {1, n, (int64_t)n * n};
      const bool in[3] = {ix + 1 < n, iy + 1 < n, iz + 1 < n};
      float z[3], zb[3], dl[3];
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        if (in[e]) {
          const float pk = at(p, j + off[e]), gk = at(g, j + off[e]);
          const float xk = proj(__fsub_rn(pk, __fmul_rn(s, gk)));
          z[e] = __fsub_rn(pk, pj);
          zb[e] = __fsub_rn(xk, xb);
          dl[e] = __fsub_rn(__fsub_rn(xk, pk), d);
        } else {
          z[e] = zb[e] = dl[e] = 0.f;
        }
      }
      ff_add(a2, huber_bregman(z, norm3(z), zb, dl, tau));
    }
  }
  FF acc[4] = {a0, a1, a2, a3};
  double tot[4];
  if (col_reduce<4>(acc, slot, tot) && threadIdx.x < KS) {
    DevState *sc = &sd->col[threadIdx.x];
    if (!sc->done)
      for (int k = 0; k < 4; ++k) sc->r_step[k] = tot[k];
  }
}

// ---- UPN extrapolation; also refreshes the gathered residual RG ----
template <bool BF>
__global__ void __launch_bounds__(TVR_BLOCK)
    k_sw_yform(MatDev A, float *__restrict__ RG, SweepDev *sd, RedSlot slot) {
  ColIter it;
  DevState *st = &sd->col[it.c];
  const bool active = !st->done && st->need_grad;
  const float beta = (float)st->beta, bp = (float)st->beta_prev;
  const float *X = st->vN[RN_X];
  const float *T = st->vN[RN_T];
  float *Y = st->vN[RN_Y];
  const float *R = st->vM[RM_R];
  const float *AD = st->vM[RM_AD];
  float *U = st->vM[RM_U];
  float *RY = st->vM[RM_RY];
  FF a0 = ff_zero(), a1 = ff_zero();
  if (active) {
    const int64_t lim = A.N > A.m ? A.N : A.m;
    for (int64_t i = it.i; i < lim; i += it.stride) {
      if (i < A.N) {
        const float xn = at(X, i);
        const float dx = __fsub_rn(xn, at(T, i));
        Y[i * KS] = __fmaf_rn(beta, dx, xn);
        ff_add_prod(a0, dx, dx);
      }
      if (i < A.m) {
        const float u = __fmaf_rn(bp, at(U, i), at(AD, i));
        U[i * KS] = u;
        const float ry = __fmaf_rn(beta, u, at(R, i));
        RY[i * KS] = ry;
        RG[i * KS + it.c] = BF ? __fmul_rn(__ldg(A.rscale + i), ry) : ry;
        ff_add_prod(a1, u, u);
      }
    }
  }
  FF acc[2] = {a0, a1};
  double tot[2];
  if (col_reduce<2>(acc, slot, tot) && threadIdx.x < KS) {
    DevState *s = &sd->col[threadIdx.x];
    if (!s->done && s->need_grad) {
      s->r_yf[0] = tot[0];
      s->r_yf[1] = tot[1];
    }
  }
}

// Column c of an interleaved array -> dst[c * n + j] (column-major), and back.
__global__ void k_deinterleave(const SweepDev *sd, int64_t n, float *__restrict__ dst) {
  ColIter it;
  if (it.c >= sd->k) return;
  const float *x = sd->col[it.c].vN[RN_X];
  for (int64_t j = it.i; j < n; j += it.stride) dst[it.c * n + j] = x[j * KS];
}

__global__ void k_interleave(const float *__restrict__ src, int k, int64_t n, float *__restrict__ a,
                             float *__restrict__ b) {
  ColIter it;
  for (int64_t j = it.i; j < n; j += it.stride) {
    const float v = it.c < k ? src[it.c * n + j] : 0.f;
    a[j * KS + it.c] = v;
    if (b) b[j * KS + it.c] = v;
  }
}

int sweep_grid(int64_t n_index, int cap) {
  int64_t bl = (n_index * KS + TVR_BLOCK - 1) / TVR_BLOCK;
  if (bl < 1) bl = 1;
  return (int)(bl < cap ? bl : cap);
}

struct SweepCache {
  SweepBufs buf{};
  float *mem = nullptr;
  SweepDev *sd = nullptr;
  int *flag = nullptr;
};

}  // namespace

// The sweep's device memory lives with the system (freed with it).
struct tvr_sweep_mem {
  SweepCache c;
};

void sweep_free(tvr_sweep_mem *m) {
  if (!m) return;
  if (m->c.mem) cudaFree(m->c.mem);
  if (m->c.sd) cudaFree(m->c.sd);
  if (m->c.flag) cudaFreeHost(m->c.flag);
  delete m;
}

namespace {

using RowsFn = void (*)(MatDev, const float *, const float *, float *, float *, const SweepDev *,
                       int);
using ColsFn = void (*)(MatDev, const float *, float *, const SweepDev *, int);

// kernel instance for the row split G and the value format (A.bf16: 16-bit
// codes; A.u16: unsigned fixed point rather than bfloat16)
template <bool TWO>
RowsFn rows_fn(int G, const MatDev &A) {
  if (A.bf16 && A.u16)
    return G == 2 ? k_spmm_rows<2, TWO, true, true> : G == 8 ? k_spmm_rows<8, TWO, true, true>
                                                              : k_spmm_rows<4, TWO, true, true>;
  if (A.bf16) return G == 2 ? k_spmm_rows<2, TWO, true> : G == 8 ? k_spmm_rows<8, TWO, true>
                                                                   : k_spmm_rows<4, TWO, true>;
  return G == 2 ? k_spmm_rows<2, TWO, false> : G == 8 ? k_spmm_rows<8, TWO, false>
                                                     : k_spmm_rows<4, TWO, false>;
}
ColsFn cols_fn(int G, const MatDev &A) {
  if (A.bf16 && A.u16)
    return G == 2 ? k_spmm_cols<2, true, true> : G == 8 ? k_spmm_cols<8, true, true>
                                                        : k_spmm_cols<4, true, true>;
  if (A.bf16) return G == 2 ? k_spmm_cols<2, true> : G == 8 ? k_spmm_cols<8, true> : k_spmm_cols<4, true>;
  return G == 2 ? k_spmm_cols<2, false> : G == 8 ? k_spmm_cols<8, false> : k_spmm_cols<4, false>;
}

// Launch configuration of a sweep: the row split of each projection (lanes
// per row / column) with its kernel and grid -- the grid from the kernel's own
// occupancy (the forward gathers two interleaved arrays and holds 16 sums:
// fewer blocks fit per SM than for the single-solve kernels), capped by the
// rows / columns there are -- and one resident wave for each (index, column)
// kernel, at most a reduction slot's worth.
struct SweepGrids {
  int lanes_rows = 4, lanes_cols = 4;
  RowsFn rows_two = nullptr, rows_one = nullptr;
  ColsFn cols = nullptr;
  int g_rows_two = 1, g_rows_one = 1, g_cols = 1;  // projections
  int yform = 1, bwd_post = 1, step = 1, fwd_post = 1;
};

int proj_grid(const void *k, int lanes, int64_t items, int device) {
  const int g = occupancy_grid(k, TVR_BLOCK, device);
  const int64_t per = TVR_BLOCK / lanes;  // rows or columns per block
  const int64_t need = (items + per - 1) / per;
  return (int)(need < 1 ? 1 : (need < g ? need : g));
}

SweepGrids sweep_grids(const MatDev &A, int device, int lanes_rows, int lanes_cols) {
  const bool bf = A.bf16;
  SweepGrids g;
  g.lanes_rows = lanes_rows;
  g.lanes_cols = lanes_cols;
  g.rows_two = rows_fn<true>(lanes_rows, A);
  g.rows_one = rows_fn<false>(lanes_rows, A);
  g.cols = cols_fn(lanes_cols, A);
  g.g_rows_two = proj_grid((const void *)g.rows_two, lanes_rows, A.m, device);
  g.g_rows_one = proj_grid((const void *)g.rows_one, lanes_rows, A.m, device);
  g.g_cols = proj_grid((const void *)g.cols, lanes_cols, A.N, device);
  auto wave = [](int gr, int64_t items) {
    const int64_t need = (items * KS + TVR_BLOCK - 1) / TVR_BLOCK;
    int64_t b = need < gr ? need : gr;
    if (b > kSweepMaxGrid) b = kSweepMaxGrid;
    return (int)(b < 1 ? 1 : b);
  };
  const int64_t mx = A.N > A.m ? A.N : A.m;
  g.yform = wave(occupancy_grid(bf ? (const void *)k_sw_yform<true> : (const void *)k_sw_yform<false>,
                                TVR_BLOCK, device),
                 mx);
  g.bwd_post = wave(occupancy_grid((const void *)k_sw_bwd_post<false>, TVR_BLOCK, device), A.N);
  g.step = wave(occupancy_grid((const void *)k_sw_step, TVR_BLOCK, device), A.N);
  g.fwd_post = wave(occupancy_grid(bf ? (const void *)k_sw_fwd_post<false, true>
                                      : (const void *)k_sw_fwd_post<false, false>,
                                   TVR_BLOCK, device),
                    A.m);
  return g;
}

// Row-split autotuner: times each projection with 2, 4 and 8 lanes per row /
// column on this system (one untimed and two timed launches each, on buffers
// cleared for it; the sweep's initialisation overwrites what they write) and
// keeps the fastest, preferring 4 lanes within 5%.  The choice is cached per
// (rows, columns, entries, storage, GPU) for the life of the process.
struct TuneKey {
  int64_t m, N, nnz;
  int bf, device;
  bool operator<(const TuneKey &o) const {
    return std::tie(m, N, nnz, bf, device) < std::tie(o.m, o.N, o.nnz, o.bf, o.device);
  }
};

int sweep_tune(const MatDev &A, int device, const SweepBufs &B, const SweepDev *sd,
               cudaStream_t s, int *lanes_rows, int *lanes_cols) {
  static std::mutex mu;
  static std::map<TuneKey, std::pair<int, int>> cache;
  const TuneKey key{A.m, A.N, A.nnz, A.bf16 ? (A.u16 ? 2 : 1) : 0, device};
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      *lanes_rows = it->second.first;
      *lanes_cols = it->second.second;
      return TVR_OK;
    }
  }
  TVR_CUDA(cudaMemsetAsync(B.XB, 0, sizeof(float) * KS * A.N, s));
  TVR_CUDA(cudaMemsetAsync(B.DD, 0, sizeof(float) * KS * A.N, s));
  TVR_CUDA(cudaMemsetAsync(B.RG, 0, sizeof(float) * KS * A.m, s));
  // destroyed on every exit path, including the early returns of TVR_CUDA
  struct Events {
    cudaEvent_t e[2] = {nullptr, nullptr};
    ~Events() {
      for (cudaEvent_t v : e)
        if (v) cudaEventDestroy(v);
    }
  } ev;
  TVR_CUDA(cudaEventCreate(&ev.e[0]));
  TVR_CUDA(cudaEventCreate(&ev.e[1]));
  cudaEvent_t e0 = ev.e[0], e1 = ev.e[1];
  auto timed = [&](auto launch, float *ms) -> int {
    launch();
    TVR_CUDA(cudaEventRecord(e0, s));
    launch();
    launch();
    TVR_CUDA(cudaEventRecord(e1, s));
    TVR_CUDA(cudaEventSynchronize(e1));
    TVR_CUDA(cudaGetLastError());
    TVR_CUDA(cudaEventElapsedTime(ms, e0, e1));
    return TVR_OK;
  };
  // 4 lanes (the single solves' split, index 1) is kept unless another split
  // is faster by more than 5%: where the splits time within noise, the choice
  // -- and with it the order of additions -- stays the same from run to run
  const int cand[3] = {2, 4, 8};
  float tr[3] = {0.f, 0.f, 0.f}, tc[3] = {0.f, 0.f, 0.f};
  int rc = TVR_OK;
  for (int i = 0; i < 3 && rc == TVR_OK; ++i) {
    const int L = cand[i];
    const RowsFn fr = rows_fn<true>(L, A);
    const int gr = proj_grid((const void *)fr, L, A.m, device);
    rc = timed([&] { fr<<<gr, TVR_BLOCK, 0, s>>>(A, B.XB, B.DD, B.Z, B.ZD, sd, 1); }, &tr[i]);
    if (rc != TVR_OK) break;
    const ColsFn fc = cols_fn(L, A);
    const int gc = proj_grid((const void *)fc, L, A.N, device);
    rc = timed([&] { fc<<<gc, TVR_BLOCK, 0, s>>>(A, B.RG, B.S, sd, 1); }, &tc[i]);
  }
  auto pick = [&](const float (&t)[3]) {
    int best = 1;
    for (int i = 0; i < 3; ++i)
      if (i != 1 && t[i] < 0.95f * t[1] && t[i] < t[best]) best = i;
    return cand[best];
  };
  const int lr = pick(tr), lc = pick(tc);
  if (rc != TVR_OK) return rc;
  std::lock_guard<std::mutex> lk(mu);
  cache[key] = {lr, lc};
  *lanes_rows = lr;
  *lanes_cols = lc;
  return TVR_OK;
}

void sweep_pass(const MatDev &A, const SweepBufs &B, SweepDev *sd, int solver, const Workspace &ws,
                const SweepGrids &sg, const float *bd, cudaStream_t s) {
  const bool bf = A.bf16;
  if (solver == SOLVER_UPN) {
    if (bf)
      k_sw_yform<true><<<sg.yform, TVR_BLOCK, 0, s>>>(A, B.RG, sd, ws.yf);
    else
      k_sw_yform<false><<<sg.yform, TVR_BLOCK, 0, s>>>(A, B.RG, sd, ws.yf);
  }
  sg.cols<<<sg.g_cols, TVR_BLOCK, 0, s>>>(A, B.RG, B.S, sd, 0);
  k_sw_bwd_post<false><<<sg.bwd_post, TVR_BLOCK, 0, s>>>(A, B.S, sd, ws.bwd);
  k_sw_step<<<sg.step, TVR_BLOCK, 0, s>>>(A, B.XB, B.DD, sd, ws.step);
  sg.rows_two<<<sg.g_rows_two, TVR_BLOCK, 0, s>>>(A, B.XB, B.DD, B.Z, B.ZD, sd, 0);
  if (bf)
    k_sw_fwd_post<false, true><<<sg.fwd_post, TVR_BLOCK, 0, s>>>(A, bd, B.Z, B.ZD, B.RG, sd, ws.fwd);
  else
    k_sw_fwd_post<false, false><<<sg.fwd_post, TVR_BLOCK, 0, s>>>(A, bd, B.Z, B.ZD, B.RG, sd, ws.fwd);
}

}  // namespace

extern "C" int tvr_solve_sweep(const tvr_system *csys, int32_t method, const float *b,
                               const double *alphas, int32_t k, double tau, double eps,
                               const tvr_solve_opts *uo, float *X, tvr_solve_info *infos,
                               void *stream) {
  tvr_system *sys = const_cast<tvr_system *>(csys);
  if (!sys || !b || !alphas || !X) return fail(TVR_ERR_ARG, "tvr_solve_sweep: null argument");
  if (k < 1 || k > KS) return fail(TVR_ERR_ARG, "tvr_solve_sweep: need 1 <= k <= 8");
  if (sys->A.storage == TVR_STORAGE_MATRIX_FREE)
    return fail(TVR_ERR_ARG, "tvr_solve_sweep: needs a stored matrix (FP32 or BF16 storage)");
  if (method != SOLVER_GP && method != SOLVER_GPBB && method != SOLVER_UPN)
    return fail(TVR_ERR_ARG, "tvr_solve_sweep: method must be 1 (GP), 2 (GPBB) or 3 (UPN)");
  for (int c = 0; c < k; ++c)
    if (!(alphas[c] >= 0.0) || !std::isfinite(alphas[c]))
      return fail(TVR_ERR_ARG, "tvr_solve_sweep: alphas must be finite and >= 0");
  if (!(tau > 0.0) || !std::isfinite(tau) || !(eps > 0.0) || !std::isfinite(eps))
    return fail(TVR_ERR_ARG, "tvr_solve_sweep: need tau > 0 and eps > 0");
  tvr_solve_opts o;
  tvr_solve_opts_default(&o);
  if (uo) o = *uo;
  if (o.k_max < 1 || o.gpbb_K < 0 || o.gpbb_K > 8 || o.gpbb_max_trials < 0 || o.bt_max < 0 ||
      o.batch < 1 || o.batch > 1024 || !(o.rho_L > 1.0) || !(o.L_bar > 0.0) || !(o.mu_bar >= 0.0) ||
      !(o.gpbb_sigma > 0.0 && o.gpbb_sigma < 1.0) || !(o.gpbb_beta0 > 0.0 && o.gpbb_beta0 < 1.0) ||
      (o.stop_mode != TVR_STOP_REL && o.stop_mode != TVR_STOP_PER_N) ||
      (o.sweep_lanes != 0 && o.sweep_lanes != 2 && o.sweep_lanes != 4 && o.sweep_lanes != 8))
    return fail(TVR_ERR_ARG, "tvr_solve_sweep: invalid options");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t N = sys->N, m = sys->m;
  // device memory of the sweep, kept with the system for later sweeps
  if (!sys->sweep) {
    tvr_sweep_mem *mm = new tvr_sweep_mem();
    const size_t total = (size_t)KS * (8 * N + 8 * m);
    cudaError_t e = cudaMalloc(&mm->c.mem, sizeof(float) * total);
    if (e == cudaSuccess) e = cudaMalloc(&mm->c.sd, sizeof(SweepDev));
    if (e == cudaSuccess) e = cudaMallocHost(&mm->c.flag, sizeof(SweepDev));
    if (e != cudaSuccess) {
      sweep_free(mm);
      return cuda_fail(e, "tvr_solve_sweep: allocation");
    }
    float *p = mm->c.mem;
    float **nv[8] = {&mm->c.buf.P0, &mm->c.buf.P1, &mm->c.buf.Y, &mm->c.buf.G0,
                     &mm->c.buf.G1, &mm->c.buf.XB, &mm->c.buf.DD, &mm->c.buf.S};
    for (auto q : nv) {
      *q = p;
      p += KS * N;
    }
    float **mv[8] = {&mm->c.buf.R0, &mm->c.buf.R1, &mm->c.buf.RY, &mm->c.buf.U,
                     &mm->c.buf.AD, &mm->c.buf.RG, &mm->c.buf.Z,  &mm->c.buf.ZD};
    for (auto q : mv) {
      *q = p;
      p += KS * m;
    }
    sys->sweep = mm;
  }
  SweepCache &C = sys->sweep->c;
  const SweepBufs &B = C.buf;
  const float *bd;
  if (int rc = stage_in(b, m, &sys->stage_bM, s, &bd)) return rc;
  // x0 of each column: interleave (host data staged column by column)
  const bool xdev = is_device_ptr(X);
  float *x0 = nullptr;
  if (xdev) {
    x0 = X;
  } else {
    if (int rc = ensure_vec(&sys->stage_sweepX, KS * N)) return rc;
    TVR_CUDA(cudaMemcpyAsync(sys->stage_sweepX, X, sizeof(float) * k * N, cudaMemcpyHostToDevice, s));
    x0 = sys->stage_sweepX;
  }
  k_interleave<<<sweep_grid(N, 4096), TVR_BLOCK, 0, s>>>(x0, k, N, B.P0, B.Y);
  TVR_CUDA(cudaMemsetAsync(B.U, 0, sizeof(float) * KS * m, s));
  // per-column states
  std::vector<SweepDev> hsd(1);
  SweepDev &h = hsd[0];
  std::memset(&h, 0, sizeof(h));
  h.k = k;
  for (int c = 0; c < KS; ++c) {
    DevState &d = h.col[c];
    d.alpha = c < k ? alphas[c] : 0.0;
    d.tau = tau;
    d.eps = eps;
    d.rho = o.rho_L;
    d.sigma = o.gpbb_sigma;
    d.beta0 = o.gpbb_beta0;
    d.Lbar = o.L_bar;
    d.mubar = o.mu_bar;
    d.kmax = o.k_max;
    d.K = o.gpbb_K;
    d.max_trials = o.gpbb_max_trials;
    d.bt_max = o.bt_max;
    d.stop_mode = o.stop_mode;
    d.solver = method;
    d.N = N;
    d.b = bd;
    d.vN[RN_X] = B.P0 + c;
    d.vN[RN_T] = B.P1 + c;
    d.vN[RN_Y] = B.Y + c;
    d.vN[RN_G] = B.G0 + c;
    d.vN[RN_GN] = B.G1 + c;
    d.vM[RM_R] = B.R0 + c;
    d.vM[RM_RT] = B.R1 + c;
    d.vM[RM_RY] = B.RY + c;
    d.vM[RM_U] = B.U + c;
    d.vM[RM_AD] = B.AD + c;
    if (c >= k) {
      d.done = 1;
      d.status = TVR_OK;
    }
  }
  TVR_CUDA(cudaMemcpyAsync(C.sd, &h, sizeof(SweepDev), cudaMemcpyHostToDevice, s));
  const MatDev A = sys->mat();
  const Workspace &ws = sys->ws;
  // row split of the projections: given, or timed on this system (before the
  // initialisation, which overwrites the buffers the timing writes)
  int lanes_rows = o.sweep_lanes, lanes_cols = o.sweep_lanes;
  if (o.sweep_lanes == 0)
    if (int rc = sweep_tune(A, sys->device, B, C.sd, s, &lanes_rows, &lanes_cols)) return rc;
  const SweepGrids sg = sweep_grids(A, sys->device, lanes_rows, lanes_cols);
  // initial residuals and gradients
  const float *xinit = method == SOLVER_UPN ? B.Y : B.P0;
  sg.rows_one<<<sg.g_rows_one, TVR_BLOCK, 0, s>>>(A, xinit, nullptr, B.Z, nullptr, C.sd, 1);
  if (A.bf16)
    k_sw_fwd_post<true, true><<<sg.fwd_post, TVR_BLOCK, 0, s>>>(A, bd, B.Z, nullptr, B.RG, C.sd, ws.fwd);
  else
    k_sw_fwd_post<true, false><<<sg.fwd_post, TVR_BLOCK, 0, s>>>(A, bd, B.Z, nullptr, B.RG, C.sd, ws.fwd);
  sg.cols<<<sg.g_cols, TVR_BLOCK, 0, s>>>(A, B.RG, B.S, C.sd, 1);
  k_sw_bwd_post<true><<<sg.bwd_post, TVR_BLOCK, 0, s>>>(A, B.S, C.sd, ws.bwd);
  TVR_CUDA(cudaGetLastError());
  // passes in batches; the host reads the column states once per batch
  const int64_t trials = (o.bt_max > o.gpbb_max_trials ? o.bt_max : o.gpbb_max_trials) + 2;
  const int64_t max_passes = ((int64_t)o.k_max + 1) * trials + o.batch;
  int64_t passes = 0;
  bool all_done = false;
  while (!all_done && passes < max_passes) {
    for (int i = 0; i < o.batch; ++i) sweep_pass(A, B, C.sd, method, ws, sg, bd, s);
    TVR_CUDA(cudaGetLastError());
    passes += o.batch;
    TVR_CUDA(cudaMemcpyAsync(C.flag, C.sd, sizeof(SweepDev), cudaMemcpyDeviceToHost, s));
    TVR_CUDA(cudaStreamSynchronize(s));
    const SweepDev *f = reinterpret_cast<const SweepDev *>(C.flag);
    all_done = true;
    for (int c = 0; c < k; ++c) all_done = all_done && f->col[c].done;
  }
  const SweepDev *f = reinterpret_cast<const SweepDev *>(C.flag);
  // results: column c of x* -> X[c * N ...]
  float *dst = xdev ? X : sys->stage_sweepX;
  k_deinterleave<<<sweep_grid(N, 4096), TVR_BLOCK, 0, s>>>(C.sd, N, dst);
  TVR_CUDA(cudaGetLastError());
  if (!xdev) TVR_CUDA(cudaMemcpyAsync(X, dst, sizeof(float) * k * N, cudaMemcpyDeviceToHost, s));
  TVR_CUDA(cudaStreamSynchronize(s));
  int worst = TVR_OK;
  for (int c = 0; c < k; ++c) {
    const DevState &d = f->col[c];
    const int status = d.done ? d.status : TVR_NOT_CONVERGED;
    if (status < 0 && worst >= 0) worst = status;
    if (status == TVR_NOT_CONVERGED && worst == TVR_OK) worst = status;
    if (infos) {
      tvr_solve_info &in = infos[c];
      std::memset(&in, 0, sizeof(in));
      in.status = status;
      in.iters = d.k;
      in.f_evals = d.f_evals;
      in.g_evals = d.g_evals;
      in.trials = d.total_trials;
      in.passes = (int32_t)passes;
      in.lanes = lanes_rows | (lanes_cols << 8);
      in.phi = NAN;
      in.gnorm = d.gnorm;
      in.gnorm0 = d.gnorm0;
      in.stop_value = d.stopval;
      in.L = method == SOLVER_GPBB ? 1.0 / d.theta : d.L;
      in.theta = d.theta;
      in.mu = d.mu;
    }
  }
  if (worst < 0) fail(worst, "tvr_solve_sweep: a column stopped with an error");
  return worst;
}

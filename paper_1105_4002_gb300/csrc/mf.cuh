// Matrix-free projector: the entries of A computed on the fly from the scan
// geometry instead of read from the stored CSR / CSC arrays.
//
// Sec. II-A defines A only as the operator that maps the image to ray sums;
// the entry a_ij is the length of ray i inside voxel j.  Here that length is
// the intersection of the ray segment (source to pixel centre) with the unit
// box of voxel j (the slab method), evaluated in float32 from per-view float32
// constants.  One function, mf_len, gives a_ij for both directions:
//   forward  (row i):    walk the slabs of the ray's major axis, take the
//                        2-4 candidate voxels of each slab, keep len > 0;
//   adjoint  (column j): for each view, take the pixels inside the bounding
//                        box of the voxel's projected corners, keep len > 0;
//                        each pixel's ray constants (1/d, |d|, start) come
//                        from a per-ray table that mf_pixel_ray filled once,
//                        instead of three reciprocals and a square root per
//                        voxel-pixel pair.
// Both enumerations are conservative (a margin of 1e-3 voxel / pixel), so the
// two projections apply exactly the same matrix and are exact transposes of
// each other; they differ from the FP64 Siddon lengths of the stored matrix
// by the float32 rounding of the ray geometry (about 2^-24 of the source and
// detector distances per coordinate).
//
// A ray parallel to a grid axis keeps the voxels with lo <= s < lo + 1 on that
// axis (the voxel of the midpoint, as in the stored matrix) and, like the
// stored matrix, no voxel when it lies on the volume's lower boundary face.
#pragma once

#include "tvr_internal.cuh"


// Per-view constants (float32).  Pixel (p, q) has centre det + a u + b w with
// a = p - (Pu - 1)/2, b = q - (Pv - 1)/2; a cone-beam ray starts at src, a
// parallel-beam ray at src + a u + b w.  nrm is oriented so that dn > 0.
struct MfView {
  float src[3], det[3], u[3], w[3];
  float nrm[3];       // unit normal of the detector plane
  float uu[3], ww[3]; // dual basis of (u, w): pixel coordinates of a detector-plane offset
  float dn;           // (det - src) . nrm
  // pixel coordinates a, b of the projection of a point X:
  //   cone:     a = a0 + dn ((X - src) . uu) / ((X - src) . nrm), b likewise with ww
  //   parallel: a = ga . X + a0, b = gb . X + b0 (linear)
  float a0, b0;
  float ga[3], gb[3];
  // cone beam, 1 when the view separates into x-y and z parts: uu, nrm have
  // no z component and ww only one (so a pixel's column a depends on x, y
  // alone), and every ray of a detector column p has the same 1/d_x and 1/d_y
  // floats (checked on the ray table at build time); a circular orbit about z
  // with the detector rows along z has it.  Else 0.
  int sep;
  float pad[6];
};

struct MfRay {
  float s[3], d[3], inv[3];  // start, d = end - start, 1 / d (0 where |d| <= 1e-30: parallel)
  float dn;                  // |d|
};

__device__ __forceinline__ float mf_half(int n) { return 0.5f * (float)n; }

// Approximate reciprocal (the PTX rcp.approx instruction, relative error about
// 2^-23), for the conservative pixel boxes of the adjoint only: an error of
// 1e-7 of a pixel coordinate of at most a few hundred pixels stays far inside
// the boxes' 1e-3 pixel margin.  No length a_ij uses it.
__device__ __forceinline__ float mf_rcp_approx(float x) {
  float y;
  asm("rcp.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void mf_pixel_ray(const MfView &v, int kind, int Pu, int Pv, int p,
                                             int q, MfRay &r) {
  const float a = __fsub_rn((float)p, 0.5f * (float)(Pu - 1));
  const float b = __fsub_rn((float)q, 0.5f * (float)(Pv - 1));
  float dd = 0.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float au = __fmul_rn(a, v.u[k]), bw = __fmul_rn(b, v.w[k]);
    const float c = __fadd_rn(__fadd_rn(v.det[k], au), bw);
    r.s[k] = kind == TVR_PARALLEL ? __fadd_rn(__fadd_rn(v.src[k], au), bw) : v.src[k];
    r.d[k] = __fsub_rn(c, r.s[k]);
    r.inv[k] = fabsf(r.d[k]) > 1e-30f ? __frcp_rn(r.d[k]) : 0.f;
    dd = __fadd_rn(dd, __fmul_rn(r.d[k], r.d[k]));
  }
  r.dn = __fsqrt_rn(dd);
}

// Length of ray r inside voxel (ix, iy, iz): the intersection of t in [0, 1]
// with the three slabs of the voxel's box, times |d|.
__device__ __forceinline__ float mf_len(const MfRay &r, int ix, int iy, int iz, float half) {
  const int id[3] = {ix, iy, iz};
  float te = 0.f, tx = 1.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float lo = __fsub_rn((float)id[k], half);
    if (r.inv[k] != 0.f) {
      const float t0 = __fmul_rn(__fsub_rn(lo, r.s[k]), r.inv[k]);
      const float t1 = __fmul_rn(__fsub_rn(__fadd_rn(lo, 1.f), r.s[k]), r.inv[k]);
      te = fmaxf(te, fminf(t0, t1));
      tx = fminf(tx, fmaxf(t0, t1));
    } else if (!(r.s[k] > -half && r.s[k] >= lo && r.s[k] < __fadd_rn(lo, 1.f))) {
      return 0.f;
    }
  }
  return tx > te ? __fmul_rn(__fsub_rn(tx, te), r.dn) : 0.f;
}

// One axis of mf_len: for the voxel coordinate c on an axis with ray start s
// and 1/d = inv, the pair (min, max) of the parameters where the ray crosses
// the voxel's two planes (inv != 0), or whether the ray lies inside the slab
// (inv == 0).  mf_len's result is (min(1, max..) - max(0, min..)) |d| over the
// three axes; min and max are exact, so taking them axis by axis in any order
// gives the same float as mf_len.
__device__ __forceinline__ bool mf_axis(float s, float inv, int c, float half, float &lo_t,
                                        float &hi_t) {
  const float lo = __fsub_rn((float)c, half);
  if (inv != 0.f) {
    const float t0 = __fmul_rn(__fsub_rn(lo, s), inv);
    const float t1 = __fmul_rn(__fsub_rn(__fadd_rn(lo, 1.f), s), inv);
    lo_t = fminf(t0, t1);
    hi_t = fmaxf(t0, t1);
    return true;
  }
  lo_t = 0.f;
  hi_t = 1.f;
  return s > -half && s >= lo && s < __fadd_rn(lo, 1.f);
}

// Calls use(j, a_ij) for every voxel j with a_ij > 0 in the slabs
// k = k0 + lane, k0 + lane + G, ... of the ray's major axis.  Each length is
// mf_len's, evaluated factored: the major axis's crossing parameters once per
// slab, the other two axes' once per candidate cell.
template <int G, typename Use>
__device__ __forceinline__ void mf_row(const MfRay &r, int n, int lane, Use &&use) {
  const float half = mf_half(n);
  // parameter range inside the volume box (the forward walk only; mf_len
  // decides every entry)
  float te = 0.f, tx = 1.f;
  int ax = 0;
  float best = -1.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float ad = fabsf(r.d[k]);
    if (ad > best) {
      best = ad;
      ax = k;
    }
    if (r.inv[k] != 0.f) {
      const float t0 = __fmul_rn(__fsub_rn(-half, r.s[k]), r.inv[k]);
      const float t1 = __fmul_rn(__fsub_rn(half, r.s[k]), r.inv[k]);
      te = fmaxf(te, fminf(t0, t1));
      tx = fminf(tx, fmaxf(t0, t1));
    } else if (!(r.s[k] > -half && r.s[k] < half)) {
      return;
    }
  }
  // components along the major axis and the two others (selects, not
  // dynamic indexing, so the ray stays in registers)
  auto pick = [ax](const float v[3], int which) {
    // which = 0: major axis; 1: first other axis; 2: second other axis
    const int k = which == 0 ? ax : (which == 1 ? (ax == 0 ? 1 : 0) : (ax == 2 ? 1 : 2));
    return k == 0 ? v[0] : (k == 1 ? v[1] : v[2]);
  };
  const float sA = pick(r.s, 0), dA = pick(r.d, 0), iA = pick(r.inv, 0);
  const float s1 = pick(r.s, 1), d1 = pick(r.d, 1), i1v = pick(r.inv, 1);
  const float s2 = pick(r.s, 2), d2 = pick(r.d, 2), i2v = pick(r.inv, 2);
  if (!(tx > te) || iA == 0.f) return;
  // slab range of the major axis covered by [te, tx] (one slab of margin)
  const float ca = __fadd_rn(__fadd_rn(sA, __fmul_rn(te, dA)), half);
  const float cb = __fadd_rn(__fadd_rn(sA, __fmul_rn(tx, dA)), half);
  int k0 = (int)floorf(fminf(ca, cb)) - 1, k1 = (int)floorf(fmaxf(ca, cb)) + 1;
  k0 = k0 < 0 ? 0 : k0;
  k1 = k1 > n - 1 ? n - 1 : k1;
  constexpr float kMargin = 1e-3f;
  for (int k = k0 + lane; k <= k1; k += G) {
    // parameters of the slab's two planes (mf_len's pair for the major
    // axis), and the part of them inside the volume range
    float mA, MA;
    mf_axis(sA, iA, k, half, mA, MA);
    const float ta = fmaxf(te, mA), tb = fminf(tx, MA);
    if (!(tb >= ta)) continue;
    const float eA = fmaxf(0.f, mA), xA = fminf(1.f, MA);
    const float c10 = __fadd_rn(__fadd_rn(s1, __fmul_rn(ta, d1)), half);
    const float c11 = __fadd_rn(__fadd_rn(s1, __fmul_rn(tb, d1)), half);
    const float c20 = __fadd_rn(__fadd_rn(s2, __fmul_rn(ta, d2)), half);
    const float c21 = __fadd_rn(__fadd_rn(s2, __fmul_rn(tb, d2)), half);
    int lo1 = (int)floorf(fminf(c10, c11) - kMargin), hi1 = (int)floorf(fmaxf(c10, c11) + kMargin);
    int lo2 = (int)floorf(fminf(c20, c21) - kMargin), hi2 = (int)floorf(fmaxf(c20, c21) + kMargin);
    lo1 = lo1 < 0 ? 0 : lo1;
    lo2 = lo2 < 0 ? 0 : lo2;
    hi1 = hi1 > n - 1 ? n - 1 : hi1;
    hi2 = hi2 > n - 1 ? n - 1 : hi2;
    for (int i2 = lo2; i2 <= hi2; ++i2) {
      float m2, M2;
      if (!mf_axis(s2, i2v, i2, half, m2, M2)) continue;
      const float e2 = fmaxf(eA, m2), x2 = fminf(xA, M2);
      for (int i1 = lo1; i1 <= hi1; ++i1) {
        float m1, M1;
        if (!mf_axis(s1, i1v, i1, half, m1, M1)) continue;
        const float e = fmaxf(e2, m1), x = fminf(x2, M1);
        if (!(x > e)) continue;
        const float len = __fmul_rn(__fsub_rn(x, e), r.dn);  // = mf_len(r, voxel)
        if (!(len > 0.f)) continue;
        const int ix = ax == 0 ? k : i1;
        const int iy = ax == 1 ? k : (ax == 0 ? i1 : i2);
        const int iz = ax == 2 ? k : i2;
        use((int)(ix + n * (iy + n * iz)), len);
      }
    }
  }
}

// Calls use(i, a_ij) for every ray i with a_ij > 0 of the views
// v = lane, lane + G, ... for voxel (ix, iy, iz).
// The rays come from the per-ray table (mfr: 1/d and |d|; mfs: the start of a
// parallel-beam ray, a cone-beam ray starts at the view's source), which holds
// what mf_pixel_ray gives for each ray.
template <int G, typename Use>
__device__ __forceinline__ void mf_column(const MfView *__restrict__ views,
                                          const float4 *__restrict__ mfr,
                                          const float4 *__restrict__ mfs, int V, int kind, int Pu,
                                          int Pv, int n, int ix, int iy, int iz, int lane,
                                          Use &&use) {
  const float half = mf_half(n);
  constexpr float kMargin = 1e-3f;
  const float ca = 0.5f * (float)(Pu - 1), cb = 0.5f * (float)(Pv - 1);
  for (int vi = lane; vi < V; vi += G) {
    const MfView &v = views[vi];
    // pixel-coordinate box of the voxel's projection: the extremes of a
    // projective (cone) or linear (parallel) map over a box lie at corners
    float amin = 3.4e38f, amax = -3.4e38f, bmin = 3.4e38f, bmax = -3.4e38f;
    bool ok = true;
    const float X0[3] = {__fsub_rn((float)ix, half), __fsub_rn((float)iy, half),
                         __fsub_rn((float)iz, half)};
    if (kind == TVR_PARALLEL) {
      float ac = v.a0, bc = v.b0, ra = 0.f, rb = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float xc = __fadd_rn(X0[k], 0.5f);
        ac = __fmaf_rn(v.ga[k], xc, ac);
        bc = __fmaf_rn(v.gb[k], xc, bc);
        ra = __fmaf_rn(0.5f, fabsf(v.ga[k]), ra);
        rb = __fmaf_rn(0.5f, fabsf(v.gb[k]), rb);
      }
      amin = ac - ra;
      amax = ac + ra;
      bmin = bc - rb;
      bmax = bc + rb;
    } else {
      // numerators and denominator at the lower corner, then per corner the
      // sums of the components its offset adds
      float na = 0.f, nb = 0.f, nd = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float e = __fsub_rn(X0[k], v.src[k]);
        na = __fmaf_rn(e, v.uu[k], na);
        nb = __fmaf_rn(e, v.ww[k], nb);
        nd = __fmaf_rn(e, v.nrm[k], nd);
      }
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        float ca_ = na, cb_ = nb, cd = nd;
#pragma unroll
        for (int k = 0; k < 3; ++k)
          if ((c >> k) & 1) {
            ca_ = __fadd_rn(ca_, v.uu[k]);
            cb_ = __fadd_rn(cb_, v.ww[k]);
            cd = __fadd_rn(cd, v.nrm[k]);
          }
        ok = ok && cd > 0.f;  // a corner at or behind the source plane: use the whole detector
        const float s = __fmul_rn(v.dn, mf_rcp_approx(cd));
        const float a = __fmaf_rn(s, ca_, v.a0), b = __fmaf_rn(s, cb_, v.b0);
        amin = fminf(amin, a);
        amax = fmaxf(amax, a);
        bmin = fminf(bmin, b);
        bmax = fmaxf(bmax, b);
      }
    }
    int p0 = 0, p1 = Pu - 1, q0 = 0, q1 = Pv - 1;  // whole detector unless the box is sound
    const float lim = 1e7f;
    if (ok && fabsf(amin) < lim && fabsf(amax) < lim && fabsf(bmin) < lim && fabsf(bmax) < lim) {
      p0 = (int)ceilf(__fadd_rn(amin, ca) - kMargin);
      p1 = (int)floorf(__fadd_rn(amax, ca) + kMargin);
      q0 = (int)ceilf(__fadd_rn(bmin, cb) - kMargin);
      q1 = (int)floorf(__fadd_rn(bmax, cb) + kMargin);
      p0 = p0 < 0 ? 0 : p0;
      q0 = q0 < 0 ? 0 : q0;
      p1 = p1 > Pu - 1 ? Pu - 1 : p1;
      q1 = q1 > Pv - 1 ? Pv - 1 : q1;
    }
    // Cone beam: every ray of the view starts at its source, so mf_len's
    // differences lo - s and (lo + 1) - s per axis are the same for all of
    // this voxel's pixels; formed once here, with the same operations, they
    // give the same floats as mf_len.
    float dlo[3], dhi[3];
    bool inside[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float lo = X0[k];
      dlo[k] = __fsub_rn(lo, v.src[k]);
      dhi[k] = __fsub_rn(__fadd_rn(lo, 1.f), v.src[k]);
      inside[k] = v.src[k] > -half && v.src[k] >= lo && v.src[k] < __fadd_rn(lo, 1.f);
    }
    // pixels in groups of 4 along a detector row: the entries first, then
    // the gathers of the group together
    for (int q = q0; q <= q1; ++q)
      for (int p = p0; p <= p1; p += 4) {
        const int64_t i0 = ((int64_t)vi * Pv + q) * Pu + p;
        float lv[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          lv[t] = 0.f;
          if (p + t <= p1) {
            const float4 rc = __ldg(mfr + i0 + t);
            if (kind == TVR_PARALLEL) {
              MfRay r;
              r.inv[0] = rc.x;
              r.inv[1] = rc.y;
              r.inv[2] = rc.z;
              r.dn = rc.w;
              const float4 st = __ldg(mfs + i0 + t);
              r.s[0] = st.x;
              r.s[1] = st.y;
              r.s[2] = st.z;
              lv[t] = mf_len(r, ix, iy, iz, half);
            } else {
              const float inv[3] = {rc.x, rc.y, rc.z};
              float te = 0.f, tx = 1.f;
              bool hit = true;
#pragma unroll
              for (int k = 0; k < 3; ++k) {
                if (inv[k] != 0.f) {
                  const float t0 = __fmul_rn(dlo[k], inv[k]), t1 = __fmul_rn(dhi[k], inv[k]);
                  te = fmaxf(te, fminf(t0, t1));
                  tx = fminf(tx, fmaxf(t0, t1));
                } else {
                  hit = hit && inside[k];
                }
              }
              lv[t] = hit && tx > te ? __fmul_rn(__fsub_rn(tx, te), rc.w) : 0.f;  // = mf_len
            }
          }
        }
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (lv[t] > 0.f) use(i0 + t, lv[t]);
      }
  }
}

// Back projection of one separable view (MfView::sep) into K voxels stacked
// along z at (ix, iy, iz0 .. iz0 + K - 1): acc[k] += sum over the view's rays
// i of a_ij r_i, j the k-th voxel (voxels at iz >= n are skipped).
//   Boxes: with uu and nrm free of z, a pixel's column coordinate a and the
//   depth scale s = dn / ((X - src) . nrm) of a point X depend on its x, y
//   alone, so the 4 x-y corners of the stack give the columns p0..p1 of all K
//   voxels; with ww along z, b = b0 + s (z - src_z) ww_z, whose extremes over
//   voxel k's 8 corners lie at the extreme s and the two z faces, gives its
//   rows q0_k..q1_k (the same 1e-3 pixel margin as mf_column).
//   Entries: the rays of a detector column share 1/d_x and 1/d_y, so the x
//   and y slabs give one parameter interval per column p for all K voxels;
//   each ray then narrows it by its z slab.  These are mf_len's operations in
//   its axis order (min and max are exact), so the entries are the same
//   floats as the forward projection's.  A column whose x-y interval is
//   already empty holds no entry of these voxels.
template <int K>
__device__ __forceinline__ void mf_column_sep(const MfView &v, const float4 *__restrict__ rays,
                                              int vi, int Pu, int Pv, int n, int ix, int iy,
                                              int iz0, const float *__restrict__ r,
                                              float (&acc)[K]) {
  const float half = mf_half(n);
  constexpr float kMargin = 1e-3f;
  const float lim = 1e7f;
  const float ca = 0.5f * (float)(Pu - 1), cb = 0.5f * (float)(Pv - 1);
  const float sx = v.src[0], sy = v.src[1], sz = v.src[2];
  const float xlo = __fsub_rn((float)ix, half), ylo = __fsub_rn((float)iy, half);
  const float dlx = __fsub_rn(xlo, sx), dhx = __fsub_rn(__fadd_rn(xlo, 1.f), sx);
  const float dly = __fsub_rn(ylo, sy), dhy = __fsub_rn(__fadd_rn(ylo, 1.f), sy);
  const bool inx = sx > -half && sx >= xlo && sx < __fadd_rn(xlo, 1.f);
  const bool iny = sy > -half && sy >= ylo && sy < __fadd_rn(ylo, 1.f);
  float amin = 3.4e38f, amax = -3.4e38f, smin = 3.4e38f, smax = -3.4e38f;
  bool ok = true;  // every corner in front of the source plane
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const float ex = (c & 1) ? dhx : dlx, ey = (c & 2) ? dhy : dly;
    const float na = __fmaf_rn(ey, v.uu[1], __fmul_rn(ex, v.uu[0]));
    const float nd = __fmaf_rn(ey, v.nrm[1], __fmul_rn(ex, v.nrm[0]));
    ok = ok && nd > 0.f;
    const float s = __fmul_rn(v.dn, mf_rcp_approx(nd));
    const float a = __fmaf_rn(s, na, v.a0);
    amin = fminf(amin, a);
    amax = fmaxf(amax, a);
    smin = fminf(smin, s);
    smax = fmaxf(smax, s);
  }
  int p0 = 0, p1 = Pu - 1;  // whole detector unless the box is sound
  if (ok && fabsf(amin) < lim && fabsf(amax) < lim) {
    p0 = max(0, (int)ceilf(__fadd_rn(amin, ca) - kMargin));
    p1 = min(Pu - 1, (int)floorf(__fadd_rn(amax, ca) + kMargin));
  }
  int q0[K], q1[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float zlo = __fsub_rn((float)(iz0 + k), half);
    const float nbl = __fmul_rn(__fsub_rn(zlo, sz), v.ww[2]);
    const float nbh = __fmul_rn(__fsub_rn(__fadd_rn(zlo, 1.f), sz), v.ww[2]);
    const float b1 = __fmaf_rn(smin, nbl, v.b0), b2 = __fmaf_rn(smax, nbl, v.b0);
    const float b3 = __fmaf_rn(smin, nbh, v.b0), b4 = __fmaf_rn(smax, nbh, v.b0);
    const float bmin = fminf(fminf(b1, b2), fminf(b3, b4));
    const float bmax = fmaxf(fmaxf(b1, b2), fmaxf(b3, b4));
    q0[k] = 0;
    q1[k] = iz0 + k < n ? Pv - 1 : -1;
    if (ok && fabsf(bmin) < lim && fabsf(bmax) < lim && iz0 + k < n) {
      q0[k] = max(0, (int)ceilf(__fadd_rn(bmin, cb) - kMargin));
      q1[k] = min(Pv - 1, (int)floorf(__fadd_rn(bmax, cb) + kMargin));
    }
  }
  const int64_t vbase = (int64_t)vi * Pv * Pu;
  for (int p = p0; p <= p1; ++p) {
    // row 0 of column p: its 1/d_x, 1/d_y are every row's
    const float2 ixy = __ldg(reinterpret_cast<const float2 *>(rays + vbase + p));
    float te = 0.f, tx = 1.f;
    bool hit = true;
    if (ixy.x != 0.f) {
      const float t0 = __fmul_rn(dlx, ixy.x), t1 = __fmul_rn(dhx, ixy.x);
      te = fmaxf(te, fminf(t0, t1));
      tx = fminf(tx, fmaxf(t0, t1));
    } else {
      hit = inx;
    }
    if (ixy.y != 0.f) {
      const float t0 = __fmul_rn(dly, ixy.y), t1 = __fmul_rn(dhy, ixy.y);
      te = fmaxf(te, fminf(t0, t1));
      tx = fminf(tx, fmaxf(t0, t1));
    } else {
      hit = hit && iny;
    }
    if (!(hit && tx > te)) continue;
    // row t of every voxel's row range: the K rays' constants and residuals
    // loaded together, then used (a residual whose ray misses goes unused)
    int nt = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) nt = max(nt, q1[k] - q0[k] + 1);
    for (int t = 0; t < nt; ++t) {
      float2 zw[K];
      float ri[K];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        zw[k] = make_float2(0.f, 0.f);
        ri[k] = 0.f;
        if (q0[k] + t <= q1[k]) {
          const int64_t i = vbase + (int64_t)(q0[k] + t) * Pu + p;
          zw[k] = __ldg(reinterpret_cast<const float2 *>(rays + i) + 1);  // 1/d_z, |d|
          ri[k] = __ldg(r + i);
        }
      }
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (q0[k] + t > q1[k]) continue;
        const float zlo = __fsub_rn((float)(iz0 + k), half);
        const float dlz = __fsub_rn(zlo, sz), dhz = __fsub_rn(__fadd_rn(zlo, 1.f), sz);
        float te2 = te, tx2 = tx;
        bool h = true;
        if (zw[k].x != 0.f) {
          const float t0 = __fmul_rn(dlz, zw[k].x), t1 = __fmul_rn(dhz, zw[k].x);
          te2 = fmaxf(te2, fminf(t0, t1));
          tx2 = fminf(tx2, fmaxf(t0, t1));
        } else {
          h = sz > -half && sz >= zlo && sz < __fadd_rn(zlo, 1.f);
        }
        if (h && tx2 > te2)
          acc[k] = __fmaf_rn(__fmul_rn(__fsub_rn(tx2, te2), zw[k].y), ri[k], acc[k]);  // = mf_len
      }
    }
  }
}

// Forward projection of K rays of one detector column of a separable view
// (MfView::sep): the rays share their start and, bit for bit, their 1/d_x
// and 1/d_y (and d_x, d_y up to rounding, which only the candidate ranges
// use), so their paths through the x-y grid are one path.  It is walked once
// for all K rays: the slabs kA = k0 + lane, k0 + lane + G, ... of the x-y
// major axis, the 1-3 cells of the other axis in each slab (a 1e-3 voxel
// margin, as mf_row), and per cell the parameter interval of its x and y
// slabs; each ray k then takes the z cells its z(t) passes within that
// interval and narrows it by their z slabs.  These are mf_len's operations
// (min and max are exact), so every length is the float mf_len gives.
// r0 is ray 0's geometry (start, d_x, d_y, 1/d_x, 1/d_y); izv, dzv, dnv hold
// each ray's 1/d_z, d_z and |d|; rays with ok[k] false are skipped.  Calls
// use(k, j, a_ij) for every voxel j with a_ij > 0 on ray k.
template <int G, int K, typename Use>
__device__ __forceinline__ void mf_row_sep(const MfRay &r0, const float (&izv)[K],
                                           const float (&dzv)[K], const float (&dnv)[K],
                                           const bool (&ok)[K], int n, int lane, Use &&use) {
  const float half = mf_half(n);
  constexpr float kMargin = 1e-3f;
  // parameter range inside the volume's x-y square (the walk only)
  float te = 0.f, tx = 1.f;
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    if (r0.inv[a] != 0.f) {
      const float t0 = __fmul_rn(__fsub_rn(-half, r0.s[a]), r0.inv[a]);
      const float t1 = __fmul_rn(__fsub_rn(half, r0.s[a]), r0.inv[a]);
      te = fmaxf(te, fminf(t0, t1));
      tx = fminf(tx, fmaxf(t0, t1));
    } else if (!(r0.s[a] > -half && r0.s[a] < half)) {
      return;
    }
  }
  const int ax = fabsf(r0.d[0]) >= fabsf(r0.d[1]) ? 0 : 1;  // x-y major axis
  const float sA = ax == 0 ? r0.s[0] : r0.s[1], dA = ax == 0 ? r0.d[0] : r0.d[1];
  const float iA = ax == 0 ? r0.inv[0] : r0.inv[1];
  const float sB = ax == 0 ? r0.s[1] : r0.s[0], dB = ax == 0 ? r0.d[1] : r0.d[0];
  const float iB = ax == 0 ? r0.inv[1] : r0.inv[0];
  const float sz = r0.s[2];
  // a separable view's rays all have d . nrm = dn > 0 with nrm in the x-y
  // plane, so d_x and d_y are never both 0
  if (!(tx > te) || iA == 0.f) return;
  const float ca = __fadd_rn(__fadd_rn(sA, __fmul_rn(te, dA)), half);
  const float cb = __fadd_rn(__fadd_rn(sA, __fmul_rn(tx, dA)), half);
  int k0 = (int)floorf(fminf(ca, cb)) - 1, k1 = (int)floorf(fmaxf(ca, cb)) + 1;
  k0 = k0 < 0 ? 0 : k0;
  k1 = k1 > n - 1 ? n - 1 : k1;
  for (int kA = k0 + lane; kA <= k1; kA += G) {
    float mA, MA;
    mf_axis(sA, iA, kA, half, mA, MA);
    const float ta = fmaxf(te, mA), tb = fminf(tx, MA);
    if (!(tb >= ta)) continue;
    const float eA = fmaxf(0.f, mA), xA = fminf(1.f, MA);
    const float c0 = __fadd_rn(__fadd_rn(sB, __fmul_rn(ta, dB)), half);
    const float c1 = __fadd_rn(__fadd_rn(sB, __fmul_rn(tb, dB)), half);
    int lo = (int)floorf(fminf(c0, c1) - kMargin), hi = (int)floorf(fmaxf(c0, c1) + kMargin);
    lo = lo < 0 ? 0 : lo;
    hi = hi > n - 1 ? n - 1 : hi;
    for (int kB = lo; kB <= hi; ++kB) {
      float mB, MB;
      if (!mf_axis(sB, iB, kB, half, mB, MB)) continue;
      const float e1 = fmaxf(eA, mB), x1 = fminf(xA, MB);
      if (!(x1 > e1)) continue;
      const int ix = ax == 0 ? kA : kB, iy = ax == 0 ? kB : kA;
      const int jxy = ix + n * iy;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (!ok[k]) continue;
        const float z0 = __fadd_rn(__fadd_rn(sz, __fmul_rn(e1, dzv[k])), half);
        const float z1 = __fadd_rn(__fadd_rn(sz, __fmul_rn(x1, dzv[k])), half);
        int lz = (int)floorf(fminf(z0, z1) - kMargin), hz = (int)floorf(fmaxf(z0, z1) + kMargin);
        lz = lz < 0 ? 0 : lz;
        hz = hz > n - 1 ? n - 1 : hz;
        for (int iz = lz; iz <= hz; ++iz) {
          float mz, Mz;
          if (!mf_axis(sz, izv[k], iz, half, mz, Mz)) continue;
          const float e = fmaxf(e1, mz), x = fminf(x1, Mz);
          if (!(x > e)) continue;
          const float len = __fmul_rn(__fsub_rn(x, e), dnv[k]);  // = mf_len(ray k, voxel)
          if (!(len > 0.f)) continue;
          use(k, jxy + n * n * iz, len);
        }
      }
    }
  }
}

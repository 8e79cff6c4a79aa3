// Construction of A (Siddon ray-voxel lengths) and of its transpose.
//
// One thread traces one ray in FP64.  Every FP64 product, sum, quotient and
// square root is written with an explicit round-to-nearest intrinsic, so the
// compiler cannot fuse or reorder them: the traversal is a fixed sequence of
// correctly rounded IEEE operations, and the index sets do not depend on the
// compiler's contraction choices.
//
// Traversal (Sec. II-A defines A only as the ray-sum operator; the entries
// are the lengths of ray i inside voxel j):
//   d = c - s for source s and pixel centre c; the ray is clipped to the box
//   [-n/2, n/2]^3 by t_min / t_max; the parameters of all grid planes strictly
//   between them are merged in increasing order with equal values once; each
//   consecutive pair (t_a, t_b) is one entry: voxel floor(s + (t_a+t_b)/2 d + n/2)
//   per axis (clamped to [0, n-1]), length (t_b - t_a) |d|, stored as float32.
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "mf.cuh"
#include "tvr_internal.cuh"

namespace {

struct ViewRec {
  double v[TVR_VIEW_FIELDS];
};

__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }

// Ray endpoints of pixel (p, q): centre c = (det + a u) + b w; for parallel
// beam the start s = (src + a u) + b w, else s = src.
__device__ __forceinline__ void endpoints(const double *vw, int kind, int Pu, int Pv, int p, int q,
                                          double s[3], double c[3]) {
  const double a = dsub((double)p, dmul(0.5, (double)(Pu - 1)));
  const double b = dsub((double)q, dmul(0.5, (double)(Pv - 1)));
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double au = dmul(a, vw[6 + k]);
    const double bw = dmul(b, vw[9 + k]);
    c[k] = dadd(dadd(vw[3 + k], au), bw);
    s[k] = kind == TVR_PARALLEL ? dadd(dadd(vw[k], au), bw) : vw[k];
  }
}

__device__ __forceinline__ double plane_param(int i, double half, double s, double d) {
  return ddiv(dsub(dsub((double)i, half), s), d);
}

// Returns the number of entries of the ray; writes them when cols != nullptr.
template <bool FILL>
__device__ int trace(const double s[3], const double c[3], int n, int32_t *cols, float *vals) {
  const double half = dmul(0.5, (double)n);
  double d[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) d[k] = dsub(c[k], s[k]);
  const double dnorm =
      __dsqrt_rn(dadd(dadd(dmul(d[0], d[0]), dmul(d[1], d[1])), dmul(d[2], d[2])));
  double tmin = 0.0, tmax = 1.0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (d[k] != 0.0) {
      const double t0 = ddiv(dsub(-half, s[k]), d[k]);
      const double t1 = ddiv(dsub(half, s[k]), d[k]);
      const double lo = t0 < t1 ? t0 : t1;
      const double hi = t0 < t1 ? t1 : t0;
      if (lo > tmin) tmin = lo;
      if (hi < tmax) tmax = hi;
    } else if (!(s[k] > -half && s[k] < half)) {
      return 0;
    }
  }
  if (!(tmax > tmin)) return 0;

  int idx[3] = {0, 0, 0}, dir[3] = {0, 0, 0};
  bool act[3] = {false, false, false};
  double tn[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (d[k] == 0.0) continue;
    dir[k] = d[k] > 0.0 ? 1 : -1;
    // first plane index at or before the entry point (only a starting guess:
    // the skip loop below decides exactly which planes lie beyond t_min)
    const int i0 = (int)floor(dadd(dadd(s[k], dmul(tmin, d[k])), half));
    int i = dir[k] > 0 ? i0 - 1 : i0 + 2;
    i = i < 0 ? 0 : (i > n ? n : i);
    idx[k] = i;
    act[k] = true;
    tn[k] = plane_param(i, half, s[k], d[k]);
    for (int guard = 0; act[k] && tn[k] <= tmin && guard <= n + 2; ++guard) {
      idx[k] += dir[k];
      if (idx[k] < 0 || idx[k] > n)
        act[k] = false;
      else
        tn[k] = plane_param(idx[k], half, s[k], d[k]);
    }
  }

  int cnt = 0;
  double cur = tmin;
  for (int it = 0; it < 3 * n + 4; ++it) {
    double nxt = tmax;
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (act[k] && tn[k] < nxt) nxt = tn[k];
    if (FILL) {
      const double mid = dmul(dadd(cur, nxt), 0.5);
      int v[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        int iv = (int)floor(dadd(dadd(s[k], dmul(mid, d[k])), half));
        v[k] = iv < 0 ? 0 : (iv > n - 1 ? n - 1 : iv);
      }
      cols[cnt] = (int32_t)(v[0] + n * (v[1] + n * v[2]));
      vals[cnt] = (float)dmul(dsub(nxt, cur), dnorm);
    }
    ++cnt;
    if (nxt >= tmax) break;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      for (int guard = 0; act[k] && tn[k] <= nxt && guard <= n + 2; ++guard) {
        idx[k] += dir[k];
        if (idx[k] < 0 || idx[k] > n)
          act[k] = false;
        else
          tn[k] = plane_param(idx[k], half, s[k], d[k]);
      }
    }
    cur = nxt;
  }
  return cnt;
}

__global__ void k_siddon_count(const ViewRec *__restrict__ views, int n, int Pu, int Pv, int kind,
                               int64_t m, int64_t *__restrict__ counts) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int64_t per = (int64_t)Pu * Pv;
  const int v = (int)(i / per);
  const int64_t rem = i - (int64_t)v * per;
  const int q = (int)(rem / Pu);
  const int p = (int)(rem - (int64_t)q * Pu);
  double s[3], c[3];
  endpoints(views[v].v, kind, Pu, Pv, p, q, s, c);
  counts[i] = trace<false>(s, c, n, nullptr, nullptr);
}

__global__ void k_siddon_fill(const ViewRec *__restrict__ views, int n, int Pu, int Pv, int kind,
                              int64_t m, const int64_t *__restrict__ row_ptr,
                              int32_t *__restrict__ cols, float *__restrict__ vals) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int64_t per = (int64_t)Pu * Pv;
  const int v = (int)(i / per);
  const int64_t rem = i - (int64_t)v * per;
  const int q = (int)(rem / Pu);
  const int p = (int)(rem - (int64_t)q * Pu);
  double s[3], c[3];
  endpoints(views[v].v, kind, Pu, Pv, p, q, s, c);
  const int64_t o = row_ptr[i];
  const int len = trace<true>(s, c, n, cols + o, vals + o);
  // padding up to the next multiple of 4: last real voxel, length 0
  const int64_t padded = row_ptr[i + 1] - o;
  for (int64_t k = len; k < padded; ++k) {
    cols[o + k] = len > 0 ? cols[o + len - 1] : 0;
    vals[o + k] = 0.f;
  }
}

// padded[i] = count rounded up to a multiple of 4; len[i] = count.
__global__ void k_pad4(const int64_t *__restrict__ cnt, int64_t n, int64_t *__restrict__ padded,
                       int32_t *__restrict__ len) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t c = cnt[i];
  padded[i] = (c + 3) & ~(int64_t)3;
  len[i] = (int32_t)c;
}

// ---- exclusive scan of int64 counts: out[0] = 0, out[i+1] = sum(in[0..i]) ----
constexpr int kScanItems = 4;
constexpr int kScanTile = TVR_BLOCK * kScanItems;

__device__ __forceinline__ int64_t block_exclusive(int64_t v, int64_t *total) {
  __shared__ int64_t sh[TVR_BLOCK / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t w = lane < TVR_BLOCK / 32 ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < TVR_BLOCK / 32) sh[lane] = w;
  }
  __syncthreads();
  const int64_t warp_off = warp > 0 ? sh[warp - 1] : 0;
  *total = sh[TVR_BLOCK / 32 - 1];
  __syncthreads();
  return warp_off + x - v;
}

__global__ void k_scan_tiles(const int64_t *__restrict__ in, int64_t n, int64_t *__restrict__ out,
                             int64_t *__restrict__ tile_sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems], local = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = base + k < n ? in[base + k] : 0;
    local += v[k];
  }
  int64_t total;
  int64_t run = block_exclusive(local, &total);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// Single block: exclusive scan of the tile sums in place; writes the grand total.
__global__ void k_scan_sums(int64_t *__restrict__ sums, int64_t tiles, int64_t *__restrict__ total_out) {
  int64_t carry = 0;
  for (int64_t b0 = 0; b0 < tiles; b0 += TVR_BLOCK) {
    const int64_t i = b0 + threadIdx.x;
    const int64_t v = i < tiles ? sums[i] : 0;
    int64_t tot;
    const int64_t ex = block_exclusive(v, &tot);
    if (i < tiles) sums[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) *total_out = carry;
}

__global__ void k_scan_add(int64_t *__restrict__ out, int64_t n, const int64_t *__restrict__ sums) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += sums[i / kScanTile];
}

// ---- transpose: stable LSD radix sort of the CSR entries by column ----
//
// The CSR entries are already in row order, so a stable sort by column gives
// the CSC order (rows ascending within a column) without any per-column sort.
// Each pass sorts by one 8-bit digit of the column.  Work unit: one warp walks
// kSubItems consecutive entries in chunks of 32; within a chunk,
// __match_any_sync groups lanes with equal digits and the rank of a lane is
// the number of lower lanes in its group, so the order inside a chunk, a
// warp's range and the whole array is kept.  Offsets come from an exclusive
// scan of the per-(digit, warp-range) counts in digit-major order.
constexpr int kSubItems = 8192;                 // entries per warp range
constexpr int kWarpsPerBlock = TVR_BLOCK / 32;  // 8

// Column counts of the real (non-padding) entries.
__global__ void k_col_hist(const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ row_len,
                           const int32_t *__restrict__ col, int64_t m, int64_t *__restrict__ cnt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int64_t o = row_ptr[i];
  for (int k = 0; k < row_len[i]; ++k)
    atomicAdd(reinterpret_cast<unsigned long long *>(cnt + col[o + k]), 1ull);
}

// Sort keys (the column; N for padding, so padding sorts last) and the row of
// every stored CSR entry.
__global__ void k_radix_keys(const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ row_len,
                             const int32_t *__restrict__ col, int64_t m, int32_t N,
                             int32_t *__restrict__ key, int32_t *__restrict__ row_of) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int64_t o = row_ptr[i], end = row_ptr[i + 1];
  const int len = row_len[i];
  for (int64_t e = o; e < end; ++e) {
    key[e] = e - o < len ? col[e] : N;
    row_of[e] = (int32_t)i;
  }
}

template <typename P>
__global__ void k_iota(P *__restrict__ out, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) out[i] = (P)i;
}

// hist[d * nsub + sub] = entries of warp range `sub` whose digit is d.
__global__ void k_radix_hist(const int32_t *__restrict__ key, int64_t n, int shift, int64_t nsub,
                             int64_t *__restrict__ hist) {
  __shared__ unsigned cnt[kWarpsPerBlock][256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int d = lane; d < 256; d += 32) cnt[w][d] = 0u;
  __syncwarp();
  const int64_t sub = (int64_t)blockIdx.x * kWarpsPerBlock + w;
  if (sub < nsub) {
    const int64_t base = sub * kSubItems;
    for (int c = 0; c < kSubItems; c += 32) {
      const int64_t i = base + c + lane;
      if (i < n) atomicAdd(&cnt[w][(key[i] >> shift) & 255], 1u);
    }
  }
  __syncwarp();
  if (sub < nsub)
    for (int d = lane; d < 256; d += 32) hist[(int64_t)d * nsub + sub] = cnt[w][d];
}

template <typename P>
__global__ void k_radix_scatter(const int32_t *__restrict__ key_in, const P *__restrict__ pay_in,
                                int64_t n, int shift, int64_t nsub,
                                const int64_t *__restrict__ offs, int32_t *__restrict__ key_out,
                                P *__restrict__ pay_out) {
  __shared__ int64_t run[kWarpsPerBlock][256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t sub = (int64_t)blockIdx.x * kWarpsPerBlock + w;
  for (int d = lane; d < 256; d += 32) run[w][d] = sub < nsub ? offs[(int64_t)d * nsub + sub] : 0;
  __syncwarp();
  if (sub >= nsub) return;  // whole warp leaves together
  const unsigned lower = (1u << lane) - 1u;
  const int64_t base = sub * kSubItems;
  for (int c = 0; c < kSubItems; c += 32) {
    const int64_t i = base + c + lane;
    const bool ok = i < n;
    const int32_t k = ok ? key_in[i] : 0;
    const int d = ok ? (k >> shift) & 255 : 256;  // 256: lanes past the end form their own group
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & lower);
    if (ok) {
      const int64_t pos = run[w][d] + rank;
      key_out[pos] = k;
      pay_out[pos] = pay_in[i];
    }
    __syncwarp();
    if (ok && rank == 0) run[w][d] += __popc(peers);
    __syncwarp();
  }
}

// Column c's entries (sorted positions [cu[c], cu[c+1])) to the padded CSC
// at cp[c], then padding: last real row, value 0.
template <typename P>
__global__ void k_csc_place(const int64_t *__restrict__ cu, const int64_t *__restrict__ cp,
                            const P *__restrict__ perm, const int32_t *__restrict__ row_of,
                            const float *__restrict__ val, int64_t N, int32_t *__restrict__ row,
                            float *__restrict__ cval) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  const int64_t u0 = cu[c], len = cu[c + 1] - u0, o = cp[c], padded = cp[c + 1] - o;
  for (int64_t k = 0; k < len; ++k) {
    const int64_t e = (int64_t)perm[u0 + k];
    row[o + k] = row_of[e];
    cval[o + k] = val[e];
  }
  for (int64_t k = len; k < padded; ++k) {
    row[o + k] = len > 0 ? row[o + len - 1] : 0;
    cval[o + k] = 0.f;
  }
}

}  // namespace

// Exclusive scan: out has n+1 entries; out[n] = total.  tmp: >= tiles + 1 int64.
cudaError_t scan_exclusive_i64(const int64_t *in, int64_t n, int64_t *out, int64_t *tmp,
                               cudaStream_t s) {
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles > 0) {
    k_scan_tiles<<<(unsigned)tiles, TVR_BLOCK, 0, s>>>(in, n, out, tmp);
    k_scan_sums<<<1, TVR_BLOCK, 0, s>>>(tmp, tiles, out + n);
    k_scan_add<<<(unsigned)((n + TVR_BLOCK - 1) / TVR_BLOCK), TVR_BLOCK, 0, s>>>(out, n, tmp);
  } else {
    cudaMemsetAsync(out, 0, sizeof(int64_t), s);
  }
  return cudaGetLastError();
}

int64_t scan_tmp_len(int64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

namespace {

struct Scratch {
  std::vector<void *> ptrs;
  ~Scratch() {
    for (void *p : ptrs) cudaFree(p);
  }
  template <typename T>
  cudaError_t get(T **out, int64_t count) {
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, sizeof(T) * (size_t)(count > 0 ? count : 1));
    if (e == cudaSuccess) ptrs.push_back(p);
    *out = static_cast<T *>(p);
    return e;
  }
};

#define BM_TRY(call)                        \
  do {                                      \
    cudaError_t e_ = (call);                \
    if (e_ != cudaSuccess) return e_;       \
  } while (0)

template <typename T>
cudaError_t owned(T **out, int64_t count) {
  return cudaMalloc(reinterpret_cast<void **>(out), sizeof(T) * (size_t)(count > 0 ? count : 1));
}

unsigned blocks_for(int64_t n) { return (unsigned)((n + TVR_BLOCK - 1) / TVR_BLOCK); }

// Stable radix sort of the padded CSR entries by column (padding last); then
// placement into the padded CSC.
template <typename P>
cudaError_t transpose(MatStore &A, cudaStream_t s) {
  Scratch t;
  const int64_t n = A.nnz_pad, N = A.N, m = A.m;
  const int64_t nsub = (n + kSubItems - 1) / kSubItems;
  const int64_t nh = 256 * nsub;
  int32_t *row_of, *k0, *k1;
  P *p0, *p1;
  int64_t *hist, *offs, *stmp, *cu, *cnt;
  BM_TRY(t.get(&row_of, n));
  BM_TRY(t.get(&k0, n));
  BM_TRY(t.get(&k1, n));
  BM_TRY(t.get(&p0, n));
  BM_TRY(t.get(&p1, n));
  BM_TRY(t.get(&hist, nh));
  BM_TRY(t.get(&offs, nh + 1));
  BM_TRY(t.get(&stmp, scan_tmp_len(nh > N ? nh : N)));
  BM_TRY(t.get(&cu, N + 1));
  BM_TRY(t.get(&cnt, N));
  // unpadded column offsets (positions of each column in the sorted order)
  BM_TRY(cudaMemsetAsync(cnt, 0, sizeof(int64_t) * N, s));
  k_col_hist<<<blocks_for(m), TVR_BLOCK, 0, s>>>(A.row_ptr, A.row_len, A.col, m, cnt);
  BM_TRY(scan_exclusive_i64(cnt, N, cu, stmp, s));
  k_radix_keys<<<blocks_for(m), TVR_BLOCK, 0, s>>>(A.row_ptr, A.row_len, A.col, m, (int32_t)N, k0,
                                                    row_of);
  k_iota<P><<<1216, TVR_BLOCK, 0, s>>>(p0, n);
  int bits = 1;
  while (bits < 31 && ((int64_t)1 << bits) <= N) ++bits;  // keys 0..N
  const unsigned blocks = (unsigned)((nsub + kWarpsPerBlock - 1) / kWarpsPerBlock);
  for (int shift = 0; shift < bits; shift += 8) {
    k_radix_hist<<<blocks, TVR_BLOCK, 0, s>>>(k0, n, shift, nsub, hist);
    BM_TRY(scan_exclusive_i64(hist, nh, offs, stmp, s));
    k_radix_scatter<P><<<blocks, TVR_BLOCK, 0, s>>>(k0, p0, n, shift, nsub, offs, k1, p1);
    int32_t *tk = k0; k0 = k1; k1 = tk;
    P *tp = p0; p0 = p1; p1 = tp;
  }
  k_csc_place<P><<<blocks_for(N), TVR_BLOCK, 0, s>>>(cu, A.col_ptr, p0, row_of, A.val, N, A.row,
                                                      A.cval);
  BM_TRY(cudaGetLastError());
  return cudaStreamSynchronize(s);  // scratch is freed on return
}

}  // namespace

void free_matrix(MatStore &A) {
  void *ptrs[] = {A.row_ptr, A.col_ptr, A.row_len, A.col_len, A.col,   A.row,
                  A.val,     A.cval,    A.qval,    A.qcval,   A.rscale, A.mfv,
                  A.mfr,     A.mfs,     A.mfz,     A.mfy};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  A = MatStore{};
}

// A for one scan: Siddon counts -> rows padded to multiples of 4 -> fill ->
// padded CSC.  Synchronises `s` (sizes are read back twice).  On failure the
// partially built arrays stay in A for free_matrix.
cudaError_t build_matrix(const double *views_dev, int n, int Pu, int Pv, int kind, int64_t m,
                         int64_t N, MatStore &A, cudaStream_t s) {
  A = MatStore{};
  A.m = m;
  A.N = N;
  Scratch t;
  int64_t *counts, *padded, *tmp, *rp_real, *ccnt, *cpad;
  BM_TRY(t.get(&counts, m));
  BM_TRY(t.get(&padded, m > N ? m : N));
  BM_TRY(t.get(&tmp, scan_tmp_len(m > N ? m : N)));
  BM_TRY(t.get(&rp_real, m + 1));
  BM_TRY(owned(&A.row_ptr, m + 1));
  BM_TRY(owned(&A.row_len, m));
  const unsigned rays = (unsigned)((m + 127) / 128);
  k_siddon_count<<<rays, 128, 0, s>>>(reinterpret_cast<const ViewRec *>(views_dev), n, Pu, Pv,
                                      kind, m, counts);
  k_pad4<<<blocks_for(m), TVR_BLOCK, 0, s>>>(counts, m, padded, A.row_len);
  BM_TRY(scan_exclusive_i64(padded, m, A.row_ptr, tmp, s));
  BM_TRY(scan_exclusive_i64(counts, m, rp_real, tmp, s));
  BM_TRY(cudaMemcpyAsync(&A.nnz_pad, A.row_ptr + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  BM_TRY(cudaMemcpyAsync(&A.nnz, rp_real + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  BM_TRY(cudaStreamSynchronize(s));
  BM_TRY(owned(&A.col, A.nnz_pad));
  BM_TRY(owned(&A.val, A.nnz_pad));
  k_siddon_fill<<<rays, 128, 0, s>>>(reinterpret_cast<const ViewRec *>(views_dev), n, Pu, Pv, kind,
                                     m, A.row_ptr, A.col, A.val);
  // column counts -> padded column pointers
  BM_TRY(t.get(&ccnt, N));
  BM_TRY(t.get(&cpad, N));
  BM_TRY(owned(&A.col_ptr, N + 1));
  BM_TRY(owned(&A.col_len, N));
  BM_TRY(cudaMemsetAsync(ccnt, 0, sizeof(int64_t) * N, s));
  k_col_hist<<<blocks_for(m), TVR_BLOCK, 0, s>>>(A.row_ptr, A.row_len, A.col, m, ccnt);
  k_pad4<<<blocks_for(N), TVR_BLOCK, 0, s>>>(ccnt, N, cpad, A.col_len);
  BM_TRY(scan_exclusive_i64(cpad, N, A.col_ptr, tmp, s));
  BM_TRY(cudaMemcpyAsync(&A.nnz_cpad, A.col_ptr + N, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  BM_TRY(cudaStreamSynchronize(s));
  BM_TRY(owned(&A.row, A.nnz_cpad));
  BM_TRY(owned(&A.cval, A.nnz_cpad));
  BM_TRY(cudaGetLastError());
  if (A.nnz_pad == 0) return cudaStreamSynchronize(s);
  if (A.nnz_pad >= ((int64_t)1 << 31)) return transpose<int64_t>(A, s);
  return transpose<int32_t>(A, s);
}

// ---- matrix-free storage: float32 view constants ----
namespace {

// One thread per view: the FP64 record rounded to float32, the detector
// normal (oriented away from the source) and the dual basis of (u, w) in the
// detector plane, all formed in FP64 with explicit rounding.
__global__ void k_mf_views(const ViewRec *__restrict__ views, int V, int kind,
                           MfView *__restrict__ out) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  const double *r = views[v].v;
  const double *src = r, *det = r + 3, *u = r + 6, *w = r + 9;
  double nr[3] = {dsub(dmul(u[1], w[2]), dmul(u[2], w[1])), dsub(dmul(u[2], w[0]), dmul(u[0], w[2])),
                  dsub(dmul(u[0], w[1]), dmul(u[1], w[0]))};
  const double nn = __dsqrt_rn(dadd(dadd(dmul(nr[0], nr[0]), dmul(nr[1], nr[1])), dmul(nr[2], nr[2])));
  double dn = 0.0;
  for (int k = 0; k < 3; ++k) {
    nr[k] = nn > 0.0 ? ddiv(nr[k], nn) : 0.0;
    dn = dadd(dn, dmul(dsub(det[k], src[k]), nr[k]));
  }
  if (dn < 0.0) {
    for (int k = 0; k < 3; ++k) nr[k] = -nr[k];
    dn = -dn;
  }
  const double guu = dadd(dadd(dmul(u[0], u[0]), dmul(u[1], u[1])), dmul(u[2], u[2]));
  const double gww = dadd(dadd(dmul(w[0], w[0]), dmul(w[1], w[1])), dmul(w[2], w[2]));
  const double guw = dadd(dadd(dmul(u[0], w[0]), dmul(u[1], w[1])), dmul(u[2], w[2]));
  const double g = dsub(dmul(guu, gww), dmul(guw, guw));
  MfView o;
  for (int k = 0; k < 3; ++k) {
    o.src[k] = (float)src[k];
    o.det[k] = (float)det[k];
    o.u[k] = (float)u[k];
    o.w[k] = (float)w[k];
    o.nrm[k] = (float)nr[k];
    o.uu[k] = g > 0.0 ? (float)ddiv(dsub(dmul(gww, u[k]), dmul(guw, w[k])), g) : 0.f;
    o.ww[k] = g > 0.0 ? (float)ddiv(dsub(dmul(guu, w[k]), dmul(guw, u[k])), g) : 0.f;
  }
  o.dn = (float)dn;
  // projection constants (see MfView): cone a0 = (src - det) . uu; parallel
  // ga = uu - nrm (dir . uu) / (dir . nrm) with dir = det - src, a0 = -det . ga
  double uu[3], ww[3], dir[3];
  for (int k = 0; k < 3; ++k) {
    uu[k] = g > 0.0 ? ddiv(dsub(dmul(gww, u[k]), dmul(guw, w[k])), g) : 0.0;
    ww[k] = g > 0.0 ? ddiv(dsub(dmul(guu, w[k]), dmul(guw, u[k])), g) : 0.0;
    dir[k] = dsub(det[k], src[k]);
  }
  double du = 0.0, dw = 0.0, dd = 0.0, a0 = 0.0, b0 = 0.0;
  for (int k = 0; k < 3; ++k) {
    du = dadd(du, dmul(dir[k], uu[k]));
    dw = dadd(dw, dmul(dir[k], ww[k]));
    dd = dadd(dd, dmul(dir[k], nr[k]));
  }
  double ga[3], gb[3];
  for (int k = 0; k < 3; ++k) {
    ga[k] = dd != 0.0 ? dsub(uu[k], ddiv(dmul(nr[k], du), dd)) : 0.0;
    gb[k] = dd != 0.0 ? dsub(ww[k], ddiv(dmul(nr[k], dw), dd)) : 0.0;
  }
  if (kind == TVR_PARALLEL) {
    for (int k = 0; k < 3; ++k) {
      a0 = dsub(a0, dmul(det[k], ga[k]));
      b0 = dsub(b0, dmul(det[k], gb[k]));
    }
  } else {
    for (int k = 0; k < 3; ++k) {
      a0 = dadd(a0, dmul(dsub(src[k], det[k]), uu[k]));
      b0 = dadd(b0, dmul(dsub(src[k], det[k]), ww[k]));
    }
  }
  o.a0 = (float)a0;
  o.b0 = (float)b0;
  for (int k = 0; k < 3; ++k) {
    o.ga[k] = (float)ga[k];
    o.gb[k] = (float)gb[k];
  }
  // separable view (cleared by k_mf_sep where the ray table disagrees)
  o.sep = kind != TVR_PARALLEL && o.uu[2] == 0.f && o.nrm[2] == 0.f && o.ww[0] == 0.f &&
          o.ww[1] == 0.f;
  for (int k = 0; k < 6; ++k) o.pad[k] = 0.f;
  out[v] = o;
}

// One thread per ray: the constants mf_len reads, from the same mf_pixel_ray
// the forward projection evaluates per ray, so both directions apply
// bit-identical entries.
__global__ void k_mf_rays(const MfView *__restrict__ views, int kind, int Pu, int Pv, int64_t m,
                          float4 *__restrict__ rays, float4 *__restrict__ starts) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int64_t per = (int64_t)Pu * Pv;
  const int vi = (int)(i / per);
  const int64_t rem = i - (int64_t)vi * per;
  const int q = (int)(rem / Pu), p = (int)(rem - (int64_t)q * Pu);
  MfRay r;
  mf_pixel_ray(views[vi], kind, Pu, Pv, p, q, r);
  rays[i] = make_float4(r.inv[0], r.inv[1], r.inv[2], r.dn);
  if (starts) starts[i] = make_float4(r.s[0], r.s[1], r.s[2], 0.f);
}

// One thread per ray of rows q > 0: clears the view's sep flag where the ray's
// 1/d_x or 1/d_y differs, bit for bit, from that of row 0 of its column.
__global__ void k_mf_sep(const float4 *__restrict__ rays, int Pu, int Pv, int64_t m,
                         MfView *__restrict__ views) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int64_t per = (int64_t)Pu * Pv;
  const int vi = (int)(i / per);
  const int64_t rem = i - (int64_t)vi * per;
  const int q = (int)(rem / Pu), p = (int)(rem - (int64_t)q * Pu);
  if (q == 0) return;
  const float4 a = rays[i], c = rays[(int64_t)vi * per + p];
  if (__float_as_int(a.x) != __float_as_int(c.x) || __float_as_int(a.y) != __float_as_int(c.y))
    atomicAnd(&views[vi].sep, 0);
}

}  // namespace

// Matrix-free storage: the view constants and the per-ray table (16 bytes a
// ray, 32 for parallel beam: no matrix).  Synchronises `s`.
cudaError_t build_matrix_free(const double *views_dev, int n, int V, int Pu, int Pv, int kind,
                              int64_t m, int64_t N, MatStore &A, cudaStream_t s) {
  A = MatStore{};
  A.m = m;
  A.N = N;
  A.storage = TVR_STORAGE_MATRIX_FREE;
  A.V = V;
  A.Pu = Pu;
  A.Pv = Pv;
  A.kind = kind;
  (void)n;
  BM_TRY(owned(&A.mfv, V));
  k_mf_views<<<(V + 127) / 128, 128, 0, s>>>(reinterpret_cast<const ViewRec *>(views_dev), V,
                                              kind, A.mfv);
  BM_TRY(cudaGetLastError());
  BM_TRY(owned(&A.mfr, m > 0 ? m : 1));
  if (kind == TVR_PARALLEL) BM_TRY(owned(&A.mfs, m > 0 ? m : 1));
  if (m > 0)
    k_mf_rays<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(A.mfv, kind, Pu, Pv, m, A.mfr, A.mfs);
  BM_TRY(cudaGetLastError());
  if (m > 0 && kind != TVR_PARALLEL) {
    k_mf_sep<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(A.mfr, Pu, Pv, m, A.mfv);
    BM_TRY(cudaGetLastError());
  }
  // every view separable: the back projection runs per stack of voxels
  // (k_mf_adjoint_sep) into a buffer of N values, the forward projection per
  // stack of rays (k_mf_forward_sep) into one of 4 m row sums
  std::vector<MfView> hv((size_t)V);
  BM_TRY(cudaMemcpyAsync(hv.data(), A.mfv, sizeof(MfView) * V, cudaMemcpyDeviceToHost, s));
  BM_TRY(cudaStreamSynchronize(s));
  bool sep = m > 0;
  for (const MfView &v : hv) sep = sep && v.sep;
  if (sep) {
    BM_TRY(owned(&A.mfz, N));
    BM_TRY(owned(&A.mfy, 4 * m));
  }
  return cudaSuccess;
}

// ---- BF16 storage with per-row scale ----
namespace {

__global__ void k_row_scale(const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ row_len,
                            const float *__restrict__ val, int64_t m, float *__restrict__ sc) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  float mx = 0.f;
  for (int k = 0; k < row_len[i]; ++k) mx = fmaxf(mx, val[row_ptr[i] + k]);
  sc[i] = mx > 0.f ? mx : 1.f;
}

// q = bf16_rn(a / s_row) for real entries, 0 for padding.  Thread per row (CSR)
// or per column (CSC, row of each entry from `rows`).
__global__ void k_quantize(const int64_t *__restrict__ ptr, const int32_t *__restrict__ len,
                           const int32_t *__restrict__ rows, const float *__restrict__ val,
                           const float *__restrict__ sc, int64_t nseg,
                           __nv_bfloat16 *__restrict__ q) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nseg) return;
  const int64_t o = ptr[c], end = ptr[c + 1];
  for (int64_t e = o; e < end; ++e) {
    if (e - o < len[c]) {
      const float s = sc[rows ? rows[e] : c];
      q[e] = __float2bfloat16_rn(__fdiv_rn(val[e], s));
    } else {
      q[e] = __float2bfloat16_rn(0.f);
    }
  }
}

// 16-bit unsigned fixed point: the per-row step t = fl(s / 65535) replaces the
// row maximum s in sc, then q = min(65535, rint(a / t)) for real entries, 0
// for padding.  Thread per row (CSR) or per column (CSC, row from `rows`).
__global__ void k_row_step(float *__restrict__ sc, int64_t m) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) sc[i] = __fdiv_rn(sc[i], 65535.f);
}

__global__ void k_quantize_u16(const int64_t *__restrict__ ptr, const int32_t *__restrict__ len,
                               const int32_t *__restrict__ rows, const float *__restrict__ val,
                               const float *__restrict__ sc, int64_t nseg,
                               uint16_t *__restrict__ q) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nseg) return;
  const int64_t o = ptr[c], end = ptr[c + 1];
  for (int64_t e = o; e < end; ++e) {
    uint16_t code = 0;
    if (e - o < len[c]) {
      const unsigned u = __float2uint_rn(__fdiv_rn(val[e], sc[rows ? rows[e] : c]));
      code = (uint16_t)(u < 65535u ? u : 65535u);
    }
    q[e] = code;
  }
}

// Effective float32 values t_i * code of 16-bit codes (decode16's formats).
__global__ void k_effective(const int64_t *__restrict__ ptr, const int32_t *__restrict__ rows,
                            const __nv_bfloat16 *__restrict__ q, const float *__restrict__ sc,
                            int64_t nseg, int u16, float *__restrict__ out) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nseg) return;
  const uint16_t *q16 = reinterpret_cast<const uint16_t *>(q);
  for (int64_t e = ptr[c]; e < ptr[c + 1]; ++e) {
    const float code = u16 ? __uint2float_rn(q16[e]) : __bfloat162float(q[e]);
    out[e] = __fmul_rn(sc[rows ? rows[e] : c], code);
  }
}

}  // namespace

// Replace the FP32 values by per-row scales and BF16 codes (CSR and CSC get
// the same code for the same entry: the same quotient, rounded once).
cudaError_t quantize_bf16(MatStore &A, cudaStream_t s) {
  BM_TRY(owned(&A.rscale, A.m));
  BM_TRY(owned(&A.qval, A.nnz_pad));
  BM_TRY(owned(&A.qcval, A.nnz_cpad));
  k_row_scale<<<blocks_for(A.m), TVR_BLOCK, 0, s>>>(A.row_ptr, A.row_len, A.val, A.m, A.rscale);
  k_quantize<<<blocks_for(A.m), TVR_BLOCK, 0, s>>>(A.row_ptr, A.row_len, nullptr, A.val, A.rscale,
                                                   A.m, A.qval);
  k_quantize<<<blocks_for(A.N), TVR_BLOCK, 0, s>>>(A.col_ptr, A.col_len, A.row, A.cval, A.rscale,
                                                   A.N, A.qcval);
  BM_TRY(cudaGetLastError());
  BM_TRY(cudaStreamSynchronize(s));
  cudaFree(A.val);
  cudaFree(A.cval);
  A.val = A.cval = nullptr;
  A.storage = TVR_STORAGE_BF16_ROWSCALE;
  return cudaSuccess;
}

// Replace the FP32 values by per-row steps and 16-bit unsigned fixed-point
// codes (CSR and CSC get the same code for the same entry: the same quotient,
// rounded once).
cudaError_t quantize_u16(MatStore &A, cudaStream_t s) {
  BM_TRY(owned(&A.rscale, A.m));
  BM_TRY(owned(&A.qval, A.nnz_pad));
  BM_TRY(owned(&A.qcval, A.nnz_cpad));
  k_row_scale<<<blocks_for(A.m), TVR_BLOCK, 0, s>>>(A.row_ptr, A.row_len, A.val, A.m, A.rscale);
  k_row_step<<<blocks_for(A.m), TVR_BLOCK, 0, s>>>(A.rscale, A.m);
  k_quantize_u16<<<blocks_for(A.m), TVR_BLOCK, 0, s>>>(
      A.row_ptr, A.row_len, nullptr, A.val, A.rscale, A.m, reinterpret_cast<uint16_t *>(A.qval));
  k_quantize_u16<<<blocks_for(A.N), TVR_BLOCK, 0, s>>>(
      A.col_ptr, A.col_len, A.row, A.cval, A.rscale, A.N, reinterpret_cast<uint16_t *>(A.qcval));
  BM_TRY(cudaGetLastError());
  BM_TRY(cudaStreamSynchronize(s));
  cudaFree(A.val);
  cudaFree(A.cval);
  A.val = A.cval = nullptr;
  A.storage = TVR_STORAGE_U16_ROWSCALE;
  return cudaSuccess;
}

namespace {

// out[o + p] = in[o + lane_logical(p, L)] within every segment (row or column).
template <typename T>
__global__ void k_interleave(const int64_t *__restrict__ ptr, int64_t nseg,
                             const T *__restrict__ in, T *__restrict__ out) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nseg) return;
  const int64_t o = ptr[c], L = ptr[c + 1] - o;
  for (int64_t p = 0; p < L; ++p) out[o + p] = in[o + lane_logical(p, L)];
}

template <typename T>
cudaError_t interleave(const int64_t *ptr, int64_t nseg, int64_t stored, T *&arr, cudaStream_t s) {
  if (!arr) return cudaSuccess;
  T *out = nullptr;
  BM_TRY(owned(&out, stored));
  k_interleave<T><<<blocks_for(nseg), TVR_BLOCK, 0, s>>>(ptr, nseg, arr, out);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaFree(out);
    return e;
  }
  cudaFree(arr);
  arr = out;
  return cudaSuccess;
}

}  // namespace

// Final stored order (lane_logical) of every entry array, CSR and CSC; run
// after all per-entry processing that assumes the padding at the end.
cudaError_t interleave_lanes(MatStore &A, cudaStream_t s) {
  BM_TRY(interleave(A.row_ptr, A.m, A.nnz_pad, A.col, s));
  BM_TRY(interleave(A.row_ptr, A.m, A.nnz_pad, A.val, s));
  BM_TRY(interleave(A.row_ptr, A.m, A.nnz_pad, A.qval, s));
  BM_TRY(interleave(A.col_ptr, A.N, A.nnz_cpad, A.row, s));
  BM_TRY(interleave(A.col_ptr, A.N, A.nnz_cpad, A.cval, s));
  BM_TRY(interleave(A.col_ptr, A.N, A.nnz_cpad, A.qcval, s));
  return cudaSuccess;
}

// FP32 values the kernels apply, in stored (padded) order: CSR or CSC.
cudaError_t effective_values(const MatStore &A, bool csc, float *out, cudaStream_t s) {
  if (csc)
    k_effective<<<blocks_for(A.N), TVR_BLOCK, 0, s>>>(A.col_ptr, A.row, A.qcval, A.rscale, A.N,
                                                      A.storage == TVR_STORAGE_U16_ROWSCALE, out);
  else
    k_effective<<<blocks_for(A.m), TVR_BLOCK, 0, s>>>(A.row_ptr, nullptr, A.qval, A.rscale, A.m,
                                                      A.storage == TVR_STORAGE_U16_ROWSCALE, out);
  BM_TRY(cudaGetLastError());
  return cudaStreamSynchronize(s);
}

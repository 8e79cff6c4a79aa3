/*
 * ORACLE -- test infrastructure only.  Only tests/, __graft_entry__.smoke()
 * and bench.py's cpu_baseline / reference legs may load this library.  It
 * shares no code with the CUDA path.
 *
 * System matrix A of the TV-CT problem (Sec. II-A: A maps the voxel image to
 * ray sums; the paper does not say how A is built).  Entry a_ij is the length
 * of ray i inside voxel j, computed by Siddon's parametric ray-voxel
 * intersection in FP64:
 *
 *   ray point(t) = s + t (c - s), t in [0, 1], s = source, c = pixel centre;
 *   t_min / t_max clip the ray to the volume box [-n/2, n/2]^3;
 *   the crossing parameters of every x, y and z grid plane strictly inside
 *   (t_min, t_max) are merged with t_min and t_max into one increasing list,
 *   equal values counting once (no zero-length segments);
 *   each consecutive pair (t_a, t_b) is one segment: its voxel is
 *   floor(s + ((t_a + t_b) / 2) d + n/2) per axis, clamped to [0, n-1], and
 *   its length is (t_b - t_a) |d|.
 *
 * Entries of a row are stored in traversal order (increasing t).
 * Compile with -ffp-contract=off: every product and sum is rounded on its own.
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <stdint.h>
#include <string.h>

#define VIEW_FIELDS 12

/* Pixel centre (and, for parallel beam, ray start) of pixel (p, q) of a view. */
static void ray_endpoints(const double *vw, int kind, int Pu, int Pv, int p, int q,
                          double s[3], double c[3]) {
  double a = (double)p - 0.5 * (double)(Pu - 1);
  double b = (double)q - 0.5 * (double)(Pv - 1);
  for (int k = 0; k < 3; ++k) {
    double au = a * vw[6 + k];
    double bw = b * vw[9 + k];
    c[k] = (vw[3 + k] + au) + bw;
    if (kind == 1)
      s[k] = (vw[0 + k] + au) + bw;
    else
      s[k] = vw[0 + k];
  }
}

/* Crossing parameter of plane number i (coordinate i - n/2) along axis k. */
static double plane_t(int i, double half, double s, double d) {
  double p = (double)i - half;
  return (p - s) / d;
}

/*
 * Trace one ray.  Writes up to 3n+3 (col, len) pairs when cols != NULL and
 * returns the number of segments.
 */
int64_t orc_trace_ray(const double s[3], const double c[3], int n, int32_t *cols,
                      double *vals) {
  const double half = 0.5 * (double)n;
  double d[3];
  for (int k = 0; k < 3; ++k) d[k] = c[k] - s[k];
  double dn2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
  double dnorm = sqrt(dn2);

  double tmin = 0.0, tmax = 1.0;
  for (int k = 0; k < 3; ++k) {
    if (d[k] != 0.0) {
      double t0 = (-half - s[k]) / d[k];
      double t1 = (half - s[k]) / d[k];
      double lo = t0 < t1 ? t0 : t1;
      double hi = t0 < t1 ? t1 : t0;
      if (lo > tmin) tmin = lo;
      if (hi < tmax) tmax = hi;
    } else if (!(s[k] > -half && s[k] < half)) {
      return 0;
    }
  }
  if (!(tmax > tmin)) return 0;

  /* per-axis cursor on the next plane crossing with t > current */
  int idx[3], dir[3], active[3];
  double tn[3];
  for (int k = 0; k < 3; ++k) {
    active[k] = 0;
    if (d[k] == 0.0) continue;
    dir[k] = d[k] > 0.0 ? 1 : -1;
    double e = (s[k] + tmin * d[k]) + half;
    int i0 = (int)floor(e);
    int i = dir[k] > 0 ? i0 - 1 : i0 + 2;
    if (i < 0) i = 0;
    if (i > n) i = n;
    idx[k] = i;
    active[k] = 1;
    tn[k] = plane_t(i, half, s[k], d[k]);
    while (active[k] && tn[k] <= tmin) {
      idx[k] += dir[k];
      if (idx[k] < 0 || idx[k] > n)
        active[k] = 0;
      else
        tn[k] = plane_t(idx[k], half, s[k], d[k]);
    }
  }

  int64_t cnt = 0;
  double cur = tmin;
  for (int guard = 0; guard < 3 * n + 4; ++guard) {
    double nxt = tmax;
    for (int k = 0; k < 3; ++k)
      if (active[k] && tn[k] < nxt) nxt = tn[k];
    if (cols) {
      double mid = (cur + nxt) * 0.5;
      int v[3];
      for (int k = 0; k < 3; ++k) {
        double coord = (s[k] + mid * d[k]) + half;
        int iv = (int)floor(coord);
        if (iv < 0) iv = 0;
        if (iv > n - 1) iv = n - 1;
        v[k] = iv;
      }
      cols[cnt] = (int32_t)(v[0] + n * (v[1] + n * v[2]));
      vals[cnt] = (nxt - cur) * dnorm;
    }
    ++cnt;
    if (nxt >= tmax) break;
    for (int k = 0; k < 3; ++k) {
      while (active[k] && tn[k] <= nxt) {
        idx[k] += dir[k];
        if (idx[k] < 0 || idx[k] > n)
          active[k] = 0;
        else
          tn[k] = plane_t(idx[k], half, s[k], d[k]);
      }
    }
    cur = nxt;
  }
  return cnt;
}

/* Row counts of the whole scan; returns nnz.  Row i = v*Pu*Pv + q*Pu + p. */
int64_t orc_siddon_count(int n, int V, int Pu, int Pv, int kind, const double *views,
                         int64_t *row_counts) {
  int64_t total = 0;
  for (int v = 0; v < V; ++v)
    for (int q = 0; q < Pv; ++q)
      for (int p = 0; p < Pu; ++p) {
        double s[3], c[3];
        ray_endpoints(views + (int64_t)v * VIEW_FIELDS, kind, Pu, Pv, p, q, s, c);
        int64_t k = orc_trace_ray(s, c, n, NULL, NULL);
        row_counts[((int64_t)v * Pv + q) * Pu + p] = k;
        total += k;
      }
  return total;
}

/* Fill CSR column indices and FP64 lengths given row_ptr (length m+1). */
void orc_siddon_fill(int n, int V, int Pu, int Pv, int kind, const double *views,
                     const int64_t *row_ptr, int32_t *cols, double *vals) {
  for (int v = 0; v < V; ++v)
    for (int q = 0; q < Pv; ++q)
      for (int p = 0; p < Pu; ++p) {
        double s[3], c[3];
        ray_endpoints(views + (int64_t)v * VIEW_FIELDS, kind, Pu, Pv, p, q, s, c);
        int64_t i = ((int64_t)v * Pv + q) * Pu + p;
        orc_trace_ray(s, c, n, cols + row_ptr[i], vals + row_ptr[i]);
      }
}

/* Matrix-free row: ray i of the scan, for volumes whose A does not fit in RAM. */
int64_t orc_siddon_row(int n, int Pu, int Pv, int kind, const double *views, int64_t i,
                       int32_t *cols, double *vals) {
  int64_t per_view = (int64_t)Pu * Pv;
  int v = (int)(i / per_view);
  int64_t rem = i - (int64_t)v * per_view;
  int q = (int)(rem / Pu);
  int p = (int)(rem - (int64_t)q * Pu);
  double s[3], c[3];
  ray_endpoints(views + (int64_t)v * VIEW_FIELDS, kind, Pu, Pv, p, q, s, c);
  return orc_trace_ray(s, c, n, cols, vals);
}

/* y = A x without storing A, for volumes whose A does not fit in RAM: each
   row's entries in traversal order, summed in FP64 (Sec. II-A: A x is the
   vector of ray sums of x).  Rays are independent; with OpenMP they are
   spread over threads, each row still summed in its own order. */
void orc_forward(int n, int V, int Pu, int Pv, int kind, const double *views, const double *x,
                 double *y) {
  const int64_t m = (int64_t)V * Pu * Pv;
#pragma omp parallel
  {
    int32_t *cols = (int32_t *)malloc(sizeof(int32_t) * (3 * (size_t)n + 4));
    double *vals = (double *)malloc(sizeof(double) * (3 * (size_t)n + 4));
#pragma omp for schedule(dynamic, 1024)
    for (int64_t i = 0; i < m; ++i) {
      const int64_t per = (int64_t)Pu * Pv;
      const int v = (int)(i / per);
      const int64_t rem = i - (int64_t)v * per;
      const int q = (int)(rem / Pu), p = (int)(rem - (int64_t)q * Pu);
      double s[3], c[3];
      ray_endpoints(views + (int64_t)v * VIEW_FIELDS, kind, Pu, Pv, p, q, s, c);
      const int64_t k = orc_trace_ray(s, c, n, cols, vals);
      double acc = 0.0;
      for (int64_t e = 0; e < k; ++e) acc += vals[e] * x[cols[e]];
      y[i] = acc;
    }
    free(cols);
    free(vals);
  }
}

/* z = A^T r without storing A: every ray i adds r_i a_ij to z_j for its
   entries, in FP64.  With OpenMP each thread accumulates the rays of its
   share into its own copy of z and the copies are added in thread order, so
   the rounding depends on the number of threads (not on scheduling). */
void orc_adjoint(int n, int V, int Pu, int Pv, int kind, const double *views, const double *r,
                 double *z) {
  const int64_t N = (int64_t)n * n * n;
  const int64_t m = (int64_t)V * Pu * Pv;
  for (int64_t j = 0; j < N; ++j) z[j] = 0.0;
  int nt = 1;
#ifdef _OPENMP
  nt = omp_get_max_threads();
#endif
  double **part = (double **)calloc((size_t)nt, sizeof(double *));
#pragma omp parallel num_threads(nt)
  {
    int t = 0;
#ifdef _OPENMP
    t = omp_get_thread_num();
#endif
    double *zt = (double *)calloc((size_t)N, sizeof(double));
    part[t] = zt;
    int32_t *cols = (int32_t *)malloc(sizeof(int32_t) * (3 * (size_t)n + 4));
    double *vals = (double *)malloc(sizeof(double) * (3 * (size_t)n + 4));
    /* static split: thread t takes one contiguous block of rays */
    const int64_t lo = m * t / nt, hi = m * (t + 1) / nt;
    for (int64_t i = lo; i < hi; ++i) {
      const int64_t per = (int64_t)Pu * Pv;
      const int v = (int)(i / per);
      const int64_t rem = i - (int64_t)v * per;
      const int q = (int)(rem / Pu), p = (int)(rem - (int64_t)q * Pu);
      double s[3], c[3];
      ray_endpoints(views + (int64_t)v * VIEW_FIELDS, kind, Pu, Pv, p, q, s, c);
      const int64_t k = orc_trace_ray(s, c, n, cols, vals);
      for (int64_t e = 0; e < k; ++e) zt[cols[e]] += vals[e] * r[i];
    }
    free(cols);
    free(vals);
  }
  for (int t = 0; t < nt; ++t) {
    for (int64_t j = 0; j < N; ++j) z[j] += part[t][j];
    free(part[t]);
  }
  free(part);
}

"""Pins of the oracle's system matrix A (Siddon ray lengths, Sec. II-A).

Each check comes from geometry, not from the tracer itself: chord lengths by
slab clipping, exact voxel paths of axis-aligned and diagonal rays, brute
force marching on a 4^3 grid, and reversal symmetry.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from conftest import small_geometry


def centre(i, n):
    return i - n / 2 + 0.5


def chord(s, c, n):
    """Length of segment [s, c] inside [-n/2, n/2]^3 (slab clipping)."""
    s = np.asarray(s, float)
    c = np.asarray(c, float)
    d = c - s
    lo, hi = 0.0, 1.0
    for k in range(3):
        if d[k] == 0:
            if not (-n / 2 < s[k] < n / 2):
                return 0.0
            continue
        a = (-n / 2 - s[k]) / d[k]
        b = (n / 2 - s[k]) / d[k]
        lo, hi = max(lo, min(a, b)), min(hi, max(a, b))
    return max(0.0, hi - lo) * float(np.linalg.norm(d))


@pytest.mark.parametrize("n", [1, 4, 7])
def test_axis_aligned_ray_through_centres(n):
    iy, iz = n // 2, max(0, n - 2)
    s = [-3.0 * n, centre(iy, n), centre(iz, n)]
    c = [3.0 * n, centre(iy, n), centre(iz, n)]
    cols, vals = oracle.trace_ray(s, c, n)
    assert list(cols) == [ix + n * iy + n * n * iz for ix in range(n)]
    assert np.allclose(vals, 1.0, rtol=0, atol=1e-13)
    # reversed direction: reversed order
    cols_r, vals_r = oracle.trace_ray(c, s, n)
    assert list(cols_r) == list(cols[::-1])
    assert np.allclose(vals_r, 1.0, rtol=0, atol=1e-13)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_axis_aligned_each_axis(axis):
    n = 5
    s = np.array([centre(1, n), centre(3, n), centre(2, n)])
    c = s.copy()
    s[axis] = -20.0
    c[axis] = 20.0
    cols, vals = oracle.trace_ray(s, c, n)
    idx = [1, 3, 2]
    expect = []
    for i in range(n):
        v = list(idx)
        v[axis] = i
        expect.append(v[0] + n * v[1] + n * n * v[2])
    assert list(cols) == expect
    assert np.allclose(vals, 1.0, rtol=0, atol=1e-14)


def test_diagonal_ray_through_edges_merges_ties():
    # passes exactly through the voxel edges (x and y planes crossed together)
    n = 6
    zc = centre(2, n)
    cols, vals = oracle.trace_ray([-n, -n, zc], [n, n, zc], n)
    assert list(cols) == [i + n * i + n * n * 2 for i in range(n)]
    assert np.allclose(vals, math.sqrt(2.0), rtol=0, atol=1e-13)
    assert np.all(vals > 0)


def test_space_diagonal_through_corners():
    n = 4
    cols, vals = oracle.trace_ray([-n, -n, -n], [n, n, n], n)
    assert list(cols) == [i * (1 + n + n * n) for i in range(n)]
    assert np.allclose(vals, math.sqrt(3.0), rtol=0, atol=1e-13)


def test_ray_missing_volume_is_empty():
    n = 4
    cols, _ = oracle.trace_ray([-10, 3.0, 0.1], [10, 3.0, 0.1], n)   # y outside
    assert cols.size == 0
    cols, _ = oracle.trace_ray([-10, 2.0, 0.1], [10, 2.0, 0.1], n)   # on the boundary plane
    assert cols.size == 0
    cols, _ = oracle.trace_ray([-10, -10, 0.1], [-9, -9, 0.1], n)    # segment ends before
    assert cols.size == 0


def test_random_ray_lengths_sum_to_chord():
    rng = np.random.default_rng(7)
    n = 9
    for _ in range(300):
        s = rng.normal(size=3) * 4 * n
        c = rng.normal(size=3) * 4 * n
        cols, vals = oracle.trace_ray(s, c, n)
        assert abs(vals.sum() - chord(s, c, n)) <= 1e-10 * max(1.0, chord(s, c, n))
        assert np.all(vals > 0)
        assert np.all((cols >= 0) & (cols < n ** 3))
        assert len(set(cols.tolist())) == cols.size   # each voxel once per ray


def test_reversal_symmetry():
    rng = np.random.default_rng(11)
    n = 6
    for _ in range(100):
        s = rng.normal(size=3) * 3 * n
        c = rng.normal(size=3) * 3 * n
        a_cols, a_vals = oracle.trace_ray(s, c, n)
        b_cols, b_vals = oracle.trace_ray(c, s, n)
        da = dict(zip(a_cols.tolist(), a_vals.tolist()))
        db = dict(zip(b_cols.tolist(), b_vals.tolist()))
        big_a = {k for k, v in da.items() if v > 1e-9}
        big_b = {k for k, v in db.items() if v > 1e-9}
        assert big_a == big_b
        for k in big_a:
            assert abs(da[k] - db[k]) < 1e-9


def test_brute_force_marching_4cubed():
    """Per-voxel lengths vs dense midpoint sampling of the segment."""
    rng = np.random.default_rng(3)
    n = 4
    M = 200000
    for _ in range(40):
        s = rng.uniform(-8, 8, size=3)
        c = rng.uniform(-8, 8, size=3)
        cols, vals = oracle.trace_ray(s, c, n)
        t = (np.arange(M) + 0.5) / M
        p = s[None, :] + t[:, None] * (c - s)[None, :] + n / 2
        inside = np.all((p > 0) & (p < n), axis=1)
        v = np.floor(p[inside]).astype(int)
        j = v[:, 0] + n * v[:, 1] + n * n * v[:, 2]
        seg = np.linalg.norm(c - s) / M
        brute = np.bincount(j, minlength=n ** 3) * seg
        got = np.zeros(n ** 3)
        np.add.at(got, cols, vals)
        assert np.max(np.abs(brute - got)) <= 3 * seg + 1e-12


def test_geometry_rows_match_chords():
    g = small_geometry(n=4, views=5, det=7)
    A = oracle.system_matrix(g)
    assert A.shape == (g.m, g.N)
    rs = np.asarray(A.sum(axis=1)).ravel()
    V, Pu, Pv = g.n_views, g.det_cols, g.det_rows
    i = 0
    for v in range(V):
        vw = g.views[v]
        for q in range(Pv):
            for p in range(Pu):
                cpix = vw[3:6] + (p - (Pu - 1) / 2) * vw[6:9] + (q - (Pv - 1) / 2) * vw[9:12]
                assert abs(rs[i] - chord(vw[0:3], cpix, g.n)) < 1e-9
                i += 1


def test_row_order_and_matrix_free_row_agree():
    cfg = synth.get_config("c8")
    g = cfg.geometry()
    A = oracle.system_matrix(g)
    for i in [0, 5, g.m // 2, g.m - 1]:
        cols, vals = oracle.row(g, i)
        lo, hi = A.indptr[i], A.indptr[i + 1]
        assert np.array_equal(A.indices[lo:hi], cols)
        assert np.array_equal(A.data[lo:hi], vals)


def test_adjoint_identity():
    g = small_geometry(n=5, views=6, det=8)
    A = oracle.system_matrix(g)
    rng = np.random.default_rng(0)
    x = rng.normal(size=g.N)
    y = rng.normal(size=g.m)
    lhs = float((A @ x) @ y)
    # explicit row loop for A^T y
    aty = np.zeros(g.N)
    for i in range(g.m):
        for k in range(A.indptr[i], A.indptr[i + 1]):
            aty[A.indices[k]] += A.data[k] * y[i]
    assert abs(lhs - float(x @ aty)) <= 1e-12 * (abs(lhs) + 1)
    assert np.allclose(A.T @ y, aty, rtol=1e-13, atol=1e-13)


def test_matrix_free_forward_and_adjoint_equal_the_stored_matrix():
    """The ray-by-ray A x and A^T r (for volumes whose A does not fit in RAM)
    agree with the stored FP64 matrix: same entries, same order per row."""
    import synth
    for g in [synth.get_config("c8").geometry(), synth.cone_geometry(7, 5, 11, 21.0, 14.0, det_rows=9),
              synth.parallel_geometry(6, np.array([[1, 0, 0], [0, 1, 0], [1, 1, 1]]), 9)]:
        A = oracle.system_matrix(g)
        rng = np.random.default_rng(4)
        x = rng.uniform(0, 1, g.N)
        r = rng.normal(size=g.m)
        y = oracle.forward(g, x)
        assert np.allclose(y, A @ x, rtol=1e-14, atol=1e-14 * np.abs(A @ x).max())
        z = oracle.adjoint(g, r)
        zr = A.T @ r
        assert np.allclose(z, zr, rtol=1e-13, atol=1e-13 * np.abs(zr).max())
        # adjoint identity of the two on their own
        assert abs(y @ r - x @ z) <= 1e-12 * abs(y @ r)


def test_sphere_directions_are_spread_evenly():
    """Unit vectors; equal-area bands in height; no two directions closer than
    a fraction of the spacing of an even covering (4 pi / count per point)."""
    import synth
    for count in (19, 55):
        d = synth.sphere_directions(count)
        assert d.shape == (count, 3)
        assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-14)
        assert np.allclose(np.sort(d[:, 2]), np.sort(1 - 2 * (np.arange(count) + 0.5) / count))
        cosang = np.clip(d @ d.T - 2 * np.eye(count), -1, 1)
        min_angle = np.arccos(cosang.max())
        assert min_angle > 0.5 * np.sqrt(4 * np.pi / count)
    g = synth.sphere_parallel_geometry(8, 19, 13)
    assert g.n_views == 19 and g.m == 19 * 13 * 13
    ax = np.random.default_rng(0).uniform(size=50)
    e = synth.noise_exact(ax, np.random.default_rng(1).normal(size=50), 0.01)
    assert abs(np.linalg.norm(e) / np.linalg.norm(ax) - 0.01) < 1e-15

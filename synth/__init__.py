"""Seeded synthetic inputs for the TV-regularised CT problem.

This module is shared by the FP64 oracle (``oracle/``) and by the CUDA path
(``paper_1105_4002_gb300``).  It produces *input data only*: scan geometry
records, ellipsoid phantoms and standard-normal noise draws.  It holds none of
the method's arithmetic (no projection, no TV, no objective), so neither side
depends on the other through it.

Stand-ins.  The paper's test image is the 3-D FORBILD head phantom on a 64^3
grid scanned in parallel beam (Sec. IV-A); that phantom is not available, so
the workloads use seeded random axis-aligned ellipsoids on a zero background,
scanned by a circular cone-beam geometry with the sizes of the five
configurations listed in ``CONFIGS``.

Conventions (shared by both sides; the paper leaves A undefined, Sec. II-A):
  * the volume is an n x n x n grid of unit voxels centred at the origin;
    voxel j = ix + n*iy + n*n*iz (x fastest);
  * view v of V sits at angle 2*pi*v/V (endpoint excluded); the source is at
    (Dso cos, Dso sin, 0), the detector centre at -Dod (cos, sin, 0), the
    detector column axis u = (-sin, cos, 0) and row axis w = (0, 0, 1), both
    scaled by the pixel pitch;
  * pixel (p, q) has centre det_centre + (p - (Pu-1)/2) u + (q - (Pv-1)/2) w
    and ray index i = v*Pu*Pv + q*Pu + p.
The trigonometric values are computed here, once, and passed to both sides as
data, so the oracle and the GPU never evaluate cos/sin separately.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Record layout of one view: 12 float64 values.
VIEW_FIELDS = 12  # src[3], det_centre[3], u[3], w[3]

KIND_CONE = 0
KIND_PARALLEL = 1


@dataclasses.dataclass
class Geometry:
    """A scan: grid edge n, detector Pu x Pv, V views of VIEW_FIELDS doubles."""

    n: int
    det_cols: int
    det_rows: int
    views: np.ndarray  # float64 [V, 12], C-contiguous
    kind: int = KIND_CONE

    @property
    def n_views(self) -> int:
        return int(self.views.shape[0])

    @property
    def m(self) -> int:
        return self.n_views * self.det_cols * self.det_rows

    @property
    def N(self) -> int:
        return self.n ** 3


def cone_geometry(n: int, n_views: int, det: int, dso: float, dod: float,
                  pitch: float = 1.0, det_rows: int | None = None) -> Geometry:
    """Circular cone-beam scan with ``n_views`` views uniform over 360 degrees."""
    rows = det if det_rows is None else det_rows
    v = np.arange(n_views, dtype=np.float64)
    ang = 2.0 * math.pi * v / n_views
    c, s = np.cos(ang), np.sin(ang)
    views = np.zeros((n_views, VIEW_FIELDS), dtype=np.float64)
    views[:, 0] = dso * c
    views[:, 1] = dso * s
    views[:, 3] = -dod * c
    views[:, 4] = -dod * s
    views[:, 6] = -s * pitch
    views[:, 7] = c * pitch
    views[:, 11] = pitch
    return Geometry(n=n, det_cols=det, det_rows=rows, views=np.ascontiguousarray(views))


def parallel_geometry(n: int, directions: np.ndarray, det: int, pitch: float = 1.0,
                      dist: float | None = None) -> Geometry:
    """Parallel-beam scan, one view per unit direction (rows of ``directions``).

    For ``KIND_PARALLEL`` the ``src`` field is the centre of the source plane;
    the ray of pixel (p, q) starts at src + (same pixel offset) and ends at the
    pixel centre, so all rays of a view share the direction.
    """
    d = np.asarray(directions, dtype=np.float64)
    d = d / np.linalg.norm(d, axis=1, keepdims=True)
    T = float(2 * n) if dist is None else float(dist)
    views = np.zeros((d.shape[0], VIEW_FIELDS), dtype=np.float64)
    for i, dv in enumerate(d):
        # detector axes orthogonal to the direction
        a = np.array([0.0, 0.0, 1.0]) if abs(dv[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
        u = np.cross(a, dv)
        u /= np.linalg.norm(u)
        w = np.cross(dv, u)
        views[i, 0:3] = -T * dv
        views[i, 3:6] = T * dv
        views[i, 6:9] = u * pitch
        views[i, 9:12] = w * pitch
    return Geometry(n=n, det_cols=det, det_rows=det, views=np.ascontiguousarray(views),
                    kind=KIND_PARALLEL)


def sphere_directions(count: int) -> np.ndarray:
    """``count`` unit vectors spread evenly over the unit sphere: the
    golden-angle spiral (heights uniform in (-1, 1) at the midpoints of
    ``count`` equal bands, azimuth advancing by pi (3 - sqrt 5) per point)."""
    k = np.arange(count, dtype=np.float64) + 0.5
    z = 1.0 - 2.0 * k / count
    phi = k * math.pi * (3.0 - math.sqrt(5.0))
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def sphere_parallel_geometry(n: int, views: int, det: int) -> Geometry:
    """Parallel-beam scan with view directions spread evenly over the unit
    sphere, det^2 pixels of unit pitch (det = 91 covers the diagonal of a 64^3
    volume)."""
    return parallel_geometry(n, sphere_directions(views), det)


def noise_exact(ax: np.ndarray, z: np.ndarray, level: float) -> np.ndarray:
    """Noise e = level * ||ax|| * z / ||z||, so that ||e|| / ||ax|| = level exactly."""
    return level * float(np.linalg.norm(ax)) * z / float(np.linalg.norm(z))


def ellipsoid_phantom(n: int, count: int, semi_axes: tuple[float, float],
                      values: tuple[float, float], seed: int) -> np.ndarray:
    """Piecewise-constant phantom of ``count`` axis-aligned ellipsoids.

    Centres are uniform in the inner 60% of the volume, semi-axes uniform in
    ``semi_axes`` (voxels), values uniform in ``values``; a voxel belongs to an
    ellipsoid iff its centre satisfies sum(((c - c0) / a)^2) <= 1, and later
    ellipsoids overwrite earlier ones.  Returns float64 [n^3] in voxel order.
    """
    rng = np.random.default_rng(seed)
    h = 0.5 * n
    coords = np.arange(n, dtype=np.float64) - h + 0.5
    z, y, x = np.meshgrid(coords, coords, coords, indexing="ij")
    img = np.zeros((n, n, n), dtype=np.float64)
    for _ in range(count):
        c0 = rng.uniform(-0.3 * n, 0.3 * n, size=3)
        ax = rng.uniform(semi_axes[0], semi_axes[1], size=3)
        val = rng.uniform(values[0], values[1])
        inside = (((x - c0[0]) / ax[0]) ** 2 + ((y - c0[1]) / ax[1]) ** 2
                  + ((z - c0[2]) / ax[2]) ** 2) <= 1.0
        img[inside] = val
    return img.reshape(-1)


def standard_normal(size: int, seed: int) -> np.ndarray:
    """Seeded N(0, 1) draws (float64) used as the noise direction of b."""
    return np.random.default_rng(seed).standard_normal(size)


def uniform(size: int, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """Seeded U[lo, hi) draws (float64) for generic test vectors."""
    return np.random.default_rng(seed).uniform(lo, hi, size)


@dataclasses.dataclass
class Config:
    name: str
    n: int
    views: int
    det: int
    dso: float
    dod: float
    ellipsoids: int
    semi_axes: tuple[float, float]
    values: tuple[float, float]
    noise: float
    alpha: float
    tau: float
    eps: float
    seed: int

    def geometry(self) -> Geometry:
        return cone_geometry(self.n, self.views, self.det, self.dso, self.dod)

    def phantom(self) -> np.ndarray:
        return ellipsoid_phantom(self.n, self.ellipsoids, self.semi_axes, self.values,
                                 self.seed)

    def noise_direction(self) -> np.ndarray:
        g = self.geometry()
        return standard_normal(g.m, self.seed + 1000)


# Workload presets.  Distances for sizes the scan spec leaves open follow the
# 3n / 2n source/detector ratio of the 32^3 and 64^3 scans.
CONFIGS: dict[str, Config] = {
    # 32^3, 12 views, 48^2 detector: GPBB to relative gradient-map norm 1e-4.
    "c32": Config("c32", 32, 12, 48, 96.0, 64.0, 5, (3.0, 10.0), (0.2, 1.0), 0.01,
                  1e-2, 1e-4, 1e-4, 1),
    # 64^3, 25 views, 96^2 detector: the paper-scale few-view problem.
    "c64": Config("c64", 64, 25, 96, 192.0, 128.0, 10, (4.0, 20.0), (0.0, 1.0), 0.01,
                  1e-2, 1e-4, 1e-4, 2),
    # 8^3, 4 views, 12^2 detector: the autograd check size.
    "c8": Config("c8", 8, 4, 12, 24.0, 16.0, 2, (1.5, 3.0), (0.2, 1.0), 0.01,
                 1e-2, 1e-2, 1e-4, 3),
    # 128^3, 60 views, 192^2 detector: the autograd timing size.
    "c128": Config("c128", 128, 60, 192, 384.0, 256.0, 20, (8.0, 40.0), (0.0, 1.0), 0.005,
                   1e-2, 1e-4, 1e-4, 3),
    # 256^3, 90 views, 384^2 detector: the storage-precision size.
    "c256": Config("c256", 256, 90, 384, 768.0, 512.0, 40, (16.0, 80.0), (0.0, 1.0), 0.01,
                   1e-2, 1e-4, 1e-5, 4),
}


def get_config(name: str) -> Config:
    return CONFIGS[name]

"""Seeded synthetic inputs: voxel grids, coil current segments and right-hand sides.

This module holds geometry and random numbers only -- none of the method's
arithmetic (no Green's function, no Tucker, no ACA).  Both the CUDA path and the
FP64 oracle take their inputs from here, so they see identical data.

Conventions (paper Sec. III.A, Fig. 2 and Algorithm 1):
  * voxel index v = i1 + n1*(i2 + n2*i3)  (column-major reshape of a column),
  * voxel centres at ((i - (n-1)/2) * h) per axis (grid centred at the origin),
  * a segment is (centre[3], unit tangent[3], length) in metres,
  * complex right-hand sides are CN(0,1): real and imaginary parts N(0, 1/2).

The coil layouts are the synthetic stand-ins for the paper's head and body coils
(Sec. IV.B, which uses RWG meshes of real coils that are not available here).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

C0 = 299_792_458.0


@dataclasses.dataclass(frozen=True)
class Grid:
    n1: int
    n2: int
    n3: int
    h: float
    mask_radius: float = 0.0  # voxels with sqrt(x^2+y^2) > mask_radius are zero rows (0 = no mask)
    mask_box: float = 0.0     # voxels with max(|x|, |y|) > mask_box are zero rows (0 = no mask)

    @property
    def nv(self) -> int:
        return self.n1 * self.n2 * self.n3

    @property
    def shape(self):
        return (self.n1, self.n2, self.n3)

    def axis(self, d: int) -> np.ndarray:
        n = self.shape[d]
        return (np.arange(n, dtype=np.float64) - (n - 1) / 2.0) * self.h

    def half_extent(self) -> np.ndarray:
        """Half-extent of the box spanned by the voxel centres, per axis."""
        return np.array([(n - 1) / 2.0 * self.h for n in self.shape])


@dataclasses.dataclass
class Segments:
    centre: np.ndarray   # (m, 3) float64
    tangent: np.ndarray  # (m, 3) float64, unit
    length: np.ndarray   # (m,) float64

    @property
    def m(self) -> int:
        return int(self.length.shape[0])

    def subset(self, idx) -> "Segments":
        idx = np.asarray(idx)
        return Segments(self.centre[idx].copy(), self.tangent[idx].copy(), self.length[idx].copy())


# --------------------------------------------------------------------------------------------
# coil geometries
# --------------------------------------------------------------------------------------------

def circle_coil(radius: float, m: int) -> Segments:
    """m straight segments on the z=0 circle: phi_e = 2*pi*e/m, tangent (-sin, cos, 0),
    length 2*pi*radius/m (workload 'tiny')."""
    phi = 2.0 * np.pi * np.arange(m) / m
    c = np.stack([radius * np.cos(phi), radius * np.sin(phi), np.zeros(m)], axis=1)
    t = np.stack([-np.sin(phi), np.cos(phi), np.zeros(m)], axis=1)
    ln = np.full(m, 2.0 * np.pi * radius / m)
    return Segments(c, t, ln)


def loop_coil_y(radius: float, d: float, m: int) -> Segments:
    """m straight segments on the loop of the given radius in the plane y = d, centred at
    (0, d, 0): phi_e = 2*pi*(e + 1/2)/m, centre (r cos phi, d, r sin phi), tangent
    (-sin phi, 0, cos phi), length 2*pi*r/m (the loop-and-cube geometry of the rank studies)."""
    phi = 2.0 * np.pi * (np.arange(m) + 0.5) / m
    c = np.stack([radius * np.cos(phi), np.full(m, d), radius * np.sin(phi)], axis=1)
    t = np.stack([-np.sin(phi), np.zeros(m), np.cos(phi)], axis=1)
    return Segments(c, t, np.full(m, 2.0 * np.pi * radius / m))


def triangle_coil_y(circumradius: float, d: float, n_per_side: int) -> Segments:
    """The sides of an equilateral triangle in the plane y = d with centroid (0, d, 0) and one
    vertex at (0, d, circumradius), each side cut into n_per_side equal straight segments."""
    ang = np.pi / 2 + 2.0 * np.pi * np.arange(3) / 3
    verts = np.stack([circumradius * np.cos(ang), np.full(3, d), circumradius * np.sin(ang)], axis=1)
    cs, ts, ls = [], [], []
    for a in range(3):
        p0, p1 = verts[a], verts[(a + 1) % 3]
        side = p1 - p0
        L = float(np.linalg.norm(side))
        for i in range(n_per_side):
            cs.append(p0 + side * (i + 0.5) / n_per_side)
            ts.append(side / L)
            ls.append(L / n_per_side)
    return Segments(np.array(cs), np.array(ts), np.array(ls))


def _largest_remainder(total: int, weights) -> list:
    w = np.asarray(weights, dtype=np.float64)
    raw = total * w / w.sum()
    base = np.floor(raw).astype(int)
    rem = raw - base
    left = total - int(base.sum())
    # ties broken by side order (stable sort on -remainder)
    order = np.argsort(-rem, kind="stable")
    for i in order[:left]:
        base[i] += 1
    return [int(b) for b in base]


def cylinder_array(radius: float, length: float, n_elem: int, m_total: int) -> Segments:
    """n_elem rectangular loops on a cylinder of the given radius, each covering
    phi in phi_l +/- 0.4*(2*pi/n_elem) (20 % gap) and z in +/- length/2.

    The m_total/n_elem segments of a loop are split over its four sides in
    proportion to side length (largest remainder, ties in side order).  Arc
    segments use the arc midpoint, the tangent there and the arc length.  The
    circulation is counter-clockwise seen from outside (moment along +r):
    bottom arc along +phi, right side along +z, top arc along -phi, left side along -z.
    """
    assert m_total % n_elem == 0
    per = m_total // n_elem
    half_w = 0.4 * (2.0 * np.pi / n_elem)
    arc_len = radius * 2.0 * half_w
    counts = _largest_remainder(per, [arc_len, length, arc_len, length])
    cs, ts, ls = [], [], []
    for el in range(n_elem):
        phi_l = 2.0 * np.pi * el / n_elem
        p0, p1 = phi_l - half_w, phi_l + half_w
        zb, zt = -length / 2.0, length / 2.0
        # bottom arc, +phi
        n = counts[0]
        for s in range(n):
            pa = p0 + (p1 - p0) * s / n
            pb = p0 + (p1 - p0) * (s + 1) / n
            pm = 0.5 * (pa + pb)
            cs.append([radius * math.cos(pm), radius * math.sin(pm), zb])
            ts.append([-math.sin(pm), math.cos(pm), 0.0])
            ls.append(radius * (pb - pa))
        # right side (phi = p1), +z
        n = counts[1]
        for s in range(n):
            zm = zb + (zt - zb) * (s + 0.5) / n
            cs.append([radius * math.cos(p1), radius * math.sin(p1), zm])
            ts.append([0.0, 0.0, 1.0])
            ls.append(length / n)
        # top arc, -phi
        n = counts[2]
        for s in range(n):
            pa = p1 - (p1 - p0) * s / n
            pb = p1 - (p1 - p0) * (s + 1) / n
            pm = 0.5 * (pa + pb)
            cs.append([radius * math.cos(pm), radius * math.sin(pm), zt])
            ts.append([math.sin(pm), -math.cos(pm), 0.0])
            ls.append(radius * (pa - pb))
        # left side (phi = p0), -z
        n = counts[3]
        for s in range(n):
            zm = zt - (zt - zb) * (s + 0.5) / n
            cs.append([radius * math.cos(p0), radius * math.sin(p0), zm])
            ts.append([0.0, 0.0, -1.0])
            ls.append(length / n)
    return Segments(np.array(cs, dtype=np.float64), np.array(ts, dtype=np.float64),
                    np.array(ls, dtype=np.float64))


def bbox_distance(grid: Grid, centre: np.ndarray) -> np.ndarray:
    """Euclidean distance from each point to the box spanned by the voxel centres (0 inside)."""
    he = grid.half_extent()
    d = np.maximum(np.abs(np.atleast_2d(centre)) - he[None, :], 0.0)
    return np.sqrt((d * d).sum(axis=1))


def random_cylinder_segments(grid: Grid, m: int, seed: int, r_lo=0.12, r_hi=0.20,
                             z_half=0.125, seg_len=0.005) -> Segments:
    """Random segments on cylinders: rho~U[r_lo,r_hi], phi~U[0,2pi), z~U[-z_half,z_half],
    tangent at angle psi~U[0,2pi) in the cylinder's tangent plane (cos psi phi_hat +
    sin psi z_hat), fixed length.  A segment whose centre lies within 2h of the voxel
    box is redrawn (same stream), so every source keeps a clearance of at least 2h."""
    rng = np.random.default_rng(seed)
    out_c, out_t = [], []
    while len(out_c) < m:
        rho = rng.uniform(r_lo, r_hi)
        phi = rng.uniform(0.0, 2.0 * np.pi)
        z = rng.uniform(-z_half, z_half)
        psi = rng.uniform(0.0, 2.0 * np.pi)
        c = np.array([rho * math.cos(phi), rho * math.sin(phi), z])
        if bbox_distance(grid, c)[0] <= 2.0 * grid.h:
            continue
        ph = np.array([-math.sin(phi), math.cos(phi), 0.0])
        zh = np.array([0.0, 0.0, 1.0])
        out_c.append(c)
        out_t.append(math.cos(psi) * ph + math.sin(psi) * zh)
    return Segments(np.array(out_c), np.array(out_t), np.full(m, seg_len))


# --------------------------------------------------------------------------------------------
# workloads (the five synthetic configurations)
# --------------------------------------------------------------------------------------------

FREQ_HZ = 298.2e6


@dataclasses.dataclass
class Workload:
    name: str
    grid: Grid
    segments: Segments
    freq_hz: float
    tol: float          # Tucker tolerance (or ACA tolerance when aca=True)
    p: int              # right-hand sides
    q: int = 3
    aca: bool = False


def workload(name: str) -> Workload:
    """The named synthetic workload.

    tiny      : 24^3 grid, 5 mm, 64 segments on a circle of radius 0.15 m, tol 1e-8, p = 1
    precision : 96^3 grid, 2 mm, 8 loops x 128 segments on a cylinder (r 0.14, L 0.20), tol 1e-6, p = 16
    batching  : 160x160x128, 1.5 mm, 16 loops x 256 segments (r 0.16, L 0.25), tol 1e-6, p <= 128;
                the coil crosses the grid's corners, so voxels outside the square |x|, |y| <=
                (0.16 - 0.02) / sqrt(2) m (whose corners are 2 cm inside the coil) are masked: a box
                mask, which keeps the Tucker ranks of the kept field (a circular mask would not)
    learned   : 128^3, 2 mm, 4096 random segments on cylinders r 0.12..0.20, tol 1e-6
    large     : 320x320x256, 1 mm, 32 loops x 64 segments (r 0.30, L 0.40), ACA tol 1e-5, p = 32
    """
    if name == "tiny":
        g = Grid(24, 24, 24, 0.005)
        return Workload(name, g, circle_coil(0.15, 64), FREQ_HZ, 1e-8, 1)
    if name == "precision":
        g = Grid(96, 96, 96, 0.002)
        return Workload(name, g, cylinder_array(0.14, 0.20, 8, 1024), FREQ_HZ, 1e-6, 16)
    if name == "batching":
        h = 0.0015
        g = Grid(160, 160, 128, h, mask_box=(0.16 - 0.02) / math.sqrt(2.0))
        return Workload(name, g, cylinder_array(0.16, 0.25, 16, 4096), FREQ_HZ, 1e-6, 128, aca=True)
    if name == "learned":
        g = Grid(128, 128, 128, 0.002)
        return Workload(name, g, random_cylinder_segments(g, 4096, seed=0), FREQ_HZ, 1e-6, 1)
    if name == "large":
        g = Grid(320, 320, 256, 0.001)
        return Workload(name, g, cylinder_array(0.30, 0.40, 32, 2048), FREQ_HZ, 1e-5, 32, aca=True)
    raise KeyError(name)


def scaled_workload(name: str, n: tuple, m: int | None = None) -> Workload:
    """A smaller grid with the same voxel size and coil as the named workload
    (used for parity cases the oracle finishes in seconds).  m keeps the first m
    segments spread evenly over the coil."""
    w = workload(name)
    g = Grid(n[0], n[1], n[2], w.grid.h, w.grid.mask_radius, w.grid.mask_box)
    s = w.segments
    if m is not None and m < s.m:
        idx = np.linspace(0, s.m - 1, m).round().astype(int)
        s = s.subset(idx)
    return Workload(w.name + "-scaled", g, s, w.freq_hz, w.tol, w.p, w.q, w.aca)


# --------------------------------------------------------------------------------------------
# random right-hand sides and sketches
# --------------------------------------------------------------------------------------------

def cn01(shape, seed: int, dtype=np.complex128) -> np.ndarray:
    """Circularly-symmetric complex normal CN(0,1), column-major (Fortran) array."""
    rng = np.random.default_rng(seed)
    a = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2.0)
    return np.asfortranarray(a.astype(dtype))


def cn01_columns_c64(rows: int, cols: int, seed: int) -> np.ndarray:
    """CN(0,1) complex64 matrix (column-major) generated column by column, column s from its own
    stream default_rng([seed, s]) in float32: the right-hand sides of the largest workloads
    (tens of GB) without a complex128 intermediate."""
    out = np.empty((rows, cols), dtype=np.complex64, order="F")
    scale = np.float32(1.0 / math.sqrt(2.0))
    for s in range(cols):
        rng = np.random.default_rng([seed, s])
        col = out[:, s]
        col.real = rng.standard_normal(rows, dtype=np.float32) * scale
        col.imag = rng.standard_normal(rows, dtype=np.float32) * scale
    return out


def gaussian_sketch(rows: int, cols: int, seed: int) -> np.ndarray:
    """Complex Gaussian test matrix for randomized range finding (column-major, complex128)."""
    return cn01((rows, cols), seed)


def mode_sketches(grid: Grid, width: int, seed: int, dtype=np.complex64):
    """The three test matrices Omega_g (N_g x width) for a grid, N_1 = n2 n3, N_2 = n1 n3,
    N_3 = n1 n2 (rounded to dtype: both the GPU and the oracle use these exact values)."""
    n1, n2, n3 = grid.shape
    return [gaussian_sketch(r, width, seed + i).astype(dtype) for i, r in enumerate((n2 * n3, n1 * n3, n1 * n2))]


LENGTH_SCALE = 0.1  # metres, scale of the position features


def rank_features(grid: Grid, segs: Segments) -> np.ndarray:
    """Per-segment geometry features (m x 7, float32): centre / 0.1 m, unit tangent, distance
    to the voxel box / 0.1 m."""
    d = bbox_distance(grid, segs.centre)
    f = np.concatenate([segs.centre / LENGTH_SCALE, segs.tangent, (d / LENGTH_SCALE)[:, None]], axis=1)
    return f.astype(np.float32)


# --------------------------------------------------------------------------------------------
# rank-predictor initial weights
# --------------------------------------------------------------------------------------------

MLP_SIZES = (7, 64, 64, 64, 9)


def mlp_init_params(seed: int) -> np.ndarray:
    """He-uniform weights U(-sqrt(6/fan_in), +sqrt(6/fan_in)) and zero biases for the
    7-64-64-64-9 rank predictor, packed as float32 layer by layer: W (out x in, row-major), then b."""
    rng = np.random.default_rng(seed)
    parts = []
    for i in range(len(MLP_SIZES) - 1):
        fi, fo = MLP_SIZES[i], MLP_SIZES[i + 1]
        lim = np.sqrt(6.0 / fi)
        parts.append(rng.uniform(-lim, lim, size=(fo, fi)).reshape(-1))
        parts.append(np.zeros(fo))
    return np.concatenate(parts).astype(np.float32)


def cross_check_fibres(n, count: int, seed: int) -> np.ndarray:
    """count check fibres (g, i_a, i_b) for the fibre cross: mode g uniform in {0, 1, 2}, then the
    indices of the other two modes (a < b) uniform in their ranges; int32 (count, 3)."""
    rng = np.random.default_rng(seed)
    out = np.zeros((count, 3), dtype=np.int32)
    for c in range(count):
        g = int(rng.integers(0, 3))
        a, b = [m for m in range(3) if m != g]
        out[c] = (g, rng.integers(0, n[a]), rng.integers(0, n[b]))
    return out

"""Seeded synthetic inputs for the M_N step (meshes, initial data, coefficients, training densities).

This module only draws and lays out inputs: it holds none of the method's arithmetic (no
quadrature, no basis, no closure, no flux). Both the CUDA path and the CPU oracle consume what it
returns, so it imports neither of them.

Workloads follow the paper's test problems:
  * line source (Sec. 7.1): isotropic Gaussian initial density of width sigma around the origin,
    here with a 1e-4 floor;
  * checkerboard-like block media (Sec. 7.2): piecewise-constant sigma_a, sigma_s on a 7x7 block
    grid, with a unit isotropic source in the centre block.
The paper reads its meshes from files (Sec. 5.2); here a seeded jittered-point Delaunay
triangulation stands in for them, with triangles sorted along a Morton curve of their centroids so
that neighbouring cells sit close in memory.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Mesh:
    xy: np.ndarray   # [V, 2] float64 vertex coordinates
    tri: np.ndarray  # [C, 3] int32 vertex indices, counter-clockwise
    lo: float
    hi: float

    @property
    def ncells(self) -> int:
        return int(self.tri.shape[0])

    def centroids(self) -> np.ndarray:
        return self.xy[self.tri].mean(axis=1)


def _morton_key(ix: np.ndarray, iy: np.ndarray) -> np.ndarray:
    def spread(v):
        v = v.astype(np.uint64) & np.uint64(0xFFFF)
        v = (v | (v << np.uint64(8))) & np.uint64(0x00FF00FF)
        v = (v | (v << np.uint64(4))) & np.uint64(0x0F0F0F0F)
        v = (v | (v << np.uint64(2))) & np.uint64(0x33333333)
        v = (v | (v << np.uint64(1))) & np.uint64(0x55555555)
        return v
    return spread(ix) | (spread(iy) << np.uint64(1))


def jittered_mesh(k: int, lo: float, hi: float, seed: int, jitter: float = 0.3) -> Mesh:
    """k x k grid points on [lo,hi]^2, interior points jittered by +-jitter*h in both directions,
    boundary points only along their edge, corners fixed; Delaunay-triangulated (scipy) and
    Morton-sorted by centroid."""
    from scipy.spatial import Delaunay

    rng = np.random.default_rng(seed)
    h = (hi - lo) / (k - 1)
    g = np.linspace(lo, hi, k)
    X, Y = np.meshgrid(g, g, indexing="ij")
    X = X.copy()
    Y = Y.copy()
    J = rng.uniform(-jitter * h, jitter * h, size=(2, k, k))
    X[1:-1, 1:-1] += J[0, 1:-1, 1:-1]
    Y[1:-1, 1:-1] += J[1, 1:-1, 1:-1]
    # boundary: edges x=lo/hi move in y only, edges y=lo/hi move in x only
    Y[0, 1:-1] += J[1, 0, 1:-1]
    Y[-1, 1:-1] += J[1, -1, 1:-1]
    X[1:-1, 0] += J[0, 1:-1, 0]
    X[1:-1, -1] += J[0, 1:-1, -1]
    pts = np.stack([X.ravel(), Y.ravel()], axis=1)
    tri = Delaunay(pts).simplices.astype(np.int64)
    a = pts[tri]
    cross = (a[:, 1, 0] - a[:, 0, 0]) * (a[:, 2, 1] - a[:, 0, 1]) - (a[:, 2, 0] - a[:, 0, 0]) * (
        a[:, 1, 1] - a[:, 0, 1])
    flip = cross < 0
    tri[flip] = tri[flip][:, [0, 2, 1]]
    cen = pts[tri].mean(axis=1)
    q = np.clip(((cen - lo) / (hi - lo) * 65535.0).astype(np.int64), 0, 65535)
    order = np.argsort(_morton_key(q[:, 0], q[:, 1]), kind="stable")
    tri = tri[order]
    return Mesh(xy=np.ascontiguousarray(pts, dtype=np.float64),
                tri=np.ascontiguousarray(tri, dtype=np.int32), lo=lo, hi=hi)


def line_source_density(cen: np.ndarray, width: float = 0.03, floor: float = 1e-4) -> np.ndarray:
    """Scalar flux Phi(x) = exp(-|x|^2/(2 w^2)) / (2 pi w^2) + floor at the given points
    (Sec. 7.1 initial condition, with a floor)."""
    r2 = (cen ** 2).sum(axis=1)
    return np.exp(-r2 / (2.0 * width * width)) / (2.0 * math.pi * width * width) + floor


def isotropic_moments(phi: np.ndarray, nmom: int) -> np.ndarray:
    """Moments of the isotropic density psi = Phi/(4 pi) in an orthonormal real spherical-harmonic
    basis whose first function is the constant 1/sqrt(4 pi): only the zeroth moment,
    Phi/sqrt(4 pi), is non-zero."""
    u = np.zeros((phi.shape[0], nmom), dtype=np.float64)
    u[:, 0] = phi / math.sqrt(4.0 * math.pi)
    return u


def block_coefficients(cen: np.ndarray, lo: float, hi: float, nb: int, seed: int,
                       sa_max: float = 10.0, ss_max: float = 1.0):
    """Per-block sigma_a ~ U[0,sa_max], sigma_s ~ U[0,ss_max] on an nb x nb block grid; returns
    (block_of_cell int32, sa_block, ss_block). Blocks are indexed bx*nb + by."""
    rng = np.random.default_rng(seed)
    sa = rng.uniform(0.0, sa_max, size=nb * nb)
    ss = rng.uniform(0.0, ss_max, size=nb * nb)
    s = (cen - lo) / (hi - lo) * nb
    b = np.clip(np.floor(s).astype(np.int64), 0, nb - 1)
    blk = (b[:, 0] * nb + b[:, 1]).astype(np.int32)
    return blk, sa, ss


# Checkerboard (Sec. 7.2): on [0,7]^2 of 7 x 7 unit blocks, a source block X_q in the centre and
# absorbing blocks X_a in a checkerboard pattern around it. The paper's layout figure is lost; the
# absorbers here are the blocks (i, j), 1 <= i, j <= 5, with i + j even, except the source block
# (3, 3) and the block (3, 5) above it, so that, as the paper describes, radiation leaves the
# source freely upwards and is damped to the left, the right and below.
CHECKERBOARD_ABSORBERS = tuple((i, j) for i in range(1, 6) for j in range(1, 6)
                               if (i + j) % 2 == 0 and (i, j) not in ((3, 3), (3, 5)))


def checkerboard_medium(cen: np.ndarray):
    """Cross sections and source of the checkerboard (Sec. 7.2) at cell centroids on [0,7]^2:
    absorbers sigma_t = 10, sigma_s = 0 (sigma_a = 10); elsewhere sigma_t = sigma_s = 1
    (sigma_a = 0); isotropic source q = 1 in the centre block. Cells are assigned to blocks by
    centroid. Returns (sigma_a, sigma_s, q)."""
    b = np.clip(np.floor(cen).astype(np.int64), 0, 6)
    absorb = np.zeros(cen.shape[0], dtype=bool)
    for i, j in CHECKERBOARD_ABSORBERS:
        absorb |= (b[:, 0] == i) & (b[:, 1] == j)
    sa = np.where(absorb, 10.0, 0.0)
    ss = np.where(absorb, 0.0, 1.0)
    q = np.where((b[:, 0] == 3) & (b[:, 1] == 3), 1.0, 0.0)
    return sa, ss, q


def two_tissue_density(cen: np.ndarray, split: float = 0.0, hi: float = 5.0,
                       disc=(-0.4, 0.3, 0.25, 2.5)):
    """A heterogeneous density for the transformed CSD equation (Sec. 2): 1 left of x = split,
    `hi` right of it (the density jump 1 -> 5 of the paper's Sec. 7.1 comparison), and a disc
    (x, y, radius, value)."""
    rho = np.where(cen[:, 0] > split, hi, 1.0)
    x, y, r, v = disc
    rho[np.hypot(cen[:, 0] - x, cen[:, 1] - y) < r] = v
    return rho


def vmf_mixtures(count: int, seed: int, max_lobes: int = 4, kappa_lo: float = 0.1,
                 kappa_hi: float = 50.0):
    """Random angular densities: mixtures of 1..max_lobes von Mises-Fisher lobes on S^2.
    Returns (centres [count, max_lobes, 3], kappa [count, max_lobes], weight [count, max_lobes]);
    unused lobes have weight 0. Centres uniform on S^2, kappa log-uniform, weights Dirichlet(1)."""
    rng = np.random.default_rng(seed)
    nl = rng.integers(1, max_lobes + 1, size=count)
    c = rng.normal(size=(count, max_lobes, 3))
    c /= np.linalg.norm(c, axis=2, keepdims=True)
    kap = np.exp(rng.uniform(math.log(kappa_lo), math.log(kappa_hi), size=(count, max_lobes)))
    wt = rng.gamma(1.0, size=(count, max_lobes))
    mask = np.arange(max_lobes)[None, :] < nl[:, None]
    wt = np.where(mask, wt, 0.0)
    wt /= wt.sum(axis=1, keepdims=True)
    return c, kap, wt


def vmf_density(dirs: np.ndarray, centres: np.ndarray, kappa: np.ndarray, weight: np.ndarray):
    """Evaluate the vMF mixtures at unit 3D directions dirs [Q,3] -> [count, Q] (normalised so
    each lobe integrates to 1 over S^2)."""
    dots = np.einsum("clk,qk->clq", centres, dirs)
    # kappa/(4 pi sinh kappa) * exp(kappa (c.x)) written in an overflow-safe form
    k = kappa[:, :, None]
    norm = k / (2.0 * math.pi * (1.0 - np.exp(-2.0 * k)))
    val = norm * np.exp(k * (dots - 1.0))
    return np.einsum("cl,clq->cq", weight, val)


# Workload recipes: (grid points per side, domain, seed). Triangle counts are ~2 (k-1)^2.
WORKLOADS = {
    "m2_line_source_4k": dict(k=45, lo=-1.5, hi=1.5, seed=1, N=2, order=10),
    "m3_line_source_100k": dict(k=224, lo=-1.5, hi=1.5, seed=2, N=3, order=20),
    "m3_blocks_60k": dict(k=173, lo=0.0, hi=7.0, seed=3, N=3, order=10),
    "m5_line_source_1m": dict(k=707, lo=-1.5, hi=1.5, seed=5, N=5, order=30, blocks=True),
    # the checkerboard of Sec. 7.2 (25,000 cells in the paper; 2 x 112^2 = 25,088 here)
    "m3_checkerboard_25k": dict(k=113, lo=0.0, hi=7.0, seed=6, N=3, order=10),
}

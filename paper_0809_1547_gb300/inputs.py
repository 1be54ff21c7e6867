"""Seeded synthetic inputs: sphere packings, material maps, gain masks, configs.

The paper's sample is a granular packing of ~8000 TiO2 spheres (average
diameter 300 nm, refractive index 2.9, so eps_r = 8.41) obtained by
molecular dynamics, with the gain medium infiltrated in the voids
("Simulations" paragraph).  The MD code is not available; these generators
stand in for it: random positions, then iterative removal of overlaps
(each overlapping pair is pushed apart along its axis) until the spheres are
disjoint.  Plain random sequential addition jams near 38 % fill; the overlap
removal reaches the 45 % fill of the workloads.

This module holds none of the step's arithmetic: it only makes inputs, and
both the CUDA path and the oracle consume what it returns.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

C0 = 299_792_458.0
EPS_TIO2 = 2.9 ** 2          # n = 2.9 (paper)
DX_DEFAULT = 20e-9


def courant_dt(dx: float, courant: float = 0.99) -> float:
    """dt = courant * dx / (c sqrt 3)."""
    return courant * dx / (C0 * math.sqrt(3.0))


def sphere_packing(box, n_spheres: int, d_mean: float, d_rel_sd: float, seed: int,
                   center_lo=None, center_hi=None, tol_rel: float = 1e-3,
                   max_iter: int = 4000):
    """Disjoint spheres in an axis-aligned box (metres).

    Diameters ~ normal(d_mean, d_rel_sd d_mean), clipped to [0.5, 1.5] d_mean.
    Centres start uniform in [center_lo, center_hi] (default: the box shrunk by
    one radius) and overlaps are removed iteratively.  Returns (centres (N, 3)
    in metres, radii (N,)).  Raises RuntimeError if the overlaps do not drop
    below tol_rel d_mean.
    """
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    box = np.asarray(box, dtype=np.float64)
    if d_rel_sd > 0:
        d = rng.normal(d_mean, d_rel_sd * d_mean, size=n_spheres)
        d = np.clip(d, 0.5 * d_mean, 1.5 * d_mean)
    else:
        d = np.full(n_spheres, d_mean)
    r = 0.5 * d
    lo = np.zeros(3) if center_lo is None else np.asarray(center_lo, dtype=np.float64)
    hi = box.copy() if center_hi is None else np.asarray(center_hi, dtype=np.float64)
    lo_r = lo[None, :] + (r[:, None] if center_lo is None else 0.0)
    hi_r = hi[None, :] - (r[:, None] if center_hi is None else 0.0)
    x = lo_r + rng.random((n_spheres, 3)) * (hi_r - lo_r)
    if n_spheres < 2:
        return x, r
    rmax = r.max()
    tol = tol_rel * d_mean
    for it in range(max_iter):
        tree = cKDTree(x)
        pairs = tree.query_pairs(2.0 * rmax, output_type="ndarray")
        if len(pairs) == 0:
            break
        a, b = pairs[:, 0], pairs[:, 1]
        dv = x[b] - x[a]
        dist = np.linalg.norm(dv, axis=1)
        overlap = r[a] + r[b] - dist
        m = overlap > 0
        if not m.any() or overlap[m].max() < tol:
            if not m.any() or it > 0:
                break
        a, b, dv, dist, overlap = a[m], b[m], dv[m], dist[m], overlap[m]
        dist = np.maximum(dist, 1e-12 * d_mean)
        u = dv / dist[:, None]
        push = 0.5 * (overlap + 0.1 * tol)[:, None] * u
        disp = np.zeros_like(x)
        np.add.at(disp, a, -push)
        np.add.at(disp, b, push)
        x = np.clip(x + disp, lo_r, hi_r)
    else:
        raise RuntimeError("sphere packing did not converge")
    # final check
    tree = cKDTree(x)
    pairs = tree.query_pairs(2.0 * rmax, output_type="ndarray")
    if len(pairs):
        ov = r[pairs[:, 0]] + r[pairs[:, 1]] - np.linalg.norm(x[pairs[:, 1]] - x[pairs[:, 0]], axis=1)
        if ov.max() >= tol:
            raise RuntimeError(f"sphere packing left an overlap of {ov.max():.3g} m")
    return x, r


def rasterize(grid, dx: float, centers, radii) -> np.ndarray:
    """Boolean [k, j, i] map: cell inside a sphere iff its centre is (staircase)."""
    nx, ny, nz = grid
    inside = np.zeros((nz, ny, nx), dtype=bool)
    for c, rad in zip(np.asarray(centers), np.asarray(radii)):
        lo = np.maximum(np.floor((c - rad) / dx - 0.5).astype(int), 0)
        hi = np.minimum(np.ceil((c + rad) / dx - 0.5).astype(int) + 1, [nx, ny, nz])
        if np.any(hi <= lo):
            continue
        xs = (np.arange(lo[0], hi[0]) + 0.5) * dx - c[0]
        ys = (np.arange(lo[1], hi[1]) + 0.5) * dx - c[1]
        zs = (np.arange(lo[2], hi[2]) + 0.5) * dx - c[2]
        d2 = zs[:, None, None] ** 2 + ys[None, :, None] ** 2 + xs[None, None, :] ** 2
        inside[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] |= d2 < rad * rad
    return inside


def material_maps(grid, inside: np.ndarray, npml: int, eps_sphere: float = EPS_TIO2,
                  eps_void: float = 1.0):
    """eps_r (float32) and gain mask (uint8) of the sample in the interior
    box; the CPML layers hold the background (eps_void, no gain): spheres are
    cut at the layers' inner faces.

    A PML absorbs without reflection, and stays stable, only in a medium
    that is homogeneous along the layer's normal; a dense packing inside
    the layers supports modes that the layer amplifies (a passive pulse in
    a 97^3 realization at 45 % fill grows by e every ~340 steps from step
    ~2000, localised in a slab, while the same run with the background in
    the layers decays)."""
    nx, ny, nz = grid
    inside = np.asarray(inside, dtype=bool)
    if npml > 0:
        core = np.zeros(inside.shape, dtype=bool)
        core[npml:max(npml, nz - npml), npml:max(npml, ny - npml), npml:max(npml, nx - npml)] = True
        inside = inside & core
    eps = np.where(inside, np.float32(eps_sphere), np.float32(eps_void)).astype(np.float32)
    gain = (~inside).astype(np.uint8)
    if npml > 0:
        gain &= core.astype(np.uint8)
    return eps, gain


@dataclass
class Workload:
    """One realization: grid, spacing, materials and run parameters."""
    name: str
    grid: tuple
    dx: float
    dt: float
    eps: np.ndarray
    gain: np.ndarray
    N_a: float
    pump: float
    seed: int
    steps: int
    npml: int = 8
    n_spheres: int = 0
    fill: float = 0.0
    extra: dict = field(default_factory=dict)

    @property
    def ncell(self):
        return int(np.prod(self.grid))

    def gain_fraction(self):
        return float(self.gain.mean())


def _packed_box(n, n_spheres, d_mean, d_rel_sd, seed, dx, npml, name, N_a, pump, noise_seed, steps,
                **extra):
    grid = (n, n, n) if np.isscalar(n) else tuple(n)
    box = np.array(grid, dtype=np.float64) * dx
    centers, radii = sphere_packing(box, n_spheres, d_mean, d_rel_sd, seed)
    inside = rasterize(grid, dx, centers, radii)
    eps, gain = material_maps(grid, inside, npml)
    fill = float(np.sum(4.0 / 3.0 * np.pi * radii ** 3) / np.prod(box))
    return Workload(name, grid, dx, courant_dt(dx), eps, gain, N_a, pump, noise_seed, steps, npml,
                    len(radii), fill, dict(extra))


def n_spheres_for_fill(grid, dx, fill, d_mean, d_rel_sd=0.0):
    vol = float(np.prod(np.asarray(grid, dtype=np.float64) * dx))
    mean_d3 = d_mean ** 3 * (1.0 + 3.0 * d_rel_sd ** 2)
    return int(round(fill * vol / (np.pi / 6.0 * mean_d3)))


def workload_small_48(seed: int = 1) -> Workload:
    """48^3, dx = 20 nm, Courant 0.99, 8-cell CPML, 8 disjoint spheres (d = 300 nm,
    eps 8.41) with centres uniform in the interior, gain in the voids, N_a =
    2e24 m^-3, noise seed 0x5EED, 500 steps, a centre point probe."""
    dx = DX_DEFAULT
    grid = (48, 48, 48)
    npml = 8
    box = np.array(grid) * dx
    centers, radii = sphere_packing(box, 8, 300e-9, 0.0, seed, center_lo=npml * dx * np.ones(3),
                                    center_hi=box - npml * dx)
    inside = rasterize(grid, dx, centers, radii)
    eps, gain = material_maps(grid, inside, npml)
    return Workload("mb48_plain", grid, dx, courant_dt(dx), eps, gain, 2e24, 1e13, 0x5EED, 500,
                    npml, 8, float(np.sum(4 / 3 * np.pi * radii ** 3) / np.prod(box)),
                    {"probe": (24, 24, 24)})


def workload_paper(n: int = 320, seed: int = 7) -> Workload:
    """n^3 box (dx = 20 nm; n = 320 is the paper-scale 6.4 um sample with ~8100
    spheres), d ~ normal(300 nm, 10 %) at ~45 % fill, gain in the voids,
    N_a = 5e24 m^-3 (above threshold), active run."""
    dx = DX_DEFAULT
    grid = (n, n, n)
    count = n_spheres_for_fill(grid, dx, 0.45, 300e-9, 0.10)
    return _packed_box(grid, count, 300e-9, 0.10, seed, dx, 8, f"mb{n}_active", 5e24, 1e13, 0xACE5,
                       20000, probe=(n // 2, n // 2, n // 2))


def workload_paper_320(seed: int = 7) -> Workload:
    """The paper-scale sample: 320^3 (6.4 um box), ~8100 spheres."""
    return workload_paper(320, seed)


def workload_adjoint_96(seed: int = 3) -> Workload:
    """96^3 at 45 % fill of d = 300 nm spheres (225 spheres: 280 spheres, 56 %
    fill, jams against the walls), fixed pump and noise seed, 4000 steps."""
    dx = DX_DEFAULT
    grid = (96, 96, 96)
    n = n_spheres_for_fill(grid, dx, 0.45, 300e-9)
    return _packed_box(grid, n, 300e-9, 0.0, seed, dx, 8, "mb96_adjoint", 5e24, 1e13,
                       0xAD70, 4000, ckpt_every=200)


def workload_large_448(seed: int = 11) -> Workload:
    """448^3 (~9 um box), ~22.9k spheres d = 300 nm at ~45 % fill, 5000 steps."""
    dx = DX_DEFAULT
    grid = (448, 448, 448)
    n = n_spheres_for_fill(grid, dx, 0.45, 300e-9, 0.0)
    return _packed_box(grid, n, 300e-9, 0.0, seed, dx, 8, "mb448_sweep", 5e24, 1e13, 0x1448, 5000)


def workload_batch(n_pump: int = 16, n_seed: int = 5, side_lo: int = 96, side_hi: int = 160,
                   N_a_lo: float = 5e23, N_a_hi: float = 2e25, seed: int = 5):
    """Ensemble: n_pump N_a levels (log-spaced) x n_seed disorder seeds, each
    instance a cube with side drawn uniformly from [side_lo, side_hi], ~45 %
    fill of d = 300 nm spheres, gain in the voids."""
    rng = np.random.default_rng(seed)
    dx = DX_DEFAULT
    N_as = np.geomspace(N_a_lo, N_a_hi, n_pump)
    out = []
    for s in range(n_seed):
        side = int(rng.integers(side_lo, side_hi + 1))
        grid = (side, side, side)
        n = n_spheres_for_fill(grid, dx, 0.45, 300e-9)
        base = _packed_box(grid, n, 300e-9, 0.0, 1000 + s, dx, 8, f"batch_s{s}", 0.0, 1e13, 0, 10000)
        for q, N_a in enumerate(N_as):
            out.append(Workload(f"batch_s{s}_p{q}", grid, dx, base.dt, base.eps, base.gain, float(N_a),
                                1e13, 0xB000 + 97 * s + q, 10000, 8, base.n_spheres, base.fill))
    return out


def random_small(grid, seed: int, npml: int = 4, fill: float = 0.4, eps_sphere: float = EPS_TIO2,
                 d_cells: float = 5.0):
    """Small random test realization (any shape): spheres of d_cells cells."""
    dx = DX_DEFAULT
    grid = tuple(int(v) for v in grid)
    n = max(1, n_spheres_for_fill(grid, dx, fill, d_cells * dx))
    box = np.array(grid) * dx
    centers, radii = sphere_packing(box, n, d_cells * dx, 0.0, seed, center_lo=np.zeros(3),
                                    center_hi=box, max_iter=20000, tol_rel=1e-2)
    inside = rasterize(grid, dx, centers, radii)
    eps, gain = material_maps(grid, inside, npml, eps_sphere)
    return eps, gain

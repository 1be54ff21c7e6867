"""Helpers for running the CUDA path and the oracle on identical inputs."""
from __future__ import annotations

import math

import numpy as np

from oracle.mb_oracle import MBOracle, Params, FIELD_NAMES

DX = 20e-9
DT = 0.99 * DX / (299_792_458.0 * math.sqrt(3.0))

# Per-field tolerance after the run: relative L2 of (gpu - oracle) / oracle.
# 1e-5 is the bound stated for the FP32 step against the FP64 oracle.
REL_L2_TOL = 1e-5


def params_kw(**kw):
    base = dict(lambda0=590e-9, dlambda=230e-9, tau32=100e-15, tau21=1e-9, tau10=100e-15,
                a_se=-1.0, dipole_len=0.1e-9, n_floor_rel=1e-9, npml=8, pml_order=3.0,
                pml_sigma_factor=0.8, pml_alpha_rel=0.1)
    base.update(kw)
    return base


def make_pair(grid, eps, gain, N_a, pump, seed, pkw, dt=DT, dx=DX):
    """An oracle and a GPU simulation set up identically (fields zero)."""
    from paper_0809_1547_gb300.binding import MBSimulation, mb_default_params
    o = MBOracle(grid, dx, dt, Params(**pkw))
    o.set_material(eps, gain, N_a, pump)
    o.set_seed(seed)
    g = MBSimulation(grid, dx, dt, mb_default_params(**pkw))
    g.set_material(eps, gain, N_a, pump)
    g.set_seed(seed)
    return o, g


def rel_l2(gpu, ref):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref)
    num = np.linalg.norm(gpu - ref)
    if den == 0.0:
        return 0.0 if num == 0.0 else math.inf
    return num / den


def field_errors(o, g, names=FIELD_NAMES):
    return {name: rel_l2(g.field(name), o.field(name)) for name in names}


def assert_fields_match(o, g, tol=REL_L2_TOL, names=FIELD_NAMES):
    errs = field_errors(o, g, names)
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, f"fields beyond rel-L2 {tol}: {bad}"
    return errs


# --------------------------------------------- sampled sub-blocks at full size
# One GPU step of a large grid checked on sub-blocks [lo, lo + size)^3: the
# oracle steps the block from the GPU's state of it, with the whole grid's
# CPML profiles (the oracle's own profile function on the whole grid's
# sizes, sliced to the block), the GPU's CPML memories, the whole grid's
# noise counters and step index.  Cells whose neighbours lie outside the
# block (the one-cell halo) are left out of the comparison, except where the
# block's face is the grid's own boundary (fields beyond it are zero in both).

# oracle keys of the GPU's four memory planes f per slab axis (x, y, z)
_CPML_KEYS = {0: (("E", ("y", "x")), ("E", ("z", "x")), ("H", ("y", "x")), ("H", ("z", "x"))),
              1: (("E", ("x", "y")), ("E", ("z", "y")), ("H", ("x", "y")), ("H", ("z", "y"))),
              2: (("E", ("x", "z")), ("E", ("y", "z")), ("H", ("x", "z")), ("H", ("y", "z")))}


def _slab_layer(idx, n, L):
    inside = (idx < L) | (idx >= n - L)
    return inside, np.where(idx < L, idx, idx - n + 2 * L)


def block_cpml(psi3, lo, size, grid, L):
    """The GPU's CPML memories (psi3[axis] as MBSimulation.cpml returns them)
    on the block as the oracle's per-cell arrays {(kind, key): [k, j, i]}."""
    nx, ny, nz = grid
    i0, j0, k0 = lo
    K, J, I = np.meshgrid(np.arange(k0, k0 + size), np.arange(j0, j0 + size),
                          np.arange(i0, i0 + size), indexing="ij")
    out = {}
    for axis in range(3):
        P = psi3[axis]
        for f, kk in enumerate(_CPML_KEYS[axis]):
            v = np.zeros((size,) * 3)
            if P is not None and L > 0:
                if axis == 0:
                    m, s = _slab_layer(I, nx, L)
                    v[m] = P[f, K[m], J[m], s[m]]
                elif axis == 1:
                    m, s = _slab_layer(J, ny, L)
                    v[m] = P[f, K[m], s[m], I[m]]
                else:
                    m, s = _slab_layer(K, nz, L)
                    v[m] = P[f, s[m], J[m], I[m]]
            out[kk] = v
    return out


def device_block(g, lo, size):
    """Every field of the block (SI, FP64, [k, j, i]) read on the device."""
    i0, j0, k0 = lo
    out = {}
    for name in FIELD_NAMES:
        if name == "N0":
            continue
        t, scale = g.field_device(name)
        out[name] = t[k0:k0 + size, j0:j0 + size, i0:i0 + size].double().cpu().numpy() * scale
    return out


def block_oracle(w, lo, size, fields, psi, n_step, pkw, sources=()):
    """The oracle on the block of workload w with the GPU's state of it;
    sources: (ijk, comp, lam, t0, tau, amp) in whole-grid cells, added where
    they fall inside the block."""
    from oracle.mb_oracle import AX_X, AX_Y, AX_Z, cpml_profile
    nx, ny, nz = w.grid
    i0, j0, k0 = lo
    sl = (slice(k0, k0 + size), slice(j0, j0 + size), slice(i0, i0 + size))
    p = Params(**pkw)
    o = MBOracle((size,) * 3, w.dx, w.dt, p)
    o.set_material(w.eps[sl], w.gain[sl], w.N_a, w.pump)
    o.set_seed(w.seed)
    for name, ax, n, a0 in (("x", AX_X, nx, i0), ("y", AX_Y, ny, j0), ("z", AX_Z, nz, k0)):
        shape = [size if a == ax else 1 for a in range(3)]
        for half, tab in ((0.0, o.be), (0.5, o.bh)):
            b, c = cpml_profile(n, half, w.dx, w.dt, p)
            tab[name] = (b[a0:a0 + size].reshape(shape), c[a0:a0 + size].reshape(shape))
    kk, jj, ii = np.meshgrid(np.arange(k0, k0 + size), np.arange(j0, j0 + size),
                             np.arange(i0, i0 + size), indexing="ij")
    o.cell_index = (ii + nx * (jj + ny * kk)).astype(np.uint64)
    o.n = n_step
    for name, v in fields.items():
        o.set_field(name, v)
    gain = w.gain[sl] != 0
    o.N[0] = np.where(gain, w.N_a - fields["N1"] - fields["N2"] - fields["N3"], 0.0)
    for (kind, key), v in psi.items():
        (o.psi_E if kind == "E" else o.psi_H)[key] = v.copy()
    for ijk, comp, lam, t0, tau, amp in sources:
        loc = tuple(int(a) - int(b) for a, b in zip(ijk, lo))
        if all(0 <= v < size for v in loc):
            o.add_source(loc, comp, lam, t0, tau, amp)
    return o


def block_core(lo, size, grid):
    """Slices of the block's compared cells: the halo dropped except along a
    face that is the grid's own boundary."""
    out = []
    for a, n in zip(lo[::-1], grid[::-1]):        # [k, j, i] order
        out.append(slice(0 if a == 0 else 1, size if a + size == n else size - 1))
    return tuple(out)


def check_blocks_one_step(g, w, step, los, size, pkw, tol=REL_L2_TOL, sources=()):
    """Read the blocks of g (fields and CPML memories), call step() (one GPU
    step of g), and compare every field and memory of each block's compared
    cells with the oracle's step of the block.  Returns the worst error."""
    psi3 = [g.cpml(a) for a in range(3)]
    before = [(device_block(g, lo, size), block_cpml(psi3, lo, size, w.grid, pkw["npml"]))
              for lo in los]
    n_before = g.n
    step()
    psi3 = [g.cpml(a) for a in range(3)]
    after = [(device_block(g, lo, size), block_cpml(psi3, lo, size, w.grid, pkw["npml"]))
             for lo in los]
    worst = 0.0
    for lo, (f0, p0), (f1, p1) in zip(los, before, after):
        o = block_oracle(w, lo, size, f0, p0, n_before, pkw, sources)
        o.step(1)
        core = block_core(lo, size, w.grid)
        for name, v in f1.items():
            ref = o.field(name)[core]
            err = rel_l2(v[core], ref)
            worst = max(worst, err if np.isfinite(err) else 0.0)
            assert err <= tol or np.abs(ref).max() == 0 == np.abs(v[core]).max(), (lo, name, err)
        for kk, v in p1.items():
            ref = (o.psi_E if kk[0] == "E" else o.psi_H)[kk[1]][core]
            err = rel_l2(v[core], ref)
            worst = max(worst, err if np.isfinite(err) else 0.0)
            assert err <= tol or np.abs(ref).max() == 0 == np.abs(v[core]).max(), (lo, kk, err)
    return worst

"""The sampled sub-block check of the full-size parity tests, validated on
the CPU: a whole-grid oracle run stands in for the device (its fields read
as tensors, its CPML memories repacked into the library's slab layout of
mb_get_cpml), so the block oracle must reproduce it to rounding on blocks
at the low and high walls, across every CPML interface and in the bulk."""
import math
from types import SimpleNamespace

import numpy as np
import pytest

from oracle.mb_oracle import MBOracle, Params
from parity_util import check_blocks_one_step, params_kw

_E_KEYS = {0: (("y", "x"), ("z", "x")), 1: (("x", "y"), ("z", "y")), 2: (("x", "z"), ("y", "z"))}


class _OracleAsDevice:
    """Accessors of a simulation on the GPU path, served by a whole-grid oracle."""

    def __init__(self, o, L):
        self.o, self.L = o, L

    @property
    def n(self):
        return self.o.n

    def field_device(self, name):
        import torch
        return torch.from_numpy(np.ascontiguousarray(self.o.field(name))), 1.0

    def cpml(self, axis):
        o, L = self.o, self.L
        nz, ny, nx = o.shape
        n = (nx, ny, nz)[axis]
        layers = np.r_[np.arange(L), np.arange(n - L, n)]      # layer s -> index
        planes = [o.psi_E[k] for k in _E_KEYS[axis]] + [o.psi_H[k] for k in _E_KEYS[axis]]
        if axis == 0:
            return np.stack([p[:, :, layers] for p in planes])              # (4, nz, ny, 2L)
        if axis == 1:
            return np.stack([p[:, layers, :] for p in planes])              # (4, nz, 2L, nx)
        return np.stack([p[layers, :, :] for p in planes])                  # (4, 2L, ny, nx)


def test_block_check_reproduces_a_whole_grid_oracle():
    pytest.importorskip("torch")
    from paper_0809_1547_gb300 import inputs
    grid, L = (30, 28, 26), 4
    eps, gain = inputs.random_small(grid, seed=3, npml=L)
    dx = 20e-9
    dt = 0.99 * dx / (299_792_458.0 * math.sqrt(3.0))
    w = SimpleNamespace(grid=grid, dx=dx, dt=dt, eps=eps, gain=gain, N_a=4e24, pump=1e13, seed=99)
    pkw = params_kw(npml=L)
    o = MBOracle(grid, dx, dt, Params(**pkw))
    o.set_material(eps, gain, w.N_a, w.pump)
    o.set_seed(w.seed)
    o.add_source((15, 14, 13), 2, 532e-9, 4e-15, 1e-15, 1e9)
    o.step(40)
    size = 10
    los = [(0, 0, 0), (20, 18, 16), (0, 9, 16), (20, 0, 8), (10, 18, 0), (11, 9, 8), (1, 2, 3)]
    dev = _OracleAsDevice(o, L)
    src = ((15, 14, 13), 2, 532e-9, 4e-15, 1e-15, 1e9)
    worst = check_blocks_one_step(dev, w, lambda: o.step(1), los, size, pkw, tol=1e-12,
                                  sources=[src])
    assert worst <= 1e-12
    # the memories were live: the CPML of this run holds non-zero values
    assert np.abs(dev.cpml(0)).max() > 0 and np.abs(dev.cpml(2)).max() > 0


def test_block_check_fails_when_the_memories_are_dropped():
    """The check must see the CPML: seeding the block with zero memories
    (a plausible mistake in the layout mapping) fails it."""
    pytest.importorskip("torch")
    from paper_0809_1547_gb300 import inputs
    grid, L = (30, 28, 26), 4
    eps, gain = inputs.random_small(grid, seed=3, npml=L)
    dx = 20e-9
    dt = 0.99 * dx / (299_792_458.0 * math.sqrt(3.0))
    w = SimpleNamespace(grid=grid, dx=dx, dt=dt, eps=eps, gain=gain, N_a=4e24, pump=1e13, seed=99)
    pkw = params_kw(npml=L)
    o = MBOracle(grid, dx, dt, Params(**pkw))
    o.set_material(eps, gain, w.N_a, w.pump)
    o.set_seed(w.seed)
    o.add_source((15, 14, 13), 2, 532e-9, 4e-15, 1e-15, 1e9)
    o.step(40)
    dev = _OracleAsDevice(o, L)
    dev.cpml = lambda axis, real=dev.cpml: np.zeros_like(real(axis))
    with pytest.raises(AssertionError):
        check_blocks_one_step(dev, w, lambda: o.step(1), [(0, 0, 0)], 10, pkw, tol=1e-6)

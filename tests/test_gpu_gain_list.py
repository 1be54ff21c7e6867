"""The material bytes and the gain-cell list mb_set_material builds on the
device (distinct values by compare-and-swap, ids by first appearance;
chunked counts, an ordered scan, an ordered scatter) against the host
statement of the map (mb_material_map, a separate implementation): equal,
on grids whose cell counts end inside an 8192-cell chunk, span several
chunks, or fit in one, with two, six or more than 128 distinct values, and
at the benchmarked 320^3 size; empty lists with the gain off."""
import numpy as np
import pytest

from paper_0809_1547_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_0809_1547_gb300 import build
    build.build()


@pytest.mark.parametrize("grid,seed", [((48, 48, 48), 1), ((97, 61, 33), 2), ((16, 16, 8), 3),
                                       ((160, 96, 80), 4)])
def test_device_gain_list_equals_the_host_map(grid, seed):
    from paper_0809_1547_gb300.binding import MBSimulation, mb_default_params, mb_material_map
    eps, gain = inputs.random_small(grid, seed=seed, npml=4)
    sim = MBSimulation(grid, 20e-9, inputs.courant_dt(20e-9), mb_default_params(npml=4))
    sim.set_material(eps, gain, 3e24, 1e13)
    dev = sim.gain_list()
    mat_h, host, _, _ = mb_material_map(eps, gain, True, 16)
    assert np.array_equal(sim.material().ravel(), np.asarray(mat_h).ravel())
    assert dev.dtype == np.uint32 and dev.size == int(np.count_nonzero(gain.ravel()))
    assert np.array_equal(dev, np.asarray(host, dtype=np.uint32))
    assert np.all(np.diff(dev.astype(np.int64)) > 0)
    # the gain off: no gain cells
    sim.set_material(eps, gain, 0.0, 1e13)
    assert sim.gain_list().size == 0
    # a second map on the same context: the list follows it
    gain2 = np.ascontiguousarray(gain[::-1])
    sim.set_material(eps, gain2, 3e24, 1e13)
    _, host2, _, _ = mb_material_map(eps, gain2, True, 16)
    assert np.array_equal(sim.gain_list(), np.asarray(host2, dtype=np.uint32))
    sim.close()


@pytest.mark.parametrize("n_values", [6, 200])
def test_device_material_bytes_with_many_values(n_values):
    """Six values in runs across the grid, or more than 128 (a dense map):
    the device bytes equal the host map's."""
    from paper_0809_1547_gb300.binding import MBSimulation, mb_default_params, mb_material_map
    grid = (40, 36, 30)
    eps, gain = inputs.random_small(grid, seed=12, npml=4)
    rng = np.random.default_rng(n_values)
    vals = (1.0 + rng.random(n_values) * 9.0).astype(np.float32)
    runs = rng.integers(0, n_values, size=eps.size // 37 + 1)
    eps = np.repeat(vals[runs], 37)[:eps.size].reshape(eps.shape).astype(np.float32)
    sim = MBSimulation(grid, 20e-9, inputs.courant_dt(20e-9), mb_default_params(npml=4))
    sim.set_material(eps, gain, 3e24, 1e13)
    mat_h, host, values, dense = mb_material_map(eps, gain, True, 16)
    assert bool(dense) == (n_values > 128)
    assert np.array_equal(sim.material().ravel(), np.asarray(mat_h).ravel())
    assert np.array_equal(sim.gain_list(), np.asarray(host, dtype=np.uint32))
    sim.close()


def test_device_map_at_full_size():
    """The 320^3 packing the benchmark steps (32.8 M cells, 14.4 M gain
    cells, 4000 chunks of the gain list): material bytes and gain-cell list
    equal to the host map's, and the gain cells' count to the mask's."""
    from paper_0809_1547_gb300.binding import MBSimulation, mb_default_params, mb_material_map
    w = inputs.workload_paper_320()
    sim = MBSimulation(w.grid, w.dx, w.dt, mb_default_params(npml=w.npml))
    sim.set_material(w.eps, w.gain, w.N_a, w.pump)
    mat_h, host, _, dense = mb_material_map(w.eps, w.gain, True, 16)
    assert not dense
    assert np.array_equal(sim.material().ravel(), np.asarray(mat_h).ravel())
    dev = sim.gain_list()
    assert dev.size == int(np.count_nonzero(w.gain))
    assert np.array_equal(dev, np.asarray(host, dtype=np.uint32))
    sim.close()

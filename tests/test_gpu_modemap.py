"""CW source, whole-plane DFT probes (mode maps) and plane energy-density
snapshots on the GPU (through the C ABI) against the FP64 oracle.

Bar: mode maps and snapshots (squared quantities) within relative L2 2e-5
of the oracle, as for the spectra; the snapshot planes sum to mb_energy;
graph replay and save/load leave the accumulators bit-identical; at 192^3 one
probe step equals the definition (E of the plane times the DFT weight,
squared).
"""
import math

import numpy as np
import pytest

from parity_util import DX, DT, params_kw, make_pair, rel_l2, assert_fields_match

pytestmark = pytest.mark.gpu

TOL2 = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_0809_1547_gb300 import build
    build.build()


def _setup(sim, oracle, grid):
    src = ((grid[0] // 2, grid[1] // 2, grid[2] // 2), 2, 586.5e-9, 0.5e-15, 1.0e-15, 1e9, 10 ** 5)
    if oracle:
        sim.add_source_cw(*src)
    else:
        sim.set_source_cw(*src)
    a = sim.add_plane_probe(grid[2] // 2, 1, 3, 560e-9, 615e-9)
    b = sim.add_plane_probe(3, 3, 2, 400e-9, 800e-9)
    return a, b


@pytest.mark.parametrize("N_a", [0.0, 4e24])
def test_cw_mode_maps_and_snapshots_match_oracle(N_a):
    from paper_0809_1547_gb300 import inputs
    grid = (33, 26, 20)
    eps, gain = inputs.random_small(grid, seed=12, npml=4, d_cells=5)
    o, g = make_pair(grid, eps, gain, N_a, 1e13, 0x5A5A, params_kw(npml=4))
    pa_o, pb_o = _setup(o, True, grid)
    pa_g, pb_g = _setup(g, False, grid)
    o.step(150)
    g.step(150)
    assert_fields_match(o, g)
    for po, pg, bins in ((pa_o, pa_g, 3), (pb_o, pb_g, 2)):
        for b in range(bins):
            m_o = o.plane_mode_map(po, b)
            m_g = g.plane_mode_map(pg, b)
            assert m_o.max() > 0
            assert rel_l2(m_g, m_o) <= TOL2, (po, b, rel_l2(m_g, m_o))
    for k in (0, 3, grid[2] // 2, grid[2] - 1):
        u_o = o.plane_energy_density(k)
        u_g = g.plane_energy_density(k)
        assert rel_l2(u_g, u_o) <= TOL2, (k, rel_l2(u_g, u_o))
    g.close()


def test_snapshot_planes_sum_to_the_energy():
    from paper_0809_1547_gb300 import inputs
    grid = (24, 22, 20)
    eps, gain = inputs.random_small(grid, seed=4, npml=4, d_cells=5)
    _, g = make_pair(grid, eps, gain, 3e24, 1e13, 9, params_kw(npml=4))
    g.set_source_cw((12, 11, 10), 0, 586.5e-9, 0.0, 1e-15, 1e9, 10 ** 4)
    g.step(60)
    U, _ = g.energy()
    total = sum(g.plane_energy_density(k).sum() for k in range(grid[2])) * DX ** 3
    assert total == pytest.approx(U, rel=1e-9, abs=0)
    g.close()


def test_plane_probes_in_graphs_and_save_load_bitwise():
    from paper_0809_1547_gb300 import inputs
    grid = (32, 20, 18)
    eps, gain = inputs.random_small(grid, seed=5, npml=3, d_cells=5)
    pk = params_kw(npml=3)
    _, a = make_pair(grid, eps, gain, 4e24, 1e13, 3, pk)
    _, b = make_pair(grid, eps, gain, 4e24, 1e13, 3, pk)
    pa, _ = _setup(a, False, grid)
    pb, _ = _setup(b, False, grid)
    a.step(37)                      # graph chunks + single-step graph
    for _ in range(20):
        b.step(1)
    blob = b.save_state()
    b.step(17)
    np.testing.assert_array_equal(a.plane_mode_map(pa, 1), b.plane_mode_map(pb, 1))
    b.load_state(blob)
    b.step(17)
    np.testing.assert_array_equal(a.plane_mode_map(pa, 1), b.plane_mode_map(pb, 1))
    a.close()
    b.close()


def test_batch_rejects_plane_probes():
    from paper_0809_1547_gb300.binding import MBBatch, MBError, MB_ERR_STATE, mb_default_params
    grid = (16, 16, 16)
    bt = MBBatch([grid, grid], DX, DT, mb_default_params(npml=2))
    for q in range(2):
        bt.set_instance(q, np.ones(grid[::-1], np.float32), np.ones(grid[::-1], np.uint8), 1e24, 1e13, q)
    bt.instances[1].add_plane_probe(8, 1, 1, 590e-9, 590e-9)
    with pytest.raises(MBError) as e:
        bt.step(1)
    assert e.value.code == MB_ERR_STATE
    bt.close()


def test_plane_probe_step_is_its_definition_at_192():
    """192^3 workload: one probe step equals E of the plane (at t_{n+1}) times
    the DFT weight, squared and summed over components."""
    from paper_0809_1547_gb300 import inputs
    from paper_0809_1547_gb300.binding import MBSimulation, mb_default_params
    w = inputs.workload_paper(192, seed=7)
    g = MBSimulation(w.grid, w.dx, w.dt, mb_default_params(npml=w.npml))
    g.set_material(w.eps, w.gain, w.N_a, w.pump)
    g.set_seed(w.seed)
    g.set_source_cw((96, 96, 96), 1, 586.5e-9, 0.0, 1e-15, 1e9, 1000)
    g.step(40)
    k = 96
    pid = g.add_plane_probe(k, 1, 2, 586.5e-9, 600e-9)
    g.step(1)
    e2 = sum(g.field(c)[k].astype(np.float64) ** 2 for c in ("Ex", "Ey", "Ez"))
    expect = e2 * w.dt ** 2
    for b in range(2):
        m = g.plane_mode_map(pid, b)
        np.testing.assert_allclose(m, expect, rtol=1e-6, atol=1e-300)   # fields read back in FP32
    u = g.plane_energy_density(k)
    assert np.isfinite(u).all() and u.max() > 0
    g.close()

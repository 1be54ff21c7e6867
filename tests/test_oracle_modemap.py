"""Pins of the oracle's CW source, plane probe (mode map) and energy-density
snapshot (CPU).

The paper shows the field of a long-living mode on the sample's middle
section under continuous-wave excitation (inset of Fig. 1, at 586.5 nm) and a
snapshot of the energy density on that section during lasing (Fig. 2a).
Pins: the snapshot's per-cell terms sum to the total discrete energy; the
plane DFT equals point probes placed on its cells; the CW waveform's closed
form (zero value and slope at switch-on, the bare sinusoid once the rise is
over); a passive CW-driven box concentrates the mode map in the bin of the
drive frequency; the map scales as the drive amplitude squared (linear
medium).
"""
import math

import numpy as np
import pytest

from oracle.mb_oracle import MBOracle, Params, C0, source_waveform_cw

DX = 20e-9
DT = 0.99 * DX / (C0 * math.sqrt(3.0))


def _box(grid=(16, 15, 14), npml=4, N_a=0.0, seed=3):
    rng = np.random.default_rng(seed)
    eps = np.where(rng.random(grid[::-1]) < 0.3, 8.41, 1.0)
    gain = (eps == 1.0).astype(np.uint8)
    o = MBOracle(grid, DX, DT, Params(npml=npml))
    o.set_material(eps, gain, N_a, 1e13)
    o.set_seed(11)
    return o


def test_energy_density_planes_sum_to_the_energy():
    o = _box(N_a=3e24)
    rng = np.random.default_rng(1)
    for name in ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz"):
        o.set_field(name, rng.standard_normal(o.shape) * (1e5 if name[0] == "E" else 1e2))
    o.step(7)
    total = sum(o.plane_energy_density(k).sum() for k in range(o.nz)) * DX ** 3
    assert total == pytest.approx(o.energy(), rel=1e-12, abs=0)
    assert np.all(o.plane_energy_density(3) >= 0)


def test_plane_probe_equals_point_probes_on_its_cells():
    o = _box(N_a=3e24)
    o.add_source_cw((8, 7, 7), 1, 586.5e-9, 0.5e-15, 1.0e-15, 1e9, 10 ** 6)
    k = 6
    pid = o.add_plane_probe(k, 1, 3, 560e-9, 615e-9)
    cells = [(2, 3), (8, 7), (15, 14), (0, 0)]
    pts = [o.add_point_probe((i, j, k), 3, 560e-9, 615e-9) for i, j in cells]
    o.step(40)
    acc = o.plane_probes[pid]["acc"]
    for (i, j), q in zip(cells, pts):
        np.testing.assert_allclose(acc[:, :, j, i].T, o.point_probes[q]["acc"], rtol=1e-12, atol=0)
    assert np.abs(acc).max() > 0


def test_plane_probe_sampling_interval_does_not_change_the_map():
    """Sampling every 3 steps with the weight 3 dt instead of every step with
    dt is another Riemann sum of the same DFT integral: for the CW mode (51
    steps per period) the two maps agree to about 1 %."""
    maps = []
    for every in (1, 3):
        o = _box()
        o.add_source_cw((8, 7, 7), 1, 586.5e-9, 0.5e-15, 1.0e-15, 1e9, 10 ** 6)
        pid = o.add_plane_probe(6, every, 3, 560e-9, 615e-9)
        o.step(240)
        maps.append(o.plane_mode_map(pid, 1))
    assert np.abs(maps[1] - maps[0]).max() <= 0.05 * np.abs(maps[0]).max()


def test_cw_waveform_closed_form():
    lam, t0, tau, amp = 586.5e-9, 2e-15, 1e-15, 3.0
    ws = 2 * math.pi * C0 / lam
    assert source_waveform_cw(t0, lam, t0, tau, amp) == 0.0
    assert source_waveform_cw(t0 - 1e-16, lam, t0, tau, amp) == 0.0
    h = 1e-19
    slope = (source_waveform_cw(t0 + h, lam, t0, tau, amp) - 0.0) / h
    assert abs(slope) < 1e-6 * amp * ws          # rises as (t - t0)^3 from zero
    t = t0 + 12 * tau
    assert source_waveform_cw(t, lam, t0, tau, amp) == pytest.approx(
        amp * math.sin(ws * (t - t0)), rel=1e-12, abs=1e-12 * amp)


def _cw_run(amp, steps=500):
    o = _box(grid=(18, 18, 18), npml=4)
    o.add_source_cw((9, 9, 9), 2, 586.5e-9, 0.0, 2e-15, amp, steps)
    pid = o.add_plane_probe(9, 1, 3, 400e-9, 800e-9)     # bins 400, 600, 800 nm
    o.step(steps)
    return o, pid


def test_cw_mode_map_peaks_at_the_drive_frequency_and_is_quadratic():
    o1, pid = _cw_run(1e9)
    maps = [o1.plane_mode_map(pid, b) for b in range(3)]
    tot = [m.sum() for m in maps]
    assert tot[1] > 20 * tot[0] and tot[1] > 20 * tot[2], tot
    o3, _ = _cw_run(3e9)
    np.testing.assert_allclose(o3.plane_mode_map(pid, 1), 9.0 * maps[1], rtol=1e-9,
                               atol=1e-12 * maps[1].max())

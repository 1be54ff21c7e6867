"""The single-pass step (H half-step, Lorentz update and E / population
update in one launch, E / H / CPML memories ping-ponged between two copies)
against the two-pass step, bit for bit, and against the FP64 oracle.

Cases: tiles whose halo row / column cross CPML slabs, the grid's low
walls and ragged y / z tails; chunks of kz planes that split the z range
(the first plane recomputes the plane below); odd step counts (the state
then sits in the second copy) with field access, save / load, mode switches
and the adjoint from there; every probe kind; the dense 1/eps map.
"""
import numpy as np
import pytest

from oracle.mb_oracle import FIELD_NAMES
from parity_util import DX, DT, params_kw, make_pair, assert_fields_match

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_0809_1547_gb300 import build
    build.build()


def _setup(grid, npml, seed, dense=False):
    from paper_0809_1547_gb300 import inputs
    eps, gain = inputs.random_small(grid, seed=seed, npml=npml, d_cells=5)
    if dense:
        rng = np.random.default_rng(seed)
        eps = np.where(eps > 1.0, eps + rng.random(eps.shape).astype(np.float32) * 0.5, 1.0)
        eps = eps.astype(np.float32)
    _, g = make_pair(grid, eps, gain, 4e24, 1e13, 11 + seed, params_kw(npml=npml))
    g.set_source((grid[0] // 2, grid[1] // 2, grid[2] // 2), 2, 532e-9, 1.0e-15, 0.4e-15, 1e9)
    g.add_point_probe((grid[0] // 3, grid[1] // 2, grid[2] // 2), 16, 480e-9, 700e-9)
    g.add_face_probes(2, 1, 8, 500e-9, 650e-9)
    g.add_plane_probe(grid[2] // 2, 2, 4, 520e-9, 640e-9)
    return g


def _snapshot(g):
    out = {name: g.field(name) for name in FIELD_NAMES}
    out["point"] = g.probe_spectrum(0)[0]
    out["faces"] = [g.face_spectrum(f)[0] for f in range(6)]
    out["plane"] = g.plane_mode_map(0, 1)
    out["energy"] = g.energy()
    return out


def _assert_same(ref, got, what):
    for name in FIELD_NAMES:
        a, b = ref[name], got[name]
        if not np.array_equal(a, b):
            where = tuple(np.argwhere(a != b)[0])
            raise AssertionError(f"{what}: {name} differs at [k,j,i]={where}: {a[where]!r} vs {b[where]!r}")
    np.testing.assert_array_equal(got["point"], ref["point"], err_msg=what)
    for f in range(6):
        np.testing.assert_array_equal(got["faces"][f], ref["faces"][f], err_msg=f"{what} face {f}")
    np.testing.assert_array_equal(got["plane"], ref["plane"], err_msg=what)
    # energy is a sum of identical fields; the face flux adds FP32 per-warp
    # partials (grouped by the tile shape) into FP64 slots in launch order,
    # so it is fixed to FP32 rounding only
    assert got["energy"][0] == pytest.approx(ref["energy"][0], rel=1e-12, abs=0)
    np.testing.assert_allclose(got["energy"][1], ref["energy"][1], rtol=1e-6,
                               atol=1e-6 * np.abs(ref["energy"][1]).max())


@pytest.mark.parametrize("grid,npml", [((64, 20, 24), 4), ((96, 17, 13), 4), ((32, 40, 35), 6)])
def test_single_pass_equals_two_passes_bitwise(grid, npml):
    g = _setup(grid, npml, seed=sum(grid))
    g.step(4)
    blob = g.save_state()
    g.set_tuning((1, 32, 4, 8), (1, 32, 4, 8))
    g.set_single_pass((0, 32, 8, 32))
    g.step(11)
    ref = _snapshot(g)
    tunes = [(1, 32, 8, 64), (1, 32, 4, 8), (1, 64, 8, 5), (1, 64, 4, 1), (1, 32, 8, 3)]
    for tune in tunes:
        g.load_state(blob)
        g.set_single_pass(tune)
        assert g.single_pass() == tune
        g.step(11)                     # ends in the second copy
        _assert_same(ref, _snapshot(g), f"single pass {tune}")
        g.load_state(blob)
        for _ in range(11):
            g.step(1)                  # one step per call, the copy flips each time
        _assert_same(ref, _snapshot(g), f"single pass {tune}, step by step")
        g.load_state(blob)
        g.step_timed(5)                # direct launches
        g.step(6)
        _assert_same(ref, _snapshot(g), f"single pass {tune}, timed + graphs")
    g.close()


def test_single_pass_dense_eps_map_bitwise():
    g = _setup((48, 24, 20), 4, seed=9, dense=True)
    g.step(3)
    blob = g.save_state()
    g.set_single_pass((0, 32, 8, 32))
    g.step(8)
    ref = _snapshot(g)
    g.load_state(blob)
    g.set_single_pass((1, 32, 8, 6))
    g.step(8)
    _assert_same(ref, _snapshot(g), "dense eps")
    g.close()


def test_single_pass_workload_48_oracle_parity():
    """48^3 workload, 500 steps with the single-pass step, against the oracle."""
    from paper_0809_1547_gb300 import inputs
    w = inputs.workload_small_48()
    o, g = make_pair(w.grid, w.eps, w.gain, w.N_a, w.pump, w.seed, params_kw(npml=w.npml))
    g.set_single_pass((1, 32, 8, 16))
    pid = g.add_point_probe(w.extra["probe"], 64, 475e-9, 705e-9)
    o.add_point_probe(w.extra["probe"], 64, 475e-9, 705e-9)
    o.step(w.steps)
    g.step(w.steps)
    errs = assert_fields_match(o, g)
    assert errs["Ex"] > 0
    S_o, _ = o.probe_spectrum(pid)
    S_g, _ = g.probe_spectrum(pid)
    assert np.linalg.norm(S_g - S_o) <= 2e-5 * np.linalg.norm(S_o)
    per_step, total = g.launch_stats()
    assert per_step == 2                     # the step and the point probe
    g.close()


def test_single_pass_argument_errors():
    from paper_0809_1547_gb300.binding import MBSimulation, mb_default_params, MBError, MB_ERR_ARG
    g = MBSimulation((8, 8, 8), DX, DT, mb_default_params(npml=2))
    with pytest.raises(MBError) as e:
        g.set_single_pass((1, 32, 8, 8))        # n_x % 16 != 0
    assert e.value.code == MB_ERR_ARG
    g.close()
    g = MBSimulation((32, 8, 8), DX, DT, mb_default_params(npml=2))
    for bad in ((1, 128, 2, 8), (1, 32, 16, 8), (1, 32, 8, 0), (2, 32, 8, 8)):
        with pytest.raises(MBError) as e:
            g.set_single_pass(bad)
        assert e.value.code == MB_ERR_ARG
    assert g.single_pass()[0] == 0
    g.set_single_pass((1, 32, 4, 4))
    assert g.single_pass() == (1, 32, 4, 4)
    g.set_single_pass((0, 32, 4, 4))
    assert g.single_pass()[0] == 0
    g.close()


def test_single_pass_state_in_second_copy():
    """Odd step counts leave the state in the second copy: reads, writes,
    snapshots, mode switches and the adjoint all see the current state."""
    grid, npml = (48, 20, 18), 4
    g = _setup(grid, npml, seed=21)
    r = _setup(grid, npml, seed=21)
    g.set_single_pass((1, 32, 4, 5))
    r.set_single_pass((0, 32, 4, 5))
    for sim in (g, r):
        sim.step(3)
    _assert_same(_snapshot(r), _snapshot(g), "after 3 steps")
    blob = g.save_state()
    v = g.field("Ey")
    v[5:9, 6:10, 20:30] += 1e3
    for sim in (g, r):
        sim.set_field("Ey", v)
        sim.step(5)
    _assert_same(_snapshot(r), _snapshot(g), "after set_field + 5 steps")
    for sim in (g, r):
        sim.load_state(blob)
        sim.step(1)
    g.set_single_pass((0, 32, 4, 5))
    for sim in (g, r):
        sim.step(2)
    _assert_same(_snapshot(r), _snapshot(g), "two passes from the second copy")
    g.set_single_pass((1, 64, 4, 7))
    for sim in (g, r):
        sim.step(1)
    res = [sim.adjoint_energy_zface(12, 4) for sim in (g, r)]
    # same forward states; the FP64 sums of J and dJ/dW_p add in atomic order
    assert res[0][0] == pytest.approx(res[1][0], rel=1e-12, abs=0)
    assert res[0][2] == pytest.approx(res[1][2], rel=1e-12, abs=0)
    ga, gb = res[0][1].cpu().numpy(), res[1][1].cpu().numpy()
    np.testing.assert_allclose(ga, gb, rtol=1e-6, atol=1e-6 * np.abs(gb).max())
    assert g.single_pass() == (1, 64, 4, 7)
    for sim in (g, r):
        sim.step(3)
    _assert_same(_snapshot(r), _snapshot(g), "after the adjoint")
    g.close()
    r.close()


def test_flux_async_matches_flux():
    """The asynchronous read-back of the face energies equals the synchronous one."""
    import torch
    g = _setup((32, 20, 18), 4, seed=33)
    g.set_single_pass((1, 32, 4, 4))
    out = torch.zeros(6, dtype=torch.float64).pin_memory()
    for _ in range(3):
        g.step(5)
        g.flux_async(out)
        g.synchronize()
        ref = g.flux()
        np.testing.assert_array_equal(out.numpy(), ref)
    assert np.abs(ref).max() > 0
    with pytest.raises(ValueError):
        g.flux_async(torch.zeros(6, dtype=torch.float32))
    g.close()


def test_flux_async_pinned_and_pageable():
    """Page-locked output is written by the summing kernel directly, other
    host memory through a copy: both equal the synchronous read."""
    import torch
    g = _setup((32, 20, 18), 4, seed=35)
    g.set_single_pass((1, 32, 4, 4))
    pinned = torch.zeros(6, dtype=torch.float64).pin_memory()
    pageable = torch.zeros(6, dtype=torch.float64)
    for _ in range(3):
        g.step(3)
        g.flux_async(pinned)
        g.flux_async(pageable)
        g.synchronize()
        ref = g.flux()
        np.testing.assert_array_equal(pinned.numpy(), ref)
        np.testing.assert_array_equal(pageable.numpy(), ref)
    assert np.abs(ref).max() > 0
    g.close()


def test_single_steps_with_deferred_probes_bitwise():
    """Single steps leave their probe DFTs running beside the next step; reads
    of spectra, fields and energies between them, face-energy reads after
    every step, a save / load and an explicit join give the same bits as
    whole chunks."""
    import torch
    grid, npml = (64, 20, 24), 4
    g = _setup(grid, npml, seed=41)
    r = _setup(grid, npml, seed=41)
    for sim in (g, r):
        sim.set_single_pass((1, 32, 4, 8))
    r.step(37)
    ref = _snapshot(r)
    out = torch.zeros(6, dtype=torch.float64).pin_memory()
    blob = None
    for s in range(37):
        g.step(1)
        g.flux_async(out)
        if s % 5 == 2:
            g.probe_spectrum(0)
            g.face_spectrum(3)
        if s % 7 == 4:
            g.field("Ez")
            g.energy()
        if s == 20:
            blob = g.save_state()
            g.load_state(blob)
        if s % 6 == 1:
            g.join_probes()
            ev = torch.cuda.Event()
            ev.record(torch.cuda.current_stream())
            ev.synchronize()
    g.synchronize()
    _assert_same(ref, _snapshot(g), "single steps, deferred probes")
    np.testing.assert_array_equal(out.numpy(), r.flux())
    # from the saved state: single steps then a chunk, against the reference
    g.load_state(blob)
    for _ in range(3):
        g.step(1)
    g.step(16)                         # waits for the probes left by the single steps
    r.load_state(blob)
    r.step(19)
    _assert_same(_snapshot(r), _snapshot(g), "single steps then a chunk")
    g.close()
    r.close()


@pytest.mark.parametrize("grid,npml,tune", [
    ((16, 5, 3), 1, (1, 32, 4, 2)),     # narrower than a tile, ragged y, three planes
    ((32, 1, 1), 0, (1, 32, 8, 4)),     # one row, one plane, no CPML
    ((48, 9, 2), 2, (1, 64, 8, 1)),     # a tile wider than the grid, one-plane chunks
    ((16, 16, 40), 8, (1, 32, 4, 64)),  # all-CPML cross-section, chunk longer than n_z
])
def test_single_pass_small_and_degenerate_grids_bitwise(grid, npml, tune):
    from paper_0809_1547_gb300.binding import MBSimulation, mb_default_params
    shp = grid[::-1]
    rng = np.random.default_rng(sum(grid))
    eps = np.where(rng.random(shp) < 0.3, 8.41, 1.0).astype(np.float32)
    gain = (rng.random(shp) < 0.6).astype(np.uint8)
    sims = []
    for mode in ((0, 32, 4, 8), tune):
        g = MBSimulation(grid, DX, DT, mb_default_params(npml=npml))
        g.set_material(eps, gain, 4e24, 1e13)
        g.set_seed(91)
        g.set_single_pass(mode)
        rng2 = np.random.default_rng(5)
        for name in ("Ex", "Ey", "Ez"):
            v = (rng2.standard_normal(shp) * 1e6).astype(np.float32)
            if name != "Ex":
                v[:, :, 0] = 0
            if name != "Ey":
                v[:, 0, :] = 0
            if name != "Ez":
                v[0, :, :] = 0
            g.set_field(name, v)
        g.step(7)
        sims.append(g)
    for name in FIELD_NAMES:
        np.testing.assert_array_equal(sims[1].field(name), sims[0].field(name), err_msg=f"{grid} {name}")
    for g in sims:
        g.close()

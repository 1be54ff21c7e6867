"""CUDA path (through the C ABI) against the FP64 oracle on identical inputs.

Bar: every field within relative L2 1e-5 of the oracle after the run (the
bound stated for the FP32 step); squared read-outs (spectra, energy) within
2e-5; the Philox stream bit-exact.  Sizes span several thread blocks with
ragged tails, the degenerate grids (one-cell columns, all-CPML cubes), both
material encodings, and the full 320^3 and 448^3 workloads on sampled
sub-blocks.
"""
import math

import numpy as np
import pytest

from oracle.mb_oracle import MBOracle, Params, philox4x32_10, FIELD_NAMES, C0, MU0
from parity_util import DX, DT, REL_L2_TOL, params_kw, make_pair, rel_l2, assert_fields_match, \
    check_blocks_one_step

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_0809_1547_gb300 import build
    build.build()


def test_philox_device_bit_exact():
    from paper_0809_1547_gb300.binding import mb_philox4x32_10
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    for key in ((0, 0), (0xFFFFFFFF, 0xFFFFFFFF), (0xA4093822, 0x299F31D0), (0x5EED, 0)):
        dev = mb_philox4x32_10(ctr, key)
        ref = np.stack(philox4x32_10(ctr[:, 0], ctr[:, 1], ctr[:, 2], ctr[:, 3], *key), axis=1)
        np.testing.assert_array_equal(dev, ref)


def _spectrum_check(o, g, pid):
    S_o, lam_o = o.probe_spectrum(pid)
    S_g, lam_g = g.probe_spectrum(pid)
    np.testing.assert_allclose(lam_g, lam_o, rtol=1e-15)
    assert rel_l2(S_g, S_o) <= 2 * REL_L2_TOL


def _energy_check(o, g):
    U_g, fl_g = g.energy()
    U_o = o.energy()
    assert abs(U_g - U_o) <= 2 * REL_L2_TOL * U_o
    scale = np.abs(o.flux).max()
    if scale > 0:
        assert np.abs(fl_g - o.flux).max() <= 2 * REL_L2_TOL * scale


def test_workload_48_parity_500_steps():
    """48^3, 8-cell CPML, 8 spheres, gain in the voids, Langevin noise, 500 steps."""
    from paper_0809_1547_gb300 import inputs
    w = inputs.workload_small_48()
    pkw = params_kw(npml=w.npml)
    o, g = make_pair(w.grid, w.eps, w.gain, w.N_a, w.pump, w.seed, pkw)
    pid_o = o.add_point_probe(w.extra["probe"], 64, 475e-9, 705e-9)
    pid_g = g.add_point_probe(w.extra["probe"], 64, 475e-9, 705e-9)
    o.step(w.steps)
    g.step(w.steps)
    errs = assert_fields_match(o, g)
    assert errs["Ex"] > 0            # the comparison is not vacuous
    assert np.abs(o.field("Jx")).max() > 0 and np.abs(o.field("N2")).max() > 0
    _spectrum_check(o, g, pid_o)
    _energy_check(o, g)
    g.close()


@pytest.mark.parametrize("grid,npml,steps", [
    ((17, 23, 31), 3, 80),       # ragged in every direction
    ((40, 9, 13), 4, 60),
])
def test_ragged_grid_parity(grid, npml, steps):
    from paper_0809_1547_gb300 import inputs
    eps, gain = inputs.random_small(grid, seed=sum(grid), npml=npml, fill=0.35, d_cells=5)
    pkw = params_kw(npml=npml)
    o, g = make_pair(grid, eps, gain, 5e24, 1e13, 0xC0FFEE + sum(grid), pkw)
    src = (grid[0] // 2, grid[1] // 2, grid[2] // 2)
    for sim in (o, g):
        sim.add_point_probe((grid[0] // 3, grid[1] // 2, grid[2] // 2), 24, 450e-9, 750e-9)
        sim.add_face_probes(2, 3, 16, 480e-9, 700e-9)
    o.add_source(src, 1, 532e-9, 1.5e-15, 0.5e-15, 1e9)
    g.set_source(src, 1, 532e-9, 1.5e-15, 0.5e-15, 1e9)
    o.step(steps)
    g.step(steps)
    assert_fields_match(o, g)
    _spectrum_check(o, g, 0)
    _energy_check(o, g)
    for face in range(6):
        S_o, _ = o.face_spectrum(face)
        S_g, _ = g.face_spectrum(face)
        scale = max(np.abs(S_o).max(), 1e-300)
        assert np.abs(S_g - S_o).max() <= 4 * REL_L2_TOL * scale, face
    g.close()


def test_reset_probes_gives_the_window_spectra():
    """mb_reset_probes after 50 of 110 steps (a source pulse centred near
    step 39): the point-, face- and plane-probe spectra equal the oracle's
    with its DFT sums zeroed at the same step (the window's samples only);
    the face energies are kept."""
    from paper_0809_1547_gb300 import inputs
    grid, npml = (24, 20, 28), 4
    eps, gain = inputs.random_small(grid, seed=7, npml=npml, fill=0.35, d_cells=5)
    o, g = make_pair(grid, eps, gain, 5e24, 1e13, 0xBEEF, params_kw(npml=npml))
    src = (12, 10, 14)
    for sim in (o, g):
        sim.add_point_probe((8, 10, 14), 24, 450e-9, 750e-9)
        sim.add_face_probes(2, 3, 16, 480e-9, 700e-9)
        sim.add_plane_probe(14, 2, 4, 500e-9, 650e-9)
    o.add_source(src, 1, 532e-9, 1.5e-15, 0.5e-15, 1e9)
    g.set_source(src, 1, 532e-9, 1.5e-15, 0.5e-15, 1e9)
    o.step(50)
    g.step(50)
    S_first, _ = g.probe_spectrum(0)
    g.reset_probes()
    for pr in o.point_probes:
        pr["acc"][:] = 0
    for pp in o.plane_probes:
        pp["acc"][:] = 0
    for acc in o.face_probes["faces"].values():
        acc[:] = 0
    flux_before = o.flux.copy()
    o.step(60)
    g.step(60)
    assert_fields_match(o, g)
    _spectrum_check(o, g, 0)
    _energy_check(o, g)
    assert np.abs(o.flux - flux_before).max() > 0 and np.abs(flux_before).max() > 0
    for face in range(6):
        S_o, _ = o.face_spectrum(face)
        S_g, _ = g.face_spectrum(face)
        scale = max(np.abs(S_o).max(), 1e-300)
        assert np.abs(S_g - S_o).max() <= 4 * REL_L2_TOL * scale, face
    for b in range(4):
        M_o = o.plane_mode_map(0, b)
        M_g = g.plane_mode_map(0, b)
        assert M_o.max() > 0
        assert rel_l2(M_g, M_o) <= 4 * REL_L2_TOL, b
    # the sums did restart: the window's spectrum is not the first 50 steps'
    S_win, _ = g.probe_spectrum(0)
    assert S_first.max() > 0 and rel_l2(S_win, S_first) > 1e-3
    g.close()


@pytest.mark.parametrize("grid,npml", [((1, 1, 40), 0), ((1, 1, 40), 8), ((8, 8, 8), 8), ((2, 3, 1), 1)])
def test_degenerate_grids_parity(grid, npml):
    """One-cell columns (PEC zeroes every E), overlapping CPML slabs, a 1-cell-thick slab."""
    shp = grid[::-1]
    rng = np.random.default_rng(4)
    eps = np.where(rng.random(shp) < 0.3, 8.41, 1.0).astype(np.float32)
    gain = np.ones(shp, dtype=np.uint8)
    pkw = params_kw(npml=npml)
    o, g = make_pair(grid, eps, gain, 2e24, 1e13, 77, pkw)
    rng2 = np.random.default_rng(5)
    # a physical start: tangential E vanishes on the PEC planes i = 0, j = 0, k = 0
    # (a wall value there would leave a static field whose CPML response is
    # the difference of two nearly equal terms, beyond FP32 resolution)
    for name in ("Ex", "Ey", "Ez"):
        v = (rng2.standard_normal(shp) * 1e6).astype(np.float32)
        if name != "Ex":
            v[:, :, 0] = 0
        if name != "Ey":
            v[:, 0, :] = 0
        if name != "Ez":
            v[0, :, :] = 0
        o.set_field(name, v.astype(np.float64))
        g.set_field(name, v)
    o.step(50)
    g.step(50)
    assert_fields_match(o, g)
    g.close()


def test_dense_eps_map_parity():
    """More than 128 distinct eps values switch the device to a dense 1/eps map."""
    grid = (20, 18, 16)
    shp = grid[::-1]
    rng = np.random.default_rng(8)
    eps = rng.uniform(1.0, 8.41, size=shp).astype(np.float32)
    gain = (rng.random(shp) < 0.5).astype(np.uint8)
    o, g = make_pair(grid, eps, gain, 3e24, 1e13, 99, params_kw(npml=3))
    o.step(60)
    g.step(60)
    assert_fields_match(o, g)
    g.close()


def test_cavity_eigenmode_closed_form():
    """The exact discrete PEC-cavity mode, run on the GPU, against its closed form."""
    from paper_0809_1547_gb300.binding import MBSimulation, mb_default_params
    grid = (24, 20, 28)
    modes, amp_dir, eps_r = (2, 1, 3), (0.3, -0.7, 1.1), 2.0
    nx, ny, nz = grid
    k = [m * math.pi / (nw * DX) for m, nw in zip(modes, grid)]
    s = np.array([2 / DX * math.sin(kw * DX / 2) for kw in k])
    A = np.cross(s, amp_dir)
    A /= np.linalg.norm(A)
    omega = 2 / DT * math.asin(DT / 2 * C0 / math.sqrt(eps_r) * np.linalg.norm(s))
    B = -(DT / MU0) * np.cross(s, A) / (2 * math.sin(omega * DT / 2))
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    S, Co = np.sin, np.cos

    def fields(n, te=None, th=None):
        te = math.cos(omega * n * DT) if te is None else te
        th = math.sin(omega * (n - 0.5) * DT) if th is None else th
        xi, yi, zi = ii * DX, jj * DX, kk * DX
        xh, yh, zh = (ii + .5) * DX, (jj + .5) * DX, (kk + .5) * DX
        return {"Ex": A[0] * Co(k[0] * xh) * S(k[1] * yi) * S(k[2] * zi) * te,
                "Ey": A[1] * S(k[0] * xi) * Co(k[1] * yh) * S(k[2] * zi) * te,
                "Ez": A[2] * S(k[0] * xi) * S(k[1] * yi) * Co(k[2] * zh) * te,
                "Hx": B[0] * S(k[0] * xi) * Co(k[1] * yh) * Co(k[2] * zh) * th,
                "Hy": B[1] * Co(k[0] * xh) * S(k[1] * yi) * Co(k[2] * zh) * th,
                "Hz": B[2] * Co(k[0] * xh) * Co(k[1] * yh) * S(k[2] * zi) * th}

    g = MBSimulation(grid, DX, DT, mb_default_params(npml=0))
    g.set_material(np.full(grid[::-1], eps_r, np.float32), np.zeros(grid[::-1], np.uint8), 0.0, 0.0)
    for name, v in fields(0).items():
        g.set_field(name, v)
    n = 300
    g.step(n)
    # errors are measured against the mode's amplitude: at a temporal node the
    # instantaneous field is ~0 and a relative norm of it would mean nothing
    amp = {name: np.linalg.norm(v) for name, v in fields(0, te=1.0, th=1.0).items()}
    ampE = max(amp["Ex"], amp["Ey"], amp["Ez"])
    ampH = max(amp["Hx"], amp["Hy"], amp["Hz"])
    for name, v in fields(n).items():
        scale = ampE if name[0] == "E" else ampH
        assert np.linalg.norm(g.field(name) - v) <= 1e-5 * scale, name
    g.close()


def test_graph_chunks_equal_single_steps_bitwise():
    from paper_0809_1547_gb300 import inputs
    grid = (24, 20, 18)
    eps, gain = inputs.random_small(grid, seed=2, npml=4)
    pkw = params_kw(npml=4)
    _, a = make_pair(grid, eps, gain, 4e24, 1e13, 5, pkw)
    _, b = make_pair(grid, eps, gain, 4e24, 1e13, 5, pkw)
    a.step(37)
    for _ in range(37):
        b.step(1)
    for name in FIELD_NAMES:
        np.testing.assert_array_equal(a.field(name), b.field(name))
    a.close()
    b.close()


@pytest.mark.parametrize("grid", [(64, 20, 24), (96, 17, 13)])
def test_launch_variants_are_bitwise_identical(grid):
    """3-D tiles, z-walks, TMA-staged and quad-vectorised passes give the same bits."""
    from paper_0809_1547_gb300 import inputs
    eps, gain = inputs.random_small(grid, seed=6, npml=4, d_cells=5)
    pkw = params_kw(npml=4)
    _, g = make_pair(grid, eps, gain, 4e24, 1e13, 11, pkw)
    g.set_source((grid[0] // 2, grid[1] // 2, grid[2] // 2), 2, 532e-9, 1.5e-15, 0.5e-15, 1e9)
    g.add_face_probes(2, 1, 8, 500e-9, 650e-9)
    g.step(4)
    blob = g.save_state()
    ref_tune = ((1, 32, 4, 8), (1, 32, 4, 8))
    tunes = [((0, 32, 4, 2), (0, 32, 4, 2)), ((3, 32, 4, 8), (3, 32, 4, 8)),
             ((3, 64, 2, 16), (3, 32, 8, 4)), ((1, 64, 2, 4), (1, 32, 2, 16))]
    if grid[0] % 16 == 0:
        tunes += [((1, 32, 4, 8), (2, 32, 4, 8)), ((1, 32, 4, 8), (2, 64, 8, 16)),
                  ((2, 32, 4, 8), (1, 32, 4, 8)), ((2, 64, 8, 16), (2, 32, 8, 4)),
                  ((2, 128, 2, 3), (0, 32, 4, 2)), ((2, 32, 8, 64), (2, 128, 4, 5))]
    results = {}
    for tune in [ref_tune] + tunes:
        g.load_state(blob)
        g.set_tuning(*tune)
        g.step(9)
        results[tune] = {name: g.field(name) for name in FIELD_NAMES}
    for tune in tunes:
        for name in FIELD_NAMES:
            a, b = results[ref_tune][name], results[tune][name]
            if not np.array_equal(a, b):
                where = np.argwhere(a != b)[0]
                raise AssertionError(f"{tune} differs in {name} at [k,j,i]={tuple(where)}: "
                                     f"{a[tuple(where)]!r} vs {b[tuple(where)]!r}")
    g.close()


def test_save_load_state_roundtrip_bitwise():
    from paper_0809_1547_gb300 import inputs
    grid = (22, 21, 20)
    eps, gain = inputs.random_small(grid, seed=3, npml=4)
    _, g = make_pair(grid, eps, gain, 4e24, 1e13, 6, params_kw(npml=4))
    g.add_point_probe((10, 10, 10), 8, 500e-9, 650e-9)
    # face probes every step: the save at step 10 falls between two flushes
    # of their FP32 partial sums (every 16th call), so the blob must hold them
    g.add_face_probes(2, 1, 8, 500e-9, 650e-9)
    g.set_source((11, 10, 10), 2, 532e-9, 1.5e-15, 0.5e-15, 1e9)
    g.step(10)
    blob = g.save_state()
    g.step(15)
    ref = {name: g.field(name) for name in FIELD_NAMES}
    S_ref, _ = g.probe_spectrum(0)
    F_ref = [g.face_spectrum(face)[0] for face in range(6)]
    assert max(float(np.abs(F).max()) for F in F_ref) > 0
    g.load_state(blob)
    assert g.n == 10
    g.step(15)
    for name in FIELD_NAMES:
        np.testing.assert_array_equal(g.field(name), ref[name])
    np.testing.assert_array_equal(g.probe_spectrum(0)[0], S_ref)
    for face in range(6):
        np.testing.assert_array_equal(g.face_spectrum(face)[0], F_ref[face])
    g.close()


def test_autotune_keeps_state_and_results():
    from paper_0809_1547_gb300 import inputs
    grid = (40, 36, 30)
    eps, gain = inputs.random_small(grid, seed=4, npml=6)
    pkw = params_kw(npml=6)
    _, a = make_pair(grid, eps, gain, 4e24, 1e13, 8, pkw)
    _, b = make_pair(grid, eps, gain, 4e24, 1e13, 8, pkw)
    a.step(5)
    b.step(5)
    before = {name: a.field(name) for name in FIELD_NAMES}
    a.autotune()
    for name in FIELD_NAMES:
        np.testing.assert_array_equal(a.field(name), before[name])
    a.step(20)
    b.step(20)
    for name in FIELD_NAMES:
        np.testing.assert_array_equal(a.field(name), b.field(name))
    a.close()
    b.close()


def test_gpu_energy_balance_of_interior_box():
    """Lossless interior, source off: box energy change = -(outward flux), on the GPU."""
    from paper_0809_1547_gb300.binding import MBSimulation, mb_default_params
    from oracle.mb_oracle import EPS0
    grid = (30, 28, 32)
    shp = grid[::-1]
    eps = np.ones(shp, np.float32)
    eps[14:18, 13:17, 15:19] = 4.0
    g = MBSimulation(grid, DX, DT, mb_default_params(npml=8))
    g.set_material(eps, np.zeros(shp, np.uint8), 0.0, 0.0)
    g.set_source((15, 14, 16), 0, 400e-9, 1.2e-15, 0.4e-15, 1e9)
    g.step(45)
    g.set_source((15, 14, 16), 0, 400e-9, 1.2e-15, 0.4e-15, 0.0)

    def box_energy():
        L = 8
        sl = (slice(L, grid[2] - L), slice(L, grid[1] - L), slice(L, grid[0] - L))
        E = [g.field(n).astype(np.float64) for n in ("Ex", "Ey", "Ez")]
        Hm = [g.field(n).astype(np.float64) for n in ("Hx", "Hy", "Hz")]
        _, fl = g.energy()
        g.step(1)
        Hp = [g.field(n).astype(np.float64) for n in ("Hx", "Hy", "Hz")]
        uE = sum(np.sum((eps * F * F)[sl]) for F in E) * EPS0
        uH = sum(np.sum((a * b)[sl]) for a, b in zip(Hm, Hp)) * MU0
        return 0.5 * (uE + uH) * DX ** 3, fl

    W1, F1 = box_energy()
    g.step(60)
    W2, F2 = box_energy()
    out = float(np.sum(F2 - F1))
    assert out > 0.2 * W1
    assert abs((W1 - W2) - out) < 1e-4 * W1
    g.close()


def test_nonfinite_fields_are_reported():
    from paper_0809_1547_gb300.binding import MBSimulation, mb_default_params, MBError, MB_ERR_NONFINITE
    grid = (8, 8, 8)
    g = MBSimulation(grid, DX, DT, mb_default_params(npml=2))
    v = np.zeros(grid[::-1], np.float32)
    v[3, 3, 3] = np.nan
    g.set_field("Hy", v)
    with pytest.raises(MBError) as e:
        g.energy()
    assert e.value.code == MB_ERR_NONFINITE
    g.close()


def test_material_values_in_runs_parity():
    """Six eps_r values in runs of random length (so 64-cell blocks see one,
    several or a new value, and the value table outgrows four entries part
    way through), over two host threads' chunks: 12 steps within the bound
    of the oracle."""
    grid = (80, 64, 64)                       # 327,680 cells: two host threads
    rng = np.random.default_rng(77)
    n = grid[0] * grid[1] * grid[2]
    vals = np.array([1.0, 8.41, 2.25, 1.0, 5.5, 3.1, 6.25, 8.41], np.float32)
    lens = rng.integers(1, 200, size=n // 20)
    idx = np.repeat(rng.integers(0, 3, size=lens.size), lens)[:n]
    idx[n // 3:] = np.repeat(rng.integers(0, len(vals), size=lens.size), lens)[:n - n // 3]
    eps = vals[idx].reshape(grid[::-1])
    gain = (rng.random(grid[::-1]) < 0.5).astype(np.uint8)
    pkw = params_kw(npml=4)
    o, g = make_pair(grid, eps, gain, 4e24, 1e13, 9, pkw)
    g.set_source((40, 32, 32), 2, 532e-9, 1.0e-15, 0.4e-15, 1e9)
    o.add_source((40, 32, 32), 2, 532e-9, 1.0e-15, 0.4e-15, 1e9)
    g.step(12)
    o.step(12)
    assert_fields_match(o, g)
    n0 = g.field("N0")
    assert np.array_equal(n0 != 0, gain != 0)
    g.close()


def test_rejected_material_keeps_state():
    """A rejected eps map (a NaN in the last host thread's chunk) changes
    nothing: the N0 read-out and the next steps equal those of a twin that
    never saw it; a later valid call replaces the material as usual."""
    from paper_0809_1547_gb300 import inputs
    from paper_0809_1547_gb300.binding import MBError, MB_ERR_MATERIALS
    grid = (80, 64, 64)                       # 327,680 cells: two host threads
    eps, gain = inputs.random_small(grid, seed=3, npml=4)
    pkw = params_kw(npml=4)
    sims = [make_pair(grid, eps, gain, 4e24, 1e13, 5, pkw)[1] for _ in range(2)]
    g, r = sims
    for sim in sims:
        sim.step(6)
    n0 = g.field("N0")
    assert np.abs(n0).max() > 0
    bad = eps.copy()
    bad[60, 40, 7] = np.nan
    with pytest.raises(MBError) as e:
        g.set_material(bad, (1 - gain).astype(np.uint8), 2e24, 1e13)
    assert e.value.code == MB_ERR_MATERIALS
    np.testing.assert_array_equal(g.field("N0"), n0)
    for sim in sims:
        sim.step(5)
    for name in FIELD_NAMES:
        np.testing.assert_array_equal(g.field(name), r.field(name), err_msg=name)
    eps2 = np.where(eps > 1.0, np.float32(6.25), np.float32(1.0))
    for sim in sims:
        sim.set_material(eps2, gain, 3e24, 1e13)
        sim.step(4)
    for name in FIELD_NAMES:
        np.testing.assert_array_equal(g.field(name), r.field(name), err_msg=name)
    g.close()
    r.close()


def test_argument_errors():
    from paper_0809_1547_gb300.binding import MBSimulation, mb_default_params, MBError, MB_ERR_ARG, \
        MB_ERR_MATERIALS
    grid = (8, 8, 8)
    g = MBSimulation(grid, DX, DT, mb_default_params(npml=2))
    with pytest.raises(MBError) as e:
        g.add_point_probe((8, 0, 0), 4, 500e-9, 600e-9)
    assert e.value.code == MB_ERR_ARG
    with pytest.raises(MBError) as e:
        g.set_material(np.full(grid[::-1], 0.5, np.float32), np.zeros(grid[::-1], np.uint8), 1e24, 0)
    assert e.value.code == MB_ERR_MATERIALS
    with pytest.raises(MBError):
        g.set_field("N0", np.zeros(grid[::-1], np.float32))
    for bad in (((2, 32, 4, 8), (1, 32, 4, 8)),       # TMA passes need n_x % 16 == 0
                ((1, 48, 4, 8), (1, 32, 4, 8)),       # x not a multiple of 32
                ((2, 32, 16, 8), (1, 32, 4, 8))):     # no such TMA tile (and n_x = 8)
        with pytest.raises(MBError) as e:
            g.set_tuning(*bad)
        assert e.value.code == MB_ERR_ARG
    g.close()


def _sampled_step_parity(w, n_pre, los, B):
    """Advance workload w by n_pre steps in the launch configuration the
    benchmark times (autotuned), then check one more GPU step on the
    sub-blocks of edge B + 2 starting at los against the oracle's step of the
    same block (the whole grid's CPML profiles, the GPU's CPML memories, the
    whole grid's noise counters and step index; a one-cell halo left out
    except along the grid's own walls); then properties that hold at any
    size."""
    import torch
    from paper_0809_1547_gb300.workloads import setup_simulation
    g = setup_simulation(w, autotune=True)
    g.step(n_pre)
    g.synchronize()

    def one():
        g.step(1)
        g.synchronize()
    worst = check_blocks_one_step(g, w, one, los, B + 2, params_kw(npml=w.npml))
    U, fl = g.energy()
    assert math.isfinite(U) and np.all(np.isfinite(fl))
    t, _ = g.field_device("Jx")
    nongain = torch.from_numpy(w.gain == 0).cuda()
    assert float(t[nongain].abs().max()) == 0.0
    g.close()
    return worst


def _boundary_blocks(n, L, size):
    """Blocks of edge `size` touching the grid's boundary layers: both
    corners (the PEC walls and all six CPML slabs with their interfaces and
    the flux box's face planes), and one straddling each CPML interface on
    each axis away from the corners."""
    hi = n - size
    mid = n // 2 - size // 2
    cut_lo = max(0, L - size // 2)            # straddles the interface at L
    cut_hi = min(n - size, n - L - size // 2)  # straddles the interface at n - L
    return [(0, 0, 0), (hi, hi, hi),
            (cut_lo, mid, mid), (cut_hi, mid, mid), (mid, cut_lo, mid), (mid, cut_hi, mid),
            (mid, mid, cut_lo), (mid, mid, cut_hi), (0, hi, mid), (hi, mid, 0)]


def test_full_size_320_sampled_parity():
    """The 320^3 workload (~8100 spheres, 32.8 M cells) after 24 steps: one
    more step checked on three random interior sub-blocks, the centre and
    ten blocks on the walls, corners and CPML interfaces (fields and CPML
    memories)."""
    from paper_0809_1547_gb300 import inputs
    w = inputs.workload_paper_320()
    B = 20
    rng = np.random.default_rng(12)
    los = [tuple(int(v) for v in rng.integers(9, 320 - 9 - B - 2, size=3)) for _ in range(3)]
    los.append((150, 150, 150))
    los += _boundary_blocks(320, w.npml, B + 2)
    _sampled_step_parity(w, 24, los, B)


def test_full_size_448_sampled_parity():
    """The 448^3 sweep workload (~22.9k spheres, 89.9 M cells, 5.8 GB of
    state) after 16 steps: one more step checked on sub-blocks at random
    interior positions, across tile and plane-chunk boundaries (x = 31|32,
    y = 3|4, z = 15|16 of the launch's tiles), at the far interior corner
    and on the walls, corners and CPML interfaces."""
    from paper_0809_1547_gb300 import inputs
    w = inputs.workload_large_448()
    B = 16
    rng = np.random.default_rng(448)
    los = [tuple(int(v) for v in rng.integers(9, 448 - 9 - B - 2, size=3)) for _ in range(2)]
    los += [(216, 214, 214), (448 - 9 - B - 2,) * 3]
    los += _boundary_blocks(448, w.npml, B + 2)
    _sampled_step_parity(w, 16, los, B)
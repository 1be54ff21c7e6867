"""Seeded input generators: packings are disjoint, deterministic and hit their fill."""
import numpy as np

from paper_0809_1547_gb300 import inputs


def test_packing_is_disjoint_and_seeded():
    box = np.array([1.2e-6] * 3)
    c1, r1 = inputs.sphere_packing(box, 120, 300e-9 / 2, 0.1, seed=4)
    c2, r2 = inputs.sphere_packing(box, 120, 300e-9 / 2, 0.1, seed=4)
    np.testing.assert_array_equal(c1, c2)
    d = np.linalg.norm(c1[:, None, :] - c1[None, :, :], axis=-1)
    s = r1[:, None] + r1[None, :]
    np.fill_diagonal(d, np.inf)
    assert np.all(d >= s - 1e-3 * 150e-9)
    assert np.all(c1 - r1[:, None] >= -1e-15) and np.all(c1 + r1[:, None] <= box + 1e-15)


def test_rasterize_staircase_rule():
    dx = 20e-9
    grid = (10, 10, 10)
    c = np.array([[5 * dx, 5 * dx, 5 * dx]])
    r = np.array([2.1 * dx])
    inside = inputs.rasterize(grid, dx, c, r)
    kk, jj, ii = np.meshgrid(*(np.arange(10),) * 3, indexing="ij")
    d2 = ((ii + .5) * dx - c[0, 0]) ** 2 + ((jj + .5) * dx - c[0, 1]) ** 2 + ((kk + .5) * dx - c[0, 2]) ** 2
    np.testing.assert_array_equal(inside, d2 < r[0] ** 2)


def test_material_maps_clear_gain_in_cpml():
    inside = np.zeros((12, 12, 12), bool)
    inside[5:7, 5:7, 5:7] = True
    eps, gain = inputs.material_maps((12, 12, 12), inside, 3)
    assert eps.dtype == np.float32 and gain.dtype == np.uint8
    assert np.all(eps[inside] == np.float32(8.41)) and np.all(eps[~inside] == 1)
    assert gain[:3].sum() == 0 and gain[-3:].sum() == 0 and gain[:, :, :3].sum() == 0
    assert np.all(gain[inside] == 0)
    assert gain[3:9, 3:9, 3:9].sum() == 6 ** 3 - 8


def test_material_maps_hold_the_background_in_the_cpml():
    # a sphere reaching into the layers is cut at their inner faces
    inside = np.zeros((12, 12, 12), bool)
    inside[1:6, 4:8, 4:8] = True          # k = 1, 2 lie in the z layers (npml = 3)
    eps, gain = inputs.material_maps((12, 12, 12), inside, 3)
    assert np.all(eps[:3] == 1) and np.all(eps[-3:] == 1)
    assert np.all(eps[:, :3] == 1) and np.all(eps[:, :, -3:] == 1)
    assert np.all(eps[3:6, 4:8, 4:8] == np.float32(8.41))
    assert gain[3:6, 4:8, 4:8].sum() == 0 and gain[:3].sum() == 0
    for w in (inputs.workload_small_48(), inputs.workload_adjoint_96()):
        L = w.npml
        for sl in ((slice(0, L),), (slice(-L, None),), (slice(None), slice(0, L)),
                   (slice(None), slice(None), slice(-L, None))):
            assert np.all(w.eps[sl] == 1) and w.gain[sl].sum() == 0


def test_workload_48_matches_its_description():
    w = inputs.workload_small_48()
    assert w.grid == (48, 48, 48) and w.n_spheres == 8 and w.steps == 500
    assert abs(w.fill - 8 * np.pi / 6 * 0.3 ** 3 / 0.96 ** 3) < 1e-9
    assert 0.1 < w.gain_fraction() < 0.3
    assert w.dt == inputs.courant_dt(20e-9)


def test_batch_workload_shapes():
    ws = inputs.workload_batch(n_pump=2, n_seed=2, side_lo=24, side_hi=32)
    assert len(ws) == 4
    assert all(24 <= w.grid[0] <= 32 for w in ws)
    assert ws[0].N_a < ws[1].N_a
    assert len({w.seed for w in ws}) == 4

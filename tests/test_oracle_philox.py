"""Pins of the oracle's Langevin noise generator (Philox4x32-10 + Box–Muller)."""
import os

import numpy as np
import pytest

from oracle.mb_oracle import philox4x32_10, u32_to_unit, langevin_normals

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            vals = [int(v, 16) for v in line.split()]
            rows.append((vals[:4], vals[4:6], vals[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answers(ctr, key, expect):
    out = philox4x32_10(*ctr, *key)
    assert [int(v) for v in out] == expect


def test_philox_vectorised_matches_scalar():
    rng = np.random.default_rng(3)
    c = rng.integers(0, 2 ** 32, size=(4, 64), dtype=np.uint64)
    k = [0x01234567, 0x89ABCDEF]
    vec = philox4x32_10(c[0], c[1], c[2], c[3], *k)
    for t in range(64):
        sc = philox4x32_10(int(c[0, t]), int(c[1, t]), int(c[2, t]), int(c[3, t]), *k)
        assert [int(v[t]) for v in vec] == [int(v) for v in sc]


def test_unit_map_is_open_interval_and_exact_in_fp32():
    x = np.array([0, 1, 511, 512, 2 ** 31, 2 ** 32 - 1], dtype=np.uint32)
    u = u32_to_unit(x)
    assert np.all(u > 0) and np.all(u < 1)
    assert u[0] == 0.5 * 2.0 ** -23
    assert u[-1] == 1.0 - 0.5 * 2.0 ** -23
    np.testing.assert_array_equal(u.astype(np.float32).astype(np.float64), u)


def test_box_muller_moments():
    n = 400_000
    z = np.concatenate(langevin_normals(0x5EED, np.arange(n), 7))
    m = z.size
    assert abs(z.mean()) < 5.0 / np.sqrt(m)
    assert abs(z.var() - 1.0) < 5.0 * np.sqrt(2.0 / m)
    kurt = np.mean(z ** 4) / np.mean(z ** 2) ** 2
    assert abs(kurt - 3.0) < 5.0 * np.sqrt(24.0 / m)
    # the three components of one cell are uncorrelated
    zx, zy, zz = langevin_normals(0x5EED, np.arange(n), 7)
    for a, b in ((zx, zy), (zx, zz), (zy, zz)):
        assert abs(np.mean(a * b)) < 5.0 / np.sqrt(n)


def test_counter_distinguishes_cell_step_seed():
    a = langevin_normals(1, np.arange(8), 0)[0]
    b = langevin_normals(1, np.arange(8), 1)[0]
    c = langevin_normals(2, np.arange(8), 0)[0]
    assert not np.allclose(a, b) and not np.allclose(a, c)
    # a 64-bit seed uses both key words
    d = langevin_normals(1 + (1 << 32), np.arange(8), 0)[0]
    assert not np.allclose(a, d)

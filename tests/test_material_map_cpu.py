"""The host half of mb_set_material (no GPU): material ids, gain bits and the
gain-cell list, through the mb_material_map diagnostic, against a plain
numpy statement of the same map.

The map: each cell's eps_r bit pattern gets the id of its value in order of
first appearance (more than 128 distinct values: dense, every id 0), bit 7
marks a gain cell when the gain is on, the gain list is the gain cells'
indices in increasing order, and any value that is not finite or below 1 is
rejected.  The cases drive the library's block fast path (64-cell blocks of
values seen before), its per-cell fallback (new values, more than four
values), the branch-free gain list, several host threads' chunks, and the
edges (sizes below and off a block, values at block and chunk ends).
"""
import numpy as np
import pytest

from paper_0809_1547_gb300.binding import MBError, MB_ERR_MATERIALS, mb_material_map


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_0809_1547_gb300 import build
    build.build()


def _reference(eps, gain, gain_on):
    eps = np.ascontiguousarray(eps, np.float32).reshape(-1)
    gain = np.ascontiguousarray(gain, np.uint8).reshape(-1)
    bits = eps.view(np.uint32)
    uniq, first = np.unique(bits, return_index=True)
    keys = uniq[np.argsort(first)]                      # order of first appearance
    dense = keys.size > 128
    if dense:
        ids = np.zeros(eps.size, np.uint8)
        values = np.zeros(0, np.float32)
    else:
        order = np.argsort(keys)                        # sorted position -> id
        ids = order[np.searchsorted(keys[order], bits)].astype(np.uint8)
        values = keys.view(np.float32)
    g = (gain != 0) & bool(gain_on)
    mat = ids | (g.astype(np.uint8) << 7)
    return mat, np.nonzero(g)[0].astype(np.uint32), values, dense


def _check(eps, gain, gain_on=True, threads=(1, 3, 16)):
    ref = _reference(eps, gain, gain_on)
    for t in threads:
        mat, glist, values, dense = mb_material_map(eps, gain, gain_on, t)
        np.testing.assert_array_equal(mat, ref[0], err_msg=f"material bytes, {t} threads")
        np.testing.assert_array_equal(glist, ref[1], err_msg=f"gain list, {t} threads")
        np.testing.assert_array_equal(values.view(np.uint32), ref[2].view(np.uint32), err_msg=f"values, {t}")
        assert dense == ref[3]


def _runs(n, values, rng, max_len=200):
    lens = rng.integers(1, max_len, size=n // 2 + 1)
    idx = np.repeat(rng.integers(0, len(values), size=lens.size), lens)[:n]
    return np.asarray(values, np.float32)[idx]


N_MULTI = 1_500_000          # several host threads (one per 2^18 cells at most)


def test_two_values_in_runs_across_blocks_and_threads():
    rng = np.random.default_rng(1)
    eps = _runs(N_MULTI, [1.0, 8.41], rng)
    gain = (rng.random(N_MULTI) < 0.45).astype(np.uint8)
    _check(eps, gain)


def test_values_beyond_four_and_late_first_appearances():
    rng = np.random.default_rng(2)
    eps = _runs(N_MULTI, [1.0, 8.41], rng)
    # new values appear late, inside blocks, in several threads' chunks
    for q, v in zip((300_001, 700_013, 1_100_063, 1_499_999, 64 * 5000), (2.25, 5.5, 3.1, 6.25, 7.0)):
        eps[q] = v
    eps[900_000:900_640] = _runs(640, [1.5, 2.5, 3.5, 4.5, 1.0], rng, 9)
    gain = (rng.random(N_MULTI) < 0.5).astype(np.uint8) * 3   # any non-zero byte marks gain
    _check(eps, gain)


def test_more_than_128_values_is_dense():
    rng = np.random.default_rng(3)
    eps = (1.0 + rng.random(400_000) * 9.0).astype(np.float32)
    gain = (rng.random(eps.size) < 0.3).astype(np.uint8)
    _check(eps, gain)
    eps = np.repeat(np.arange(1, 130, dtype=np.float32), 100)   # exactly 129 values
    _check(eps, np.ones(eps.size, np.uint8))


def test_gain_off_and_small_sizes():
    rng = np.random.default_rng(4)
    for n in (1, 7, 63, 64, 65, 129, 1000):
        eps = _runs(n, [1.0, 8.41, 2.0], rng, 20)
        gain = (rng.random(n) < 0.5).astype(np.uint8)
        _check(eps, gain, gain_on=True, threads=(1, 16))
        _check(eps, gain, gain_on=False, threads=(1, 16))
    ones = np.ones(64 * 1000, np.float32)
    _check(ones, np.ones(ones.size, np.uint8))                 # every cell a gain cell
    _check(ones, np.zeros(ones.size, np.uint8))                # none


def test_extreme_valid_values():
    eps = np.array([1.0, np.finfo(np.float32).max, np.nextafter(np.float32(1), np.float32(2)), 1.0] * 40,
                   np.float32)
    _check(eps, np.arange(eps.size, dtype=np.uint8) & 1)


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf, 0.5, 0.0, -0.0, -2.0,
                                 np.nextafter(np.float32(1), np.float32(0)), 1e-40])
@pytest.mark.parametrize("where", [0, 63, 64, 1000, N_MULTI // 2, N_MULTI - 1])
def test_invalid_values_are_rejected(bad, where):
    rng = np.random.default_rng(5)
    eps = _runs(N_MULTI, [1.0, 8.41], rng)
    eps[where] = bad
    gain = np.zeros(N_MULTI, np.uint8)
    with pytest.raises(MBError) as e:
        mb_material_map(eps, gain, True, 16)
    assert e.value.code == MB_ERR_MATERIALS


def test_reference_is_not_trivial():
    """The reference itself on a hand-made case: ids by first appearance."""
    eps = np.array([8.41, 1.0, 8.41, 2.0, 1.0], np.float32)
    gain = np.array([0, 1, 0, 1, 1], np.uint8)
    mat, glist, values, dense = _reference(eps, gain, True)
    np.testing.assert_array_equal(mat, [0, 1 | 0x80, 0, 2 | 0x80, 1 | 0x80])
    np.testing.assert_array_equal(glist, [1, 3, 4])
    np.testing.assert_array_equal(values, np.array([8.41, 1.0, 2.0], np.float32))
    assert not dense

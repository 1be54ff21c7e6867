"""Batched ensemble (one persistent launch over many realizations, or the
members' own launches on concurrent streams) against single-context
stepping and the oracle.

The batched kernel reuses the single path's per-cell updates, so every
member's fields must equal, bit for bit, the same realization stepped alone;
its point spectra too (each bin accumulates the same terms in the same
order).  The face flux sums FP64 atomics in another order: 1e-9 relative.
The two modes give the same bits.  One member is also checked directly
against the FP64 oracle.
"""
import numpy as np
import pytest

from oracle.mb_oracle import FIELD_NAMES
from parity_util import DX, DT, params_kw, make_pair, assert_fields_match

pytestmark = pytest.mark.gpu

GRIDS = [(40, 36, 32), (33, 41, 17), (24, 22, 20), (1, 1, 40)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_0809_1547_gb300 import build
    build.build()


def _members(grids, npml):
    from paper_0809_1547_gb300 import inputs
    out = []
    for q, grid in enumerate(grids):
        if min(grid) >= 8:
            eps, gain = inputs.random_small(grid, seed=100 + q, npml=npml, d_cells=5)
        else:
            eps = np.ones(grid[::-1], np.float32)
            gain = np.ones(grid[::-1], np.uint8)
        out.append(dict(grid=grid, eps=eps, gain=gain, N_a=(2 + q) * 2e24, pump=1e13 * (1 + q),
                        seed=0xBA7C0 + 17 * q))
    return out


def _setup(sim, m, q, oracle=False):
    g = m["grid"]
    if q % 2 == 0:
        sim.add_point_probe((g[0] // 3, g[1] // 2, g[2] // 2), 24, 450e-9, 750e-9)
    if q == 1:
        src = ((g[0] // 2, g[1] // 2, g[2] // 2), 1, 532e-9, 1.5e-15, 0.5e-15, 1e9)
        if oracle:
            sim.add_source(*src)
        else:
            sim.set_source(*src)


def _batch(members, pkw):
    from paper_0809_1547_gb300.binding import MBBatch, mb_default_params
    b = MBBatch([m["grid"] for m in members], DX, DT, mb_default_params(**pkw))
    for q, m in enumerate(members):
        b.set_instance(q, m["eps"], m["gain"], m["N_a"], m["pump"], m["seed"])
        _setup(b.instances[q], m, q)
    return b


def _single(m, q, pkw):
    _, g = make_pair(m["grid"], m["eps"], m["gain"], m["N_a"], m["pump"], m["seed"], pkw)
    _setup(g, m, q)
    return g


def _assert_same(sa, sb, q):
    for name in FIELD_NAMES:
        a, b = sa.field(name), sb.field(name)
        if not np.array_equal(a, b):
            where = tuple(np.argwhere(a != b)[0])
            raise AssertionError(f"member {q} differs in {name} at [k,j,i]={where}")


@pytest.mark.parametrize("steps", [37, 5])
def test_batch_members_equal_single_contexts_bitwise(steps):
    """Uneven grids (incl. a one-cell column), probes, a source, graph chunks + a tail."""
    pkw = params_kw(npml=4)
    members = _members(GRIDS, 4)
    b = _batch(members, pkw)
    b.step(steps)
    b.synchronize()
    for q, m in enumerate(members):
        s = _single(m, q, pkw)
        s.step(steps)
        inst = b.instances[q]
        assert inst.n == steps
        _assert_same(inst, s, q)
        if q % 2 == 0:
            np.testing.assert_array_equal(inst.probe_spectrum(0)[0], s.probe_spectrum(0)[0])
        U_b, fl_b = inst.energy()
        U_s, fl_s = s.energy()
        assert U_b == U_s
        scale = max(np.abs(fl_s).max(), 1e-300)
        assert np.abs(fl_b - fl_s).max() <= 1e-9 * scale
        s.close()
    assert np.abs(b.instances[0].field("Ex")).max() > 0
    b.close()


def test_batch_calls_chain_and_autotune_keeps_state():
    pkw = params_kw(npml=4)
    members = _members(GRIDS[:3], 4)
    a = _batch(members, pkw)
    c = _batch(members, pkw)
    a.step(40)
    c.step(7)
    c.autotune()              # trial steps must leave no trace
    c.step(33)
    a.synchronize()
    c.synchronize()
    for q in range(len(members)):
        assert c.instances[q].n == 40
        _assert_same(a.instances[q], c.instances[q], q)
    a.close()
    c.close()


def test_batch_member_matches_oracle():
    pkw = params_kw(npml=4)
    members = _members([(24, 22, 20), (17, 23, 31)], 4)
    b = _batch(members, pkw)
    b.step(120)
    b.synchronize()
    for q, m in enumerate(members):
        o, g = make_pair(m["grid"], m["eps"], m["gain"], m["N_a"], m["pump"], m["seed"], pkw)
        g.close()
        _setup(o, m, q, oracle=True)
        o.step(120)
        assert_fields_match(o, b.instances[q])
        if q % 2 == 0:
            S_o, _ = o.probe_spectrum(0)
            S_b, _ = b.instances[q].probe_spectrum(0)
            assert np.linalg.norm(S_b - S_o) <= 2e-5 * np.linalg.norm(S_o)
    b.close()


def test_batch_rejects_out_of_lockstep_member():
    from paper_0809_1547_gb300.binding import MBError, MB_ERR_STATE
    pkw = params_kw(npml=4)
    members = _members(GRIDS[:2], 4)
    b = _batch(members, pkw)
    b.step(2)
    b.instances[1].step(1)     # stepped outside the batch
    with pytest.raises(MBError) as e:
        b.step(1)
    assert e.value.code == MB_ERR_STATE
    b.close()


def test_batch_concurrent_mode_equals_persistent_bitwise():
    """The members' own launches on concurrent streams give the bits of the
    persistent launch, across graph chunks, tails and a mode switch between
    calls; one member takes the single-pass step."""
    from paper_0809_1547_gb300.binding import MB_BATCH_PERSISTENT, MB_BATCH_CONCURRENT, MBError, \
        MB_ERR_ARG
    pkw = params_kw(npml=4)
    grids = GRIDS + [(48, 20, 18)]
    members = _members(grids, 4)
    a, c, d = (_batch(members, pkw) for _ in range(3))
    assert a.mode == MB_BATCH_PERSISTENT
    c.set_mode(MB_BATCH_CONCURRENT)
    assert c.mode == MB_BATCH_CONCURRENT
    c.instances[len(grids) - 1].set_single_pass((1, 32, 4, 8))
    a.step(37)
    c.step(37)
    d.step(20)
    d.set_mode(MB_BATCH_CONCURRENT)
    d.step(17)
    for bt in (a, c, d):
        bt.synchronize()
    for q in range(len(members)):
        for other in (c, d):
            inst = other.instances[q]
            assert inst.n == 37
            _assert_same(a.instances[q], inst, q)
            if q % 2 == 0:
                np.testing.assert_array_equal(inst.probe_spectrum(0)[0], a.instances[q].probe_spectrum(0)[0])
            U_a, fl_a = a.instances[q].energy()
            U_o, fl_o = inst.energy()
            assert U_o == U_a
            # the face flux adds FP32 per-warp partials, grouped by the tile
            # shape (the members' own launch shapes here, the persistent
            # kernel's there), into FP64 slots: equal to FP32 rounding
            assert np.abs(fl_o - fl_a).max() <= 1e-6 * max(np.abs(fl_a).max(), 1e-300)
    with pytest.raises(MBError) as e:
        c.set_mode(7)
    assert e.value.code == MB_ERR_ARG
    for bt in (a, c, d):
        bt.close()


@pytest.mark.parametrize("mode", ["persistent", "concurrent"])
def test_full_size_members_sampled_parity(mode):
    """Three members of the ensemble workload (uneven sides, ~45 % fill,
    gain in the voids, noise) stepped in the batch: after 20 steps, one more
    batched step checked against the oracle on sub-blocks of the first
    member at its walls, corners, CPML interfaces and centre (fields and
    CPML memories; the block oracle gets the member's own CPML profiles,
    noise counters and step index)."""
    from paper_0809_1547_gb300 import inputs
    from paper_0809_1547_gb300.binding import MBBatch, mb_default_params, \
        MB_BATCH_PERSISTENT, MB_BATCH_CONCURRENT
    from parity_util import check_blocks_one_step
    ws = inputs.workload_batch(n_pump=16, n_seed=5)
    # members whose sides are not multiples of 16 (the padded layouts' case)
    picks, sides = [], set()
    for w in ws:
        if w.grid[0] % 16 and w.grid[0] not in sides and len(picks) < 3:
            picks.append(w)
            sides.add(w.grid[0])
    b = MBBatch([w.grid for w in picks], picks[0].dx, picks[0].dt,
                mb_default_params(npml=picks[0].npml))
    for q, w in enumerate(picks):
        b.set_instance(q, w.eps, w.gain, w.N_a, w.pump, w.seed)
    b.set_mode(MB_BATCH_PERSISTENT if mode == "persistent" else MB_BATCH_CONCURRENT)
    b.step(20)
    b.synchronize()
    w, g = picks[0], b.instances[0]
    n, size = w.grid[0], 18
    hi, mid = n - size, n // 2 - size // 2
    los = [(0, 0, 0), (hi, hi, hi), (0, mid, hi), (hi, 0, mid), (mid, hi, 0), (mid, mid, mid)]

    def one():
        b.step(1)
        b.synchronize()
    check_blocks_one_step(g, w, one, los, size, params_kw(npml=w.npml))
    b.close()

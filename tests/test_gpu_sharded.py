"""One grid split along z into slabs, on one GPU: each slab a context of its
own (mb_create_slab), boundary planes exchanged through the C ABI before
every step (mb_halo_pack / mb_halo_unpack), against the same grid stepped
as one context.  The own cells' fields and the point-probe spectra must be
bit-identical (same arithmetic on the same inputs, noise keyed by the
whole grid's cell index); the FP64 read-outs summed over the slabs equal the
whole grid's up to the order of summation (energy) and the FP32 grouping of
the face-flux warp sums (flux)."""
import numpy as np
import pytest

from paper_0809_1547_gb300 import inputs

pytestmark = pytest.mark.gpu

FIELDS = ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz", "Px", "Py", "Pz", "Jx", "Jy", "Jz",
          "N0", "N1", "N2", "N3")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_0809_1547_gb300 import build
    build.build()


def _pair(grid, dx, dt, npml, eps, gain, N_a, pump, seed, parts=2, bounds=None, single=None,
          probe=None, source=None, faces=None):
    from paper_0809_1547_gb300.binding import MBSimulation, mb_default_params
    from paper_0809_1547_gb300.sharded import SlabGrid
    p = mb_default_params(npml=npml)
    whole = MBSimulation(grid, dx, dt, p)
    split = SlabGrid(grid, dx, dt, parts, p, bounds=bounds)
    for s in [whole] + split.slabs:
        if single is not None:
            s.set_single_pass(single)
    whole.set_material(eps, gain, N_a, pump)
    whole.set_seed(seed)
    split.set_material(eps, gain, N_a, pump)
    split.set_seed(seed)
    pw = ps = None
    if probe is not None:
        pw = whole.add_point_probe(probe, 32, 475e-9, 705e-9)
        ps = split.add_point_probe(probe, 32, 475e-9, 705e-9)
    if source is not None:
        whole.set_source(*source)
        split.set_source(*source)
    if faces is not None:                      # (stride, every)
        for s in (whole, split):
            s.add_face_probes(faces[0], faces[1], 24, 475e-9, 705e-9)
    return whole, split, pw, ps


def _compare_faces(whole, split):
    for face in range(6):
        Sw, lw = whole.face_spectrum(face)
        Ss, ls = split.face_spectrum(face)
        assert np.array_equal(lw, ls)
        scale = float(np.max(np.abs(Sw)))
        assert scale > 0, face                 # every face saw the field
        # the same per-point accumulators, summed over the slabs in another order
        assert np.max(np.abs(Ss - Sw)) <= 1e-10 * scale, (face, Ss, Sw)


def _compare(whole, split, pw, ps, flux_rel=1e-5):
    for name in FIELDS:
        a, b = split.field(name), whole.field(name)
        assert a.shape == b.shape
        assert np.array_equal(a, b), (name, float(np.max(np.abs(a - b))))
    if pw is not None:
        Sw, lw = whole.probe_spectrum(pw)
        Ss, ls = split.probe_spectrum(ps)
        assert np.array_equal(Sw, Ss) and np.array_equal(lw, ls)
    Uw, Fw = whole.energy()
    Us, Fs = split.energy()
    assert Us == pytest.approx(Uw, rel=1e-12, abs=0)
    scale = max(float(np.max(np.abs(Fw))), 1e-300)
    assert np.max(np.abs(np.asarray(Fs) - np.asarray(Fw))) <= flux_rel * scale, (Fs, Fw)


@pytest.mark.parametrize("single", [(0, 32, 8, 16), (1, 32, 4, 16)], ids=["two-pass", "single-pass"])
def test_48_workload_two_slabs_500_steps(single):
    w = inputs.workload_small_48()
    mid = tuple(v // 2 for v in w.grid)
    whole, split, pw, ps = _pair(w.grid, w.dx, w.dt, w.npml, w.eps, w.gain, w.N_a, w.pump, w.seed,
                                 parts=2, single=single, probe=mid, faces=(4, 2))
    assert [s.z_end - s.z_begin for s in split.slabs] == [24, 24]
    whole.step(w.steps)
    split.step(w.steps)
    _compare(whole, split, pw, ps)
    _compare_faces(whole, split)
    whole.close()
    split.close()


def test_ragged_grid_three_slabs_with_source_and_cuts_at_the_cpml():
    # cuts at npml + 1 and n_z - npml - 1: the ghost planes touch the z-CPML
    grid, npml = (40, 9, 37), 4
    eps, gain = inputs.random_small(grid, seed=5, npml=npml)
    dx = 20e-9
    dt = inputs.courant_dt(dx)
    bounds = [(0, 5), (5, 32), (32, 37)]
    src = ((20, 4, 18), 2, 532e-9, 4e-15, 1e-15, 1e9)
    # face lattice stride 3: z rows 4, 7, .., 31 fall on the first two slabs;
    # the low z face (plane 4, H from 3) on the first, the high one (33, H
    # from 32) on the last
    whole, split, pw, ps = _pair(grid, dx, dt, npml, eps, gain, 3e24, 1e13, 0xABCD, parts=3,
                                 bounds=bounds, probe=(11, 5, 33), source=src, faces=(3, 1))
    whole.step(300)
    split.step(300)
    _compare(whole, split, pw, ps)
    _compare_faces(whole, split)
    # probes restarted on the whole grid and on every slab: the window's
    # spectra still agree
    whole.reset_probes()
    split.reset_probes()
    whole.step(100)
    split.step(100)
    _compare(whole, split, pw, ps)
    _compare_faces(whole, split)
    whole.close()
    split.close()


def test_four_slabs_of_a_single_pass_grid():
    grid, npml = (64, 32, 60), 6
    eps, gain = inputs.random_small(grid, seed=9, npml=npml)
    dx = 20e-9
    dt = inputs.courant_dt(dx)
    whole, split, pw, ps = _pair(grid, dx, dt, npml, eps, gain, 5e24, 1e13, 77, parts=4,
                                 single=(1, 32, 8, 5), probe=(30, 16, 29), faces=(2, 3))
    whole.step(120)
    split.step(120)
    _compare(whole, split, pw, ps)
    _compare_faces(whole, split)
    whole.close()
    split.close()


def test_slab_errors():
    from paper_0809_1547_gb300.binding import MBError, MB_ERR_ARG, MB_ERR_STATE, mb_default_params
    from paper_0809_1547_gb300.sharded import MBSlab
    import torch
    p = mb_default_params(npml=8)
    dt = inputs.courant_dt(20e-9)
    for zb, ze in ((0, 8), (8, 48), (0, 40), (20, 20), (-1, 10), (0, 49)):
        with pytest.raises(MBError) as e:
            MBSlab((48, 48, 48), zb, ze, 20e-9, dt, p)
        assert e.value.code == MB_ERR_ARG, (zb, ze)
    lo = MBSlab((48, 48, 48), 0, 24, 20e-9, dt, p)
    hi = MBSlab((48, 48, 48), 24, 48, 20e-9, dt, p)
    assert (lo.kz0, lo.own_lo, lo.own_hi, lo.grid[2]) == (0, 0, 24, 25)
    assert (hi.kz0, hi.own_lo, hi.own_hi, hi.grid[2]) == (23, 1, 25, 25)
    buf = torch.zeros(lo.halo_bytes // 4, dtype=torch.float32, device="cuda")
    with pytest.raises(MBError) as e:
        lo.unpack(0, buf)                 # the grid's first slab has no ghost below
    assert e.value.code == MB_ERR_STATE
    with pytest.raises(MBError) as e:
        hi.unpack(1, buf)                 # nor the last one above
    assert e.value.code == MB_ERR_STATE
    w = inputs.workload_small_48()
    lo.set_material(w.eps[:25], w.gain[:25], w.N_a, w.pump)
    with pytest.raises(MBError) as e:
        lo.adjoint_energy_zface(4, 2)
    assert e.value.code == MB_ERR_STATE
    lo.close()
    hi.close()


def test_one_rank_distributed_slab_is_the_whole_grid():
    import os
    import socket
    import torch
    import torch.distributed as dist
    from paper_0809_1547_gb300.binding import MBSimulation, mb_default_params
    from paper_0809_1547_gb300.sharded import DistributedSlab
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("nccl", rank=0, world_size=1)
    try:
        w = inputs.workload_small_48()
        p = mb_default_params(npml=w.npml)
        d = DistributedSlab(w.grid, w.dx, w.dt, p)
        whole = MBSimulation(w.grid, w.dx, w.dt, p)
        for s in (d, whole):
            s.set_material(w.eps, w.gain, w.N_a, w.pump)
            s.set_seed(w.seed)
        d.step(60)
        whole.step(60)
        assert np.array_equal(d.sim.field("Ez"), whole.field("Ez"))
        U, F = d.energy()
        Uw, Fw = whole.energy()
        assert U == pytest.approx(Uw, rel=1e-12, abs=0)
        d.close()
        whole.close()
    finally:
        dist.destroy_process_group()

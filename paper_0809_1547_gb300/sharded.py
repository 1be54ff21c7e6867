"""One grid split along z into slabs.

The paper advances its FDTD grid "distributed on (typically) 256
processors" ("Simulations" paragraph).  Here each slab is a context of its
own (``mb_create_slab``): the slab's own planes plus a ghost plane next to
each neighbour.  Before every step the neighbours exchange one boundary
plane each way (the whole time-n state of the plane, ``mb_halo_pack`` /
``mb_halo_unpack``); every slab then takes one ordinary step, and the own
cells equal those of the whole grid bit for bit (the noise is keyed by the
cell's index in the whole grid, the CPML and the flux box are the whole
grid's).  FP64 read-outs are summed over the slabs.

* :func:`slab_partition` splits n_z planes into slabs.
* :class:`MBSlab` wraps one slab context.
* :class:`SlabGrid` holds all slabs in this process (on one GPU: the split
  run checked against the whole grid).
* :class:`DistributedSlab` holds this rank's slab of a grid split over the
  ranks of a ``torch.distributed`` group: boundary planes go to the
  neighbouring ranks by point-to-point send / receive into the receiver's
  own memory (:func:`exchange_planes`), read-outs are summed in FP64 over
  the ranks (:func:`reduce_readouts`).
"""
from __future__ import annotations

import numpy as np

from . import binding as B
from .binding import MBSimulation


def slab_partition(nz: int, parts: int, npml: int):
    """[(z_begin, z_end)] of `parts` slabs covering planes 0 .. nz-1, with
    own-plane counts as equal as the cut rule allows: every cut plane c lies
    in [npml + 1, nz - npml - 1], so that the ghost planes c - 1 and c are
    outside the z-CPML."""
    nz, parts, npml = int(nz), int(parts), int(npml)
    if parts < 1 or nz < 1:
        raise ValueError("need parts >= 1 and nz >= 1")
    if parts == 1:
        return [(0, nz)]
    lo, hi = npml + 1, nz - npml - 1
    if hi - lo + 1 < parts - 1:
        raise ValueError(f"{nz} planes with a {npml}-cell CPML cannot be cut into {parts} slabs")
    cuts = []
    for q in range(1, parts):
        c = int(round(nz * q / parts))
        c = max(c, lo + (q - 1), (cuts[-1] + 1) if cuts else lo)
        c = min(c, hi - (parts - 1 - q))
        cuts.append(c)
    bounds = [0] + cuts + [nz]
    return list(zip(bounds[:-1], bounds[1:]))


class MBSlab(MBSimulation):
    """The slab context of planes [z_begin, z_end) of a grid (``grid`` is the
    whole grid's size).  Its local grid (``self.grid``) is its own planes plus
    a ghost plane next to each neighbour; plane k of it is plane k + kz0 of
    the whole grid, and local planes own_lo .. own_hi - 1 are its own."""

    def __init__(self, grid, z_begin, z_end, dx, dt, params: B.mb_params | None = None,
                 stream=None):
        self.whole_grid = tuple(int(v) for v in grid)
        self.dx, self.dt = float(dx), float(dt)
        self.probe_nfreq = {}
        self.face_nfreq = 0
        self._owned = True
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream().cuda_stream or None
            except Exception:
                stream = None
        self._h = B.mb_create_slab(self.whole_grid, z_begin, z_end, dx, dt, params, stream)
        self.gnz, self.kz0, self.own_lo, self.own_hi = B.mb_slab_info(self._h)
        self.z_begin, self.z_end = int(z_begin), int(z_end)
        # own planes, the ghost below (own_lo = 1) and the ghost above
        self.grid = (self.whole_grid[0], self.whole_grid[1],
                     self.own_hi + (1 if self.z_end < self.gnz else 0))
        self.shape = self.grid[::-1]
        self.halo_bytes = B.mb_halo_bytes(self._h)

    def local_planes(self):
        """Whole-grid planes held by the context (ghosts included)."""
        return self.kz0, self.kz0 + self.grid[2]

    def owns(self, k: int) -> bool:
        return self.z_begin <= int(k) < self.z_end

    def to_local(self, ijk):
        return (int(ijk[0]), int(ijk[1]), int(ijk[2]) - self.kz0)

    def pack(self, side: int, buf):
        """Queue the state of the lowest (0) / highest (1) own plane into the
        device tensor `buf` (at least ``halo_bytes``)."""
        B.mb_halo_pack(self._h, side, buf.data_ptr())

    def unpack(self, side: int, buf):
        """Queue a neighbour's packed plane into the ghost plane below (0) /
        above (1)."""
        B.mb_halo_unpack(self._h, side, buf.data_ptr())

    def own_field(self, name):
        """The field on the own planes, [k, j, i] (k over z_begin .. z_end-1)."""
        return self.field(name)[self.own_lo:self.own_hi]


def _halo_buffer(nbytes: int, device):
    import torch
    return torch.empty((nbytes + 3) // 4, dtype=torch.float32, device=device)


class SlabGrid:
    """A grid split along z into `parts` slabs, all held by this process on
    the current CUDA device and queued on one stream; stepped by the slab
    protocol (exchange, then one step of every slab)."""

    def __init__(self, grid, dx, dt, parts: int, params: B.mb_params | None = None, stream=None,
                 bounds=None):
        import torch
        self.grid = tuple(int(v) for v in grid)
        self.params = params if params is not None else B.mb_default_params()
        self.bounds = list(bounds) if bounds is not None else \
            slab_partition(self.grid[2], parts, self.params.npml)
        # one stream for every slab, so that each unpack follows its pack
        if not stream:
            self._stream = torch.cuda.Stream()
            stream = self._stream.cuda_stream
        self.slabs = [MBSlab(self.grid, zb, ze, dx, dt, self.params, stream) for zb, ze in self.bounds]
        dev = torch.device("cuda", torch.cuda.current_device())
        nb = self.slabs[0].halo_bytes
        # per interface: the plane going up and the plane going down
        self._up = [_halo_buffer(nb, dev) for _ in self.slabs[1:]]
        self._down = [_halo_buffer(nb, dev) for _ in self.slabs[1:]]
        self.probes = {}

    def close(self):
        for s in self.slabs:
            s.close()
        self.slabs = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def owner(self, k: int) -> int:
        for q, s in enumerate(self.slabs):
            if s.owns(k):
                return q
        raise ValueError(f"plane {k} outside the grid")

    def set_material(self, eps_r, gain_mask, N_a, pump):
        """Whole-grid maps [k, j, i]; each slab gets its planes (ghosts included)."""
        eps = np.asarray(eps_r).reshape(self.grid[::-1])
        gm = np.asarray(gain_mask).reshape(self.grid[::-1])
        for s in self.slabs:
            a, b = s.local_planes()
            s.set_material(eps[a:b], gm[a:b], N_a, pump)

    def set_seed(self, seed):
        for s in self.slabs:
            s.set_seed(seed)

    def add_point_probe(self, ijk, n_freq, lam_min, lam_max):
        """Probe at whole-grid cell ijk, kept by the slab that owns it."""
        q = self.owner(ijk[2])
        pid = self.slabs[q].add_point_probe(self.slabs[q].to_local(ijk), n_freq, lam_min, lam_max)
        key = len(self.probes)
        self.probes[key] = (q, pid)
        return key

    def add_face_probes(self, stride, every, n_freq, lam_min, lam_max):
        """The whole grid's face probes: each slab keeps the lattice points on
        its own planes (a z face: the slab owning the plane below it)."""
        for s in self.slabs:
            s.add_face_probes(stride, every, n_freq, lam_min, lam_max)

    def face_spectrum(self, face):
        """(S, lam) of one face of the whole grid: the slabs' spectra summed
        (FP64; the per-point accumulators equal the whole grid's)."""
        S, lam = None, None
        for s in self.slabs:
            Sq, lam = s.face_spectrum(face)
            S = np.asarray(Sq, dtype=np.float64) if S is None else S + Sq
        return S, lam

    def set_source(self, ijk, comp, lam, t0, tau, amp):
        q = self.owner(ijk[2])
        self.slabs[q].set_source(self.slabs[q].to_local(ijk), comp, lam, t0, tau, amp)

    def reset_probes(self):
        """Restart every slab's probe sums (spectra of the steps from here on)."""
        for s in self.slabs:
            s.reset_probes()

    def exchange(self):
        """Every interface: the lower slab's top own plane into the upper
        slab's ghost below, the upper slab's bottom own plane into the lower
        slab's ghost above."""
        for q in range(len(self.slabs) - 1):
            lo, hi = self.slabs[q], self.slabs[q + 1]
            lo.pack(1, self._up[q])
            hi.pack(0, self._down[q])
            hi.unpack(0, self._up[q])
            lo.unpack(1, self._down[q])

    def step(self, n: int = 1):
        for _ in range(int(n)):
            self.exchange()
            for s in self.slabs:
                s.step(1)

    def synchronize(self):
        for s in self.slabs:
            s.synchronize()

    def field(self, name):
        """The whole grid's field [k, j, i] from the slabs' own planes."""
        return np.concatenate([s.own_field(name) for s in self.slabs], axis=0)

    def energy(self):
        """(U, flux6): the slabs' own-plane energies and face energies summed."""
        U, fl = 0.0, np.zeros(6)
        for s in self.slabs:
            u, f = s.energy()
            U += u
            fl += np.asarray(f)
        return U, fl

    def probe_spectrum(self, key):
        q, pid = self.probes[key]
        return self.slabs[q].probe_spectrum(pid)


# ---------------------------------------------------------------- one slab per rank

def exchange_planes(send_lo, send_hi, recv_lo, recv_hi, rank: int, world: int, group=None):
    """Point-to-point exchange of boundary planes between neighbouring ranks
    of a z-split grid: rank r sends its lowest own plane (send_lo) to r - 1
    and its highest (send_hi) to r + 1, and receives r - 1's highest into
    recv_lo and r + 1's lowest into recv_hi (tensors on the device the
    backend serves: CUDA with NCCL, CPU with gloo).  The first and last rank
    skip the missing side."""
    import torch.distributed as dist
    ops = []
    if rank > 0:
        ops.append(dist.P2POp(dist.isend, send_lo, rank - 1, group))
        ops.append(dist.P2POp(dist.irecv, recv_lo, rank - 1, group))
    if rank < world - 1:
        ops.append(dist.P2POp(dist.isend, send_hi, rank + 1, group))
        ops.append(dist.P2POp(dist.irecv, recv_hi, rank + 1, group))
    if ops:
        for r in dist.batch_isend_irecv(ops):
            r.wait()


def reduce_readouts(values, device=None, group=None):
    """FP64 sum over the ranks of per-slab read-outs (energy, face energies,
    ...): returns the summed numpy array."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(np.asarray(values, dtype=np.float64), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy()


class DistributedSlab:
    """This rank's slab of a grid split along z over the ranks of a
    torch.distributed group (one GPU per rank, NCCL)."""

    def __init__(self, grid, dx, dt, params: B.mb_params | None = None, group=None, stream=None):
        """stream: a torch.cuda.Stream for the slab's work (default: a new one)."""
        import torch
        import torch.distributed as dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.grid = tuple(int(v) for v in grid)
        self.params = params if params is not None else B.mb_default_params()
        self.bounds = slab_partition(self.grid[2], self.world, self.params.npml)
        zb, ze = self.bounds[self.rank]
        self.device = torch.device("cuda", torch.cuda.current_device())
        # the slab's work and the point-to-point transfers share one stream:
        # the backend orders its transfers after the packs queued there and
        # the unpacks after the transfers
        self.stream = torch.cuda.Stream() if stream is None else stream
        self.sim = MBSlab(self.grid, zb, ze, dx, dt, self.params, self.stream.cuda_stream)
        nb = self.sim.halo_bytes
        self._send = [_halo_buffer(nb, self.device) for _ in range(2)]
        self._recv = [_halo_buffer(nb, self.device) for _ in range(2)]

    def set_material(self, eps_r, gain_mask, N_a, pump):
        eps = np.asarray(eps_r).reshape(self.grid[::-1])
        gm = np.asarray(gain_mask).reshape(self.grid[::-1])
        a, b = self.sim.local_planes()
        self.sim.set_material(eps[a:b], gm[a:b], N_a, pump)

    def set_seed(self, seed):
        self.sim.set_seed(seed)

    def exchange(self):
        if self.world == 1:
            return
        if self.rank > 0:
            self.sim.pack(0, self._send[0])
        if self.rank < self.world - 1:
            self.sim.pack(1, self._send[1])
        import torch
        with torch.cuda.stream(self.stream):
            exchange_planes(self._send[0], self._send[1], self._recv[0], self._recv[1],
                            self.rank, self.world, self.group)
        if self.rank > 0:
            self.sim.unpack(0, self._recv[0])
        if self.rank < self.world - 1:
            self.sim.unpack(1, self._recv[1])

    def step(self, n: int = 1):
        for _ in range(int(n)):
            self.exchange()
            self.sim.step(1)

    def energy(self):
        """(U, flux6) of the whole grid (FP64 sums over the ranks)."""
        import torch
        u, f = self.sim.energy()
        with torch.cuda.stream(self.stream):
            v = reduce_readouts([u] + list(f), device=self.device, group=self.group)
        return float(v[0]), v[1:]

    def add_face_probes(self, stride, every, n_freq, lam_min, lam_max):
        self.sim.add_face_probes(stride, every, n_freq, lam_min, lam_max)

    def reset_probes(self):
        """Restart this rank's probe sums (every rank calls it at the same step)."""
        self.sim.reset_probes()

    def face_spectrum(self, face):
        """(S, lam) of one face of the whole grid (FP64 sum over the ranks)."""
        import torch
        S, lam = self.sim.face_spectrum(face)
        with torch.cuda.stream(self.stream):
            S = reduce_readouts(S, device=self.device, group=self.group)
        return S, lam

    def close(self):
        self.sim.close()

"""Set-up of the benchmark workloads on the CUDA path (probes, seeds, tuning)."""
from __future__ import annotations

from .binding import MBSimulation, mb_default_params

# Probe spectra span the gain line lambda0 -/+ dlambda/2 (475-705 nm).
LAM_MIN, LAM_MAX = 475e-9, 705e-9
N_FREQ = 128
FACE_STRIDE, FACE_EVERY = 8, 4


def setup_simulation(w, autotune: bool = True, face_probes: bool = True, point_probe: bool = True,
                     stream=None) -> MBSimulation:
    """An MBSimulation for workload ``w`` (inputs.Workload) ready to step.

    Active runs: centre point probe and the six face probes (stride 8, every
    4 steps, 128 bins over 475-705 nm), Langevin seed of the workload.
    """
    sim = MBSimulation(w.grid, w.dx, w.dt, mb_default_params(npml=w.npml), stream=stream)
    sim.set_material(w.eps, w.gain, w.N_a, w.pump)
    sim.set_seed(w.seed)
    if point_probe:
        probe = w.extra.get("probe", tuple(v // 2 for v in w.grid))
        sim.add_point_probe(probe, N_FREQ, LAM_MIN, LAM_MAX)
    if face_probes:
        sim.add_face_probes(FACE_STRIDE, FACE_EVERY, N_FREQ, LAM_MIN, LAM_MAX)
    if autotune:
        sim.autotune()
    return sim

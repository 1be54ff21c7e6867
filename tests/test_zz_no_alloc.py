"""The allocation-free energy sum against the context's own energy read-out.

mb_energy_sum_noalloc serves callers that cannot allocate device memory; it
keeps its scratch in a static device array.  Here it must reproduce
mb_energy, call after call (the array keeps the previous call's contents).
This file is collected last on purpose.
"""
import ctypes as C
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

EPS0 = 8.8541878128e-12
DX = 20e-9
DT = 0.99 * DX / (299_792_458.0 * math.sqrt(3.0))


def _noalloc_energy(sim, eps_dev, out):
    import torch
    from paper_0809_1547_gb300.binding import mb_energy_sum_noalloc
    fields = {}
    scale_e = None
    for name in ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz"):
        t, s = sim.field_device(name)
        fields[name] = t
        if name == "Ex":
            scale_e = s
    ncell = fields["Ex"].numel()
    stream = torch.cuda.current_stream().cuda_stream
    mb_energy_sum_noalloc(*(fields[n].data_ptr() for n in ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz")),
                          eps_dev.data_ptr(), ncell, out.data_ptr(), stream)
    torch.cuda.synchronize()
    total, flag = out.cpu().tolist()
    return 0.5 * EPS0 * scale_e ** 2 * DX ** 3 * total, flag


def test_noalloc_energy_matches_context_energy_on_consecutive_calls():
    import torch
    from paper_0809_1547_gb300 import build, inputs
    from paper_0809_1547_gb300.binding import MBSimulation, mb_default_params
    build.build()
    grid = (40, 36, 30)
    eps, gain = inputs.random_small(grid, seed=21, npml=4)
    sim = MBSimulation(grid, DX, DT, mb_default_params(npml=4))
    sim.set_material(eps, gain, 4e24, 1e13)
    sim.set_seed(3)
    sim.set_source((20, 18, 15), 2, 532e-9, 1.5e-15, 0.5e-15, 1e9)
    eps_dev = torch.from_numpy(np.ascontiguousarray(eps, dtype=np.float32).reshape(-1)).cuda()
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    for steps in (40, 25):
        sim.step(steps)
        U_ctx, _ = sim.energy()
        U_na, flag = _noalloc_energy(sim, eps_dev, out)
        assert U_ctx > 0 and flag == 0.0
        assert abs(U_na - U_ctx) <= 1e-10 * U_ctx, (steps, U_na, U_ctx)
    sim.close()


def test_noalloc_rejects_sizes_beyond_its_array():
    import torch
    from paper_0809_1547_gb300.binding import (load_library, mb_energy_sum_noalloc, MBError,
                                               MB_ERR_ARG)
    t = torch.zeros(4, dtype=torch.float32, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    p = t.data_ptr()
    with pytest.raises(MBError) as e:
        mb_energy_sum_noalloc(p, p, p, p, p, p, 0, 67_108_865, out.data_ptr())
    assert e.value.code == MB_ERR_ARG
    assert b"67108864" in load_library().mb_last_error(None)

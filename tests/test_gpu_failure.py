"""Failure detection without a GPU fault: the bounded waits of the batched
kernel (grid barrier) and of the TMA kernels (mbarrier) run against events
that never come, give up after their poll limit, report it, and leave the
device usable; device allocations fail on request (injected on the host)
and the calls clean up and report MB_ERR_OOM."""
import time

import numpy as np
import pytest

from parity_util import DX, DT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_0809_1547_gb300 import build
    build.build()


def test_bounded_waits_give_up_and_the_device_stays_usable():
    import torch
    from paper_0809_1547_gb300.binding import (MBBatch, MBSimulation, mb_default_params,
                                                mb_selftest_bounded_waits)
    blocks = min(torch.cuda.get_device_properties(0).multi_processor_count, 8)
    t0 = time.perf_counter()
    assert mb_selftest_bounded_waits(0, 4096) == blocks      # every block of the grid gave up
    t1 = time.perf_counter()
    assert mb_selftest_bounded_waits(1, 256) == 1
    t2 = time.perf_counter()
    assert t1 - t0 < 30 and t2 - t1 < 30
    # the device still runs the step and the batched kernel
    grid = (16, 16, 16)
    eps = np.ones(grid[::-1], np.float32)
    gain = np.ones(grid[::-1], np.uint8)
    s = MBSimulation(grid, DX, DT, mb_default_params(npml=2))
    s.set_material(eps, gain, 1e24, 1e13)
    s.step(5)
    s.synchronize()
    assert np.isfinite(s.field("Ex")).all()
    s.close()
    b = MBBatch([grid, grid], DX, DT, mb_default_params(npml=2))
    for q in range(2):
        b.set_instance(q, eps, gain, 1e24, 1e13, q)
    b.step(3)
    b.synchronize()
    b.close()


def test_selftest_argument_errors():
    from paper_0809_1547_gb300.binding import MBError, MB_ERR_ARG, mb_selftest_bounded_waits
    for which, limit in ((2, 10), (0, 0), (1, 1 << 23)):
        with pytest.raises(MBError) as e:
            mb_selftest_bounded_waits(which, limit)
        assert e.value.code == MB_ERR_ARG


def test_injected_allocation_failures_leave_nothing_behind():
    """Every device allocation of mb_create, and the single-pass step's second
    copy, can fail (injected on the host): the call reports MB_ERR_OOM, frees
    what it had taken, and the next call succeeds."""
    import torch
    from paper_0809_1547_gb300.binding import (MBSimulation, MBError, MB_ERR_OOM,
                                               mb_debug_fail_alloc, mb_default_params)
    grid = (48, 40, 36)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    try:
        for n in (0, 1, 2, 3, 5, 8):
            mb_debug_fail_alloc(n)
            with pytest.raises(MBError) as e:
                MBSimulation(grid, 20e-9, 3.8e-17, mb_default_params(npml=4))
            assert e.value.code == MB_ERR_OOM
        mb_debug_fail_alloc(-1)
        torch.cuda.synchronize()
        assert abs(torch.cuda.mem_get_info()[0] - free0) < (4 << 20)
        g = MBSimulation(grid, 20e-9, 3.8e-17, mb_default_params(npml=4))
        mb_debug_fail_alloc(0)
        with pytest.raises(MBError) as e:
            g.set_single_pass((1, 32, 4, 8))
        assert e.value.code == MB_ERR_OOM
        mb_debug_fail_alloc(-1)
        assert g.single_pass()[0] == 0
        g.step(3)                       # the two passes still run
        g.set_single_pass((1, 32, 4, 8))
        g.step(3)
        g.close()
    finally:
        mb_debug_fail_alloc(-1)

"""Failure detection without a GPU fault: the bounded waits of the batched
kernel (grid barrier) and of the TMA kernels (mbarrier) run against events
that never come, give up after their poll limit, report it, and leave the
device usable."""
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

"""Pump sweep on the batched ensemble (GPU) against the oracle run instance
by instance: the spectra within relative L2 2e-5, hence the same peaks and
widths; and the full-size ensemble's sweep runs and yields finite statistics."""
import math

import numpy as np
import pytest

from oracle.mb_oracle import MBOracle, Params
from oracle import mb_analysis as O
from parity_util import DX, DT, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_0809_1547_gb300 import build
    build.build()


def _ensemble():
    from paper_0809_1547_gb300 import inputs
    ws = []
    for q, (grid, N_a) in enumerate([((24, 22, 20), 5e23), ((26, 20, 22), 5e24), ((24, 22, 20), 2e25),
                                     ((20, 24, 23), 2e25)]):
        eps, gain = inputs.random_small(grid, seed=40 + q, npml=4, d_cells=5)
        ws.append(inputs.Workload(f"sweep{q}", grid, DX, DT, eps, gain, N_a, 1e14, 0x5E0 + q, 300, 4))
    return ws


def test_small_sweep_matches_oracle():
    from paper_0809_1547_gb300.sweep import run_pump_sweep, spectral_stats, N_FREQ, LAM_MIN, LAM_MAX
    ws = _ensemble()
    levels, spectra, lam, _ = run_pump_sweep(ws, 300, autotune=False)
    st = spectral_stats(spectra, lam)
    w = O.omegas_of(lam)
    for q, wl in enumerate(ws):
        o = MBOracle(wl.grid, DX, DT, Params(npml=wl.npml))
        o.set_material(wl.eps, wl.gain, wl.N_a, wl.pump)
        o.set_seed(wl.seed)
        pid = o.add_point_probe(tuple(v // 2 for v in wl.grid), N_FREQ, LAM_MIN, LAM_MAX)
        o.step(300)
        S_o, lam_o = o.probe_spectrum(pid)
        np.testing.assert_allclose(lam, lam_o, rtol=1e-15)
        assert rel_l2(spectra[q], S_o) <= 2e-5
        assert abs(st["peak_w"][q] - O.peak(S_o, w)[0]) <= abs(w[1] - w[0]) * 1.0001
        assert st["std_w"][q] == pytest.approx(O.std_width(S_o, w), rel=1e-4, abs=0)


def test_windowed_sweep_matches_oracle():
    """Probes restarted at step 180 of 300 in every member of the batch
    (mb_reset_probes on the instances): the spectra equal the oracle's DFT of
    steps 181-300 only, and records taken before the restart keep the
    spectra from step 0."""
    from paper_0809_1547_gb300.sweep import run_pump_sweep, N_FREQ, LAM_MIN, LAM_MAX
    ws = _ensemble()[:2]
    levels, spectra, lam, _, snaps = run_pump_sweep(ws, 300, autotune=False, record=(120,),
                                                    window_from=180)
    assert [st for st, _ in snaps] == [120]
    for q, wl in enumerate(ws):
        o = MBOracle(wl.grid, DX, DT, Params(npml=wl.npml))
        o.set_material(wl.eps, wl.gain, wl.N_a, wl.pump)
        o.set_seed(wl.seed)
        pid = o.add_point_probe(tuple(v // 2 for v in wl.grid), N_FREQ, LAM_MIN, LAM_MAX)
        o.step(120)
        S_120, _ = o.probe_spectrum(pid)
        assert rel_l2(snaps[0][1][q], S_120) <= 2e-5
        o.step(60)
        o.point_probes[pid]["acc"][:] = 0
        o.step(120)
        S_o, _ = o.probe_spectrum(pid)
        assert S_o.max() > 0
        assert rel_l2(spectra[q], S_o) <= 2e-5


def test_full_ensemble_sweep_runs():
    """The 80-realization ensemble (16 N_a levels x 5 seeds, cubes of side
    97-148) for 200 steps: every spectrum finite and non-zero, one row per
    level."""
    from paper_0809_1547_gb300 import inputs
    from paper_0809_1547_gb300.sweep import run_pump_sweep, spectral_stats, summarize
    ws = inputs.workload_batch()
    levels, spectra, lam, secs = run_pump_sweep(ws, 200)
    assert np.isfinite(spectra).all() and (spectra.sum(axis=1) > 0).all()
    rows, thr = summarize(levels, spectral_stats(spectra, lam))
    assert len(rows) == 16 and all(r["n"] == 5 for r in rows)
    assert all(np.isfinite(r["std_w"]) for r in rows)

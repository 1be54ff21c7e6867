"""The sweep's spectral statistics (product, vectorised) against the oracle's
definitions on the same spectra (CPU)."""
import numpy as np
import pytest

from oracle import mb_analysis as O
from paper_0809_1547_gb300.sweep import emission_threshold, spectral_stats, summarize


def _spectra(n=12, seed=0):
    rng = np.random.default_rng(seed)
    lam = np.linspace(475e-9, 705e-9, 128)
    w = O.omegas_of(lam)
    S = []
    for q in range(n):
        mu = rng.uniform(w.min() * 1.02, w.max() * 0.98)
        sig = rng.uniform(0.004, 0.05) * mu
        S.append(np.exp(-0.5 * ((w - mu) / sig) ** 2) * (1 + 0.05 * rng.random(128)) + 1e-6)
    return np.array(S), lam, w


def test_stats_agree_with_oracle_definitions():
    S, lam, w = _spectra()
    st = spectral_stats(S, lam)
    for q in range(S.shape[0]):
        pw, pS = O.peak(S[q], w)
        assert st["peak_w"][q] == pw and st["peak_S"][q] == pS
        assert st["std_w"][q] == pytest.approx(O.std_width(S[q], w), rel=1e-12, abs=0)
        c, sg = O.gaussian_fit(S[q], w)
        if sg is None:
            assert np.isnan(st["gauss_w"][q])
        else:
            assert st["gauss_w"][q] == pytest.approx(sg, rel=1e-7, abs=0)


def test_summary_and_threshold_agree_with_oracle():
    S, lam, w = _spectra(n=8, seed=3)
    levels = [1e24, 1e24, 3e24, 3e24, 1e25, 1e25, 2e25, 2e25]
    order = np.argsort([-np.sqrt(np.sum(s)) for s in S])     # any assignment of spectra to levels
    S = S[order]
    rows, thr = summarize(levels, spectral_stats(S, lam))
    rows_o, thr_o = O.sweep_table(levels, list(S), w)
    assert thr == thr_o
    for r, ro in zip(rows, rows_o):
        assert r["N_a"] == ro["level"]
        assert r["std_w"] == pytest.approx(ro["std_w"], rel=1e-12, abs=0)
        assert r["peak_w"] == pytest.approx(ro["peak_w"], rel=1e-12, abs=0)


def test_emission_threshold_agrees_with_oracle():
    S, lam, w = _spectra(n=8, seed=5)
    levels = [1e24, 1e24, 3e24, 3e24, 1e25, 1e25, 2e25, 2e25]
    # scale the spectra into an S-curve of emitted energy
    scale = np.array([1.0, 1.1, 3.0, 2.9, 80.0, 75.0, 9e3, 8e3])
    S = S / S.sum(axis=1, keepdims=True) * scale[:, None]
    rows, _ = summarize(levels, spectral_stats(S, lam))
    rows_o, _ = O.sweep_table(levels, list(S), w)
    for r, ro in zip(rows, rows_o):
        assert r["emitted"] == pytest.approx(ro["emitted"], rel=1e-12, abs=0)
    thr = emission_threshold(rows)
    assert thr == O.emission_threshold([r["level"] for r in rows_o], [r["emitted"] for r in rows_o])
    assert thr == 3e24

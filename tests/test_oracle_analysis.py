"""Pins of the oracle's spectral statistics (CPU): closed forms."""
import math

import numpy as np
import pytest

from oracle.mb_analysis import emission_threshold, gaussian_fit, peak, std_width, sweep_table


def test_sampled_gaussian_gives_back_centre_and_width():
    w = np.linspace(3.0e15, 3.4e15, 401)
    mu, sig = 3.1903e15, 7.0e12   # off the grid: the fitted window is not symmetric about mu
    S = 2.5 * np.exp(-0.5 * ((w - mu) / sig) ** 2)
    c, s = gaussian_fit(S, w)
    assert c == pytest.approx(mu, rel=1e-10, abs=0)
    assert s == pytest.approx(sig, rel=1e-8, abs=0)
    assert std_width(S, w) == pytest.approx(sig, rel=1e-6, abs=0)   # fully inside the window
    pw, pS = peak(S, w)
    assert abs(pw - mu) <= (w[1] - w[0]) and pS == pytest.approx(2.5, rel=1e-3, abs=0)


def test_flat_spectrum_std_width_is_uniform():
    w = np.arange(1000, dtype=np.float64)
    assert std_width(np.ones(1000), w) == pytest.approx(math.sqrt((1000 ** 2 - 1) / 12.0), rel=1e-12, abs=0)
    assert gaussian_fit(np.ones(1000), w) == (None, None)    # no curvature


def test_two_lines_std_width_is_half_the_spacing():
    w = np.linspace(0.0, 10.0, 11)
    S = np.zeros(11)
    S[2] = S[8] = 1.0
    assert std_width(S, w) == pytest.approx(3.0, rel=1e-12, abs=0)


def test_sweep_threshold_is_first_level_that_halves_the_width():
    w = np.linspace(-50.0, 50.0, 201)
    def g(sig):
        return np.exp(-0.5 * (w / sig) ** 2)
    levels = [1, 1, 2, 2, 3, 3]
    spectra = [g(20), g(20), g(14), g(14), g(8), g(8)]
    rows, thr = sweep_table(levels, spectra, w)
    assert [r["level"] for r in rows] == [1.0, 2.0, 3.0]
    assert thr == 3.0
    assert rows[2]["gauss_w"] == pytest.approx(8.0, rel=1e-8, abs=0)


def test_emission_threshold_finds_the_kink_of_an_s_curve():
    # E = L below L = 4 (spontaneous, slope 1), E = L exp(3 (L - 4)) from it on
    levels = [1.0, 2.0, 3.0, 4.0, 5.0, 6.0]
    E = [L if L < 4 else L * math.exp(3.0 * (L - 4.0)) for L in levels]
    assert emission_threshold(levels, E) == 4.0
    # power laws up to the critical slope have no threshold
    assert emission_threshold(levels, [L ** 1.5 for L in levels]) is None
    assert emission_threshold(levels, [L ** 1.95 for L in levels]) is None
    assert emission_threshold(levels, [L ** 2.2 for L in levels]) == 1.0
    # the per-level mean emitted energy of the sweep table is the mean of sum S
    w = np.linspace(-50.0, 50.0, 201)
    rows, _ = sweep_table([1, 1, 2], [np.ones(201), 3 * np.ones(201), np.ones(201)], w)
    assert rows[0]["emitted"] == pytest.approx(2 * 201, rel=1e-15, abs=0)

"""Pins of the oracle's bound-state solver for -phi'' + tau^2 phi + phi^3 = E phi
(the paper's Eq. g5) and of its spectral features (CPU)."""
import math

import numpy as np
import pytest

from oracle import gp_oracle as G


def _integrals(tau, h, phi):
    dphi = np.diff(np.concatenate(([0.0], phi, [0.0]))) / h
    A = h * np.sum(dphi ** 2)
    B = h * np.sum(tau ** 2 * phi ** 2)
    C = h * np.sum(phi ** 4)
    D = h * np.sum(phi ** 2)
    return A, B, C, D


@pytest.mark.parametrize("E", [1.003, 1.01])
def test_near_threshold_closed_form(E):
    # the grid's linear ground state sits O(h^2) below 1 (~1e-6 here): small
    # against E - 1, so the first-order closed form is the reference
    tau, h, phi = G.solve(E, n=4095)
    ref = G.near_threshold(tau, E)
    err = np.linalg.norm(phi - ref) / np.linalg.norm(ref)
    assert err < 3.0 * (E - 1.0), err            # first correction is O(E - 1) relative
    w, p = G.features(tau, h, phi)
    assert w == pytest.approx(1.0 / (2.0 * math.sqrt(2.0) * math.pi), rel=3.0 * (E - 1.0), abs=0)
    assert p == pytest.approx((E - 1.0) / (math.sqrt(2.0) * math.pi), rel=3.0 * (E - 1.0), abs=0)


@pytest.mark.parametrize("E", [1.5, 4.0, 20.0, 60.0])
def test_discrete_and_virial_identities(E):
    tau, h, phi = G.solve(E)
    assert phi.min() > -1e-12 and phi.max() > 0
    A, B, C, D = _integrals(tau, h, phi)
    # the discrete equation times phi, summed: exact for the discrete solution
    assert A + B + C == pytest.approx(E * D, rel=1e-10, abs=0)
    # the continuum virial identity, to discretisation error
    assert abs(A - 3.0 * B - 0.5 * C + E * D) <= 2e-4 * E * D


def test_threshold_and_pump_relation():
    for kappa in (0.01, 0.1, 0.14, 1.0, 3.0):
        p = G.p_threshold(kappa)
        assert G.E_of_p(p, kappa) == pytest.approx(1.0, rel=1e-13, abs=0)
        assert G.E_of_p(1.0, kappa) == 0.0
    assert G.p_threshold(1e-6) == pytest.approx(1.0, abs=2e-6)


def test_peak_grows_and_width_is_finite_above_threshold():
    Es = [1.1, 2.0, 5.0, 10.0, 30.0]
    feats = [G.features(*G.solve(E)) for E in Es]
    peaks = [f[1] for f in feats]
    assert all(b > a for a, b in zip(peaks, peaks[1:]))
    assert all(0 < f[0] < 1 for f in feats)

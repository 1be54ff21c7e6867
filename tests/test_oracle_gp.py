"""Pins of the oracle's bound state of -phi'' + tau^2 phi + phi^3 = E phi
(the paper's Eq. g5, "Gross-Pitaevskii equation" paragraph) and of its
spectral features (CPU).  The oracle solves the continuum equation
(shooting for E <= 4, a collocation boundary-value solve above); every pin
below holds for the exact solution, whatever method produced it."""
import math

import numpy as np
import pytest

from oracle import gp_oracle as G


def test_near_threshold_closed_form():
    # The paper's first-order solution 2^{1/4} sqrt(E-1) exp(-tau^2/2) (the
    # oscillator's ground state with the amplitude fixed by projecting the
    # cubic term on it): the exact solution approaches it with a relative
    # error linear in E - 1, i.e. error / (E - 1) tends to a constant.
    tau = np.linspace(-8.0, 8.0, 4001)
    ratios = []
    for E in (1.001, 1.01):
        st = G.solve(E)
        ref = G.near_threshold(tau, E)
        err = np.linalg.norm(st(tau) - ref) / np.linalg.norm(ref)
        w, p = G.features(st)
        ew = w * 2.0 * math.sqrt(2.0) * math.pi - 1.0            # w -> 1/(2 sqrt2 pi)
        ep = p * math.sqrt(2.0) * math.pi / (E - 1.0) - 1.0      # p -> (E-1)/(sqrt2 pi)
        assert max(err, abs(ew), abs(ep)) < 0.3 * (E - 1.0), (E, err, ew, ep)
        ratios.append(np.array([err, ew, ep]) / (E - 1.0))
    # first order: the two ratios agree up to the O(E - 1) next term
    np.testing.assert_allclose(ratios[0], ratios[1], rtol=5e-3)


@pytest.mark.parametrize("E", [1.5, 4.0, 20.0, 60.0])
def test_integral_identities(E):
    # Both hold for every exact solution (boundary terms vanish at infinity):
    # the equation times phi, integrated by parts:
    #     int phi'^2 + int tau^2 phi^2 + int phi^4 = E int phi^2;
    # stationarity of int (phi'^2 + tau^2 phi^2 + phi^4/2 - E phi^2) under the
    # norm-preserving dilation phi -> sqrt(l) phi(l tau) (the virial):
    #     2 int phi'^2 - 2 int tau^2 phi^2 + int phi^4 / 2 = 0.
    st = G.solve(E)
    A, B, C, D = st.I2, st.I3, st.I4, st.I1
    assert st.a > 0 and st(np.linspace(-20, 20, 401)).min() >= 0.0
    assert A + B + C == pytest.approx(E * D, rel=1e-10, abs=0)
    assert abs(2 * A - 2 * B + 0.5 * C) <= 1e-10 * E * D


@pytest.mark.parametrize("E", [150.0, 300.0])
def test_thomas_fermi_limit(E):
    # Large E: phi^2 = E - tau^2 + phi''/phi; with phi'' of the leading
    # profile sqrt(E - tau^2) the bulk correction is -E/(E - tau^2)^2, so
    # phi^2 - (E - tau^2) over that correction tends to 1 (error O(1/E)),
    # phi(0)^2 = E - 1/E + ..., and the integrals tend to their Thomas-Fermi
    # values int phi = pi E / 2 (p_phi -> E^2/16) and int phi^2 = 4 E^{3/2}/3,
    # with relative corrections of order 1/E from the edge layer.
    st = G.solve(E)
    tau = np.linspace(0.0, math.sqrt(E / 2.0), 60)
    corr = -E / (E - tau ** 2) ** 2
    ratio = (st(tau) ** 2 - (E - tau ** 2)) / corr
    assert np.max(np.abs(ratio - 1.0)) < 1.0 / E
    assert st.a ** 2 == pytest.approx(E - 1.0 / E, rel=1e-2 / E ** 2, abs=0)
    w, p = G.features(st)
    assert abs(p / (E * E / 16.0) - 1.0) < 1.5 / E
    assert abs(st.I1 / (4.0 * E ** 1.5 / 3.0) - 1.0) < 0.1 / E


def test_shooting_and_boundary_value_solve_agree():
    # two unrelated continuum methods (bisection of an initial-value problem;
    # collocation of the boundary-value problem) where both are accurate
    tau = np.linspace(-7.0, 7.0, 281)
    for E in (2.0, 3.0):
        s = G.solve_shooting(E)
        b = G.solve_bvp_continuum(E)
        assert s.a == pytest.approx(b.a, rel=1e-9, abs=0)
        assert np.max(np.abs(s(tau) - b(tau))) <= 1e-8 * s.a
        for fs, fb in zip(G.features(s), G.features(b)):
            assert fs == pytest.approx(fb, rel=1e-8, abs=0)


@pytest.mark.parametrize("E", [3.0, 20.0, 60.0])
def test_features_from_the_fourier_transform(E):
    # The features by their definition: phi~(Omega) = int phi exp(i Omega tau)
    # taken numerically (FFT of phi on a fine grid; spectrally accurate for
    # the smooth, fast-decaying phi), then p = |phi~(0)|^2 / (4 pi^2) and
    # (2 pi w)^2 = int Omega^2 |phi~|^2 / int |phi~|^2 summed over the
    # discrete frequencies; the oracle takes both from tau-space integrals.
    st = G.solve(E)
    T = math.sqrt(E) + 10.0
    n = 1 << 15
    dtau = 2.0 * T / n
    tau = -T + dtau * np.arange(n)
    ft = np.fft.fft(st(tau)) * dtau
    om = 2.0 * math.pi * np.fft.fftfreq(n, d=dtau)
    S = np.abs(ft) ** 2
    w, p = G.features(st)
    assert p == pytest.approx(S[0] / (4.0 * math.pi ** 2), rel=1e-9, abs=0)
    sig2 = float(np.sum(om ** 2 * S) / np.sum(S))
    assert w == pytest.approx(math.sqrt(sig2) / (2.0 * math.pi), rel=1e-7, abs=0)


def test_threshold_and_pump_relation():
    for kappa in (0.01, 0.1, 0.14, 1.0, 3.0):
        p = G.p_threshold(kappa)
        assert G.E_of_p(p, kappa) == pytest.approx(1.0, rel=1e-13, abs=0)
        assert G.E_of_p(1.0, kappa) == 0.0
    assert G.p_threshold(1e-6) == pytest.approx(1.0, abs=2e-6)


def test_peak_grows_and_width_is_finite_above_threshold():
    Es = [1.1, 2.0, 5.0, 10.0, 30.0]
    feats = [G.features(G.solve(E)) for E in Es]
    peaks = [f[1] for f in feats]
    assert all(b > a for a, b in zip(peaks, peaks[1:]))
    assert all(0 < f[0] < 1 for f in feats)


def test_rejects_no_bound_state():
    for E in (1.0, 0.5, float("nan")):
        with pytest.raises(ValueError):
            G.solve(E)

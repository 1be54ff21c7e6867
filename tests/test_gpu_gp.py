"""The GPU bound-state solver of -phi'' + tau^2 phi + phi^3 = E phi (the
paper's Eq. g5) against the FP64 oracle, argument errors, and the theory
curves' threshold.

The GPU solves the equation discretised by second-order differences on the
grid tau_i = -L + i h (i = 1..n, h = 2L/(n+1), L = sqrt(E) + 8); the oracle
solves the continuum equation (shooting / collocation, no grid).  So the GPU
result differs from the oracle by the grid's truncation error, C h^2 +
O(h^4), and the test checks exactly that:

  * order: halving h (n = 2047 -> 4095) divides the error by 4 (3.8 .. 4.2)
    wherever the error is above the oracle's own accuracy;
  * consistency: the Richardson value (4 f(h/2) - f(h)) / 3 agrees with the
    oracle to 2e-8 (it removes the h^2 term; measured <= 4e-9);
  * size: the error at n = 2047 is within the leading-order bound.  The
    three-point second difference underestimates -phi'' by h^2/12 times the
    fourth derivative, which lowers the oscillator's ground state from 1 to
    1 - h^2/16 (the fourth derivative of exp(-tau^2/2), weighted by it,
    averages 3/4); near threshold the amplitude goes as sqrt(E - E_ground),
    so p (~ a^2) carries the relative error (h^2/16)/(E - 1) and the profile
    half of it; away from threshold the truncation error is below 0.05 h^2
    (measured <= 0.012 h^2).
"""
import math

import numpy as np
import pytest

from oracle import gp_oracle as G

pytestmark = pytest.mark.gpu

ES = [1.003, 1.01, 1.2, 2.0, 5.0, 20.0, 60.0, 150.0]
N1, N2 = 2047, 4095


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_0809_1547_gb300 import build
    build.build()


def _grid(E, n):
    L = math.sqrt(E) + 8.0
    h = 2.0 * L / (n + 1)
    return -L + h * np.arange(1, n + 1), h


def test_features_and_profiles_converge_to_the_oracle():
    from paper_0809_1547_gb300.binding import mb_gp_features
    w1, p1, phi1 = mb_gp_features(ES, N1, want_phi=True)
    w2, p2, phi2 = mb_gp_features(ES, N2, want_phi=True)
    for q, E in enumerate(ES):
        st = G.solve(E)
        w_o, p_o = G.features(st)
        tau1, h = _grid(E, N1)
        tau2, _ = _grid(E, N2)
        near = h * h / (16.0 * (E - 1.0))
        bounds = {"w": 0.05 * h * h, "p": 1.1 * near + 0.05 * h * h}
        for name, f1, f2, fo in (("w", w1[q], w2[q], w_o), ("p", p1[q], p2[q], p_o)):
            e1, e2 = f1 / fo - 1.0, f2 / fo - 1.0
            rich = ((4.0 * f2 - f1) / 3.0) / fo - 1.0
            assert abs(rich) <= 2e-8, (E, name, e1, e2, rich)
            assert abs(e1) <= bounds[name], (E, name, e1, bounds[name])
            if abs(e1) > 1e-6:
                assert 3.8 <= e1 / e2 <= 4.2, (E, name, e1, e2)
        ref1, ref2 = st(tau1), st(tau2)
        r1 = np.linalg.norm(phi1[q] - ref1) / np.linalg.norm(ref1)
        r2 = np.linalg.norm(phi2[q] - ref2) / np.linalg.norm(ref2)
        assert r1 <= 0.55 * near + 0.05 * h * h, (E, r1)
        if r1 > 1e-6:
            assert 3.8 <= r1 / r2 <= 4.2, (E, r1, r2)


def test_many_eigenvalues_at_once():
    from paper_0809_1547_gb300.binding import mb_gp_features
    E = np.geomspace(1.005, 400.0, 512)
    w, p = mb_gp_features(E, 1023)
    assert np.all(np.isfinite(w)) and np.all(p > 0)
    assert np.all(np.diff(p) > 0)                 # the peak grows with E


def test_argument_errors():
    from paper_0809_1547_gb300.binding import MBError, MB_ERR_ARG, mb_gp_features
    for bad in ([1.0], [0.5, 2.0], [float("nan")]):
        with pytest.raises(MBError) as e:
            mb_gp_features(bad, 255)
        assert e.value.code == MB_ERR_ARG
    with pytest.raises(MBError):
        mb_gp_features([2.0], 8)


def test_theory_curves():
    from paper_0809_1547_gb300 import gp
    kappa = 0.14                                  # the paper's best fit
    pth = gp.p_threshold(kappa)
    assert pth == pytest.approx(G.p_threshold(kappa), rel=1e-15, abs=0)
    p = pth * np.array([1.001, 1.5, 3.0, 10.0])
    c = gp.theory_curves(p, kappa)
    np.testing.assert_allclose(c["E"], G.E_of_p(p, kappa), rtol=1e-14)
    # near threshold the waist is the Gaussian one: W t_g -> sqrt(kappa/2) / (2 pi) / p^{1/4}
    assert c["W_tg"][0] == pytest.approx(math.sqrt(kappa / 2) / (2 * math.pi) / p[0] ** 0.25, rel=1e-2, abs=0)
    with pytest.raises(ValueError):
        gp.theory_curves([0.9 * pth], kappa)

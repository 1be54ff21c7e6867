"""The GPU bound-state solver of -phi'' + tau^2 phi + phi^3 = E phi against
the FP64 oracle (same discrete equations, independent implementations):
features and profiles within 1e-9, argument errors, and the theory curves'
threshold."""
import math

import numpy as np
import pytest

from oracle import gp_oracle as G

pytestmark = pytest.mark.gpu

ES = [1.003, 1.01, 1.2, 2.0, 5.0, 20.0, 60.0, 150.0]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_0809_1547_gb300 import build
    build.build()


def test_features_and_profiles_match_oracle():
    from paper_0809_1547_gb300.binding import mb_gp_features
    w, p, phi = mb_gp_features(ES, 2047, want_phi=True)
    for q, E in enumerate(ES):
        tau, h, ph_o = G.solve(E)
        w_o, p_o = G.features(tau, h, ph_o)
        assert w[q] == pytest.approx(w_o, rel=1e-9, abs=0), E
        assert p[q] == pytest.approx(p_o, rel=1e-9, abs=0), E
        assert np.linalg.norm(phi[q] - ph_o) <= 1e-9 * np.linalg.norm(ph_o), E


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

"""The coefficient tables the library builds on the host (no GPU), through the
mb_host_tables diagnostic, against the oracle's model.

CPML: the library's b, c of the E update (cell positions i) and of the H
update (positions i + 1/2) against the oracle's profiles at the same
positions, to FP32 rounding.  Gain: the device-unit coefficients against
the oracle's SI constants carried through the device scaling
(E_s = E/E0, P_s = P/(eps0 E0), J_s = J dt/(eps0 E0), n = N/N_a), and the
population update n' = n + g + G n + mk S against the oracle's Crank–Nicolson
propagator with N0 = N_a - N1 - N2 - N3 eliminated.
"""
import math

import numpy as np
import pytest

from oracle.mb_oracle import (EPS0, HBAR, Params, cpml_profile, crank_nicolson, gain_constants,
                              rate_matrix)
from paper_0809_1547_gb300.binding import MBError, MB_ERR_ARG, mb_default_params, mb_host_tables
from parity_util import DT, DX, params_kw


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_0809_1547_gb300 import build
    build.build()


@pytest.mark.parametrize("npml,grid", [(8, (40, 33, 17)), (4, (9, 64, 5)), (0, (12, 12, 12)),
                                       (6, (1, 1, 40))])
def test_cpml_tables_match_the_oracle_profiles(npml, grid):
    pkw = params_kw(npml=npml)
    tables, _, _ = mb_host_tables(grid, DX, DT, mb_default_params(**pkw))
    for w, n in zip("xyz", grid):
        bE, cE, bH, cH = tables[w]
        for half, b, c in ((0.0, bE, cE), (0.5, bH, cH)):
            bo, co = cpml_profile(n, half, DX, DT, Params(**pkw))
            np.testing.assert_allclose(b, bo.astype(np.float32), rtol=2.5e-7, atol=0, err_msg=f"b {w} {half}")
            np.testing.assert_allclose(c, co.astype(np.float32), rtol=2.5e-7, atol=0, err_msg=f"c {w} {half}")
    if npml and min(grid) > 2 * npml:
        bE = tables["x"][0]
        assert np.all(bE[npml + 1:grid[0] - npml] == 0)          # interior: no CPML
        assert np.all((bE[:npml] > 0) & (bE[:npml] < 1))        # decaying memories in the layer


@pytest.mark.parametrize("N_a,W_p", [(5e24, 1e13), (2e23, 3e12), (2e25, 0.0)])
def test_gain_coefficients_match_the_oracle_model(N_a, W_p):
    pkw = params_kw(npml=4)
    prm = mb_default_params(**pkw)
    _, g, E0 = mb_host_tables((10, 10, 10), DX, DT, prm, N_a, W_p)
    P = Params(**pkw)
    gc = gain_constants(P)
    w0, dw, xi, a_se = gc["w0"], gc["dw"], gc["xi"], gc["a_se"]
    assert E0 == pytest.approx(math.sqrt(HBAR * w0 * prm.n_ref / EPS0), rel=1e-14, abs=0)
    a = 0.5 * dw * DT
    # J^{n+1/2} (1 + a) = (1 - a) J^{n-1/2} + dt (xi dN E - w0^2 P + sigma_F zeta),
    # sigma_F = a_se sqrt(N2 / (dx^3 dt)), in device units
    expect = {"cJ1": (1 - a) / (1 + a),
              "cJE": DT * DT * xi * N_a / (EPS0 * (1 + a)),
              "cJP": (w0 * DT) ** 2 / (1 + a),
              "cJN": DT * DT * a_se * math.sqrt(N_a / (DX ** 3 * DT)) / (EPS0 * E0 * (1 + a)),
              "nfloor": P.n_floor_rel}
    for k, v in expect.items():
        assert g[k] == pytest.approx(v, rel=2e-7, abs=0), k
    M, m = crank_nicolson(rate_matrix(P, W_p), DT)
    # n_r' = M[r,0] (1 - sum n) + sum_q M[r,q] n_q  (r, q = 1..3), plus m_r S
    g_exp = M[1:, 0]
    G_exp = M[1:, 1:] - M[1:, 0][:, None] - np.eye(3)
    # S = (E_s + E_s').J_s / 2 = (E + E').J dt / (2 eps0 E0^2), and the oracle's
    # source term is m s with s = (E + E').J / (2 hbar w0) = S eps0 E0^2 / (hbar w0 dt)
    mk_exp = m[1:] * EPS0 * E0 * E0 / (HBAR * w0 * N_a * DT)
    np.testing.assert_allclose(g["g"], g_exp.astype(np.float32), rtol=2e-7, atol=0)
    np.testing.assert_allclose(g["G"], G_exp.astype(np.float32), rtol=2e-6, atol=1e-30)
    np.testing.assert_allclose(g["mk"], mk_exp.astype(np.float32), rtol=2e-7, atol=0)
    # the reference itself: the columns of A sum to zero, so those of M sum to
    # one and the step keeps N0 + N1 + N2 + N3
    np.testing.assert_allclose(M.sum(axis=0), 1.0, rtol=0, atol=1e-12)


def test_no_gain_gives_zero_coefficients_and_bad_arguments_are_rejected():
    prm = mb_default_params(**params_kw(npml=2))
    _, g, _ = mb_host_tables((4, 4, 4), DX, DT, prm, 0.0, 1e13)
    assert g["cJ1"] == 0 and np.all(g["G"] == 0) and np.all(g["mk"] == 0)
    for bad in (((0, 4, 4), DX, DT), ((4, 4, 4), -DX, DT), ((4, 4, 4), DX, 0.0)):
        with pytest.raises(MBError) as e:
            mb_host_tables(*bad, prm)
        assert e.value.code == MB_ERR_ARG

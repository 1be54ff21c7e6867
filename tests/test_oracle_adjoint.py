"""Pins of the oracle's discrete adjoint (CPU).

The gradient's definition is the derivative of the forward objective, so the
adjoint is pinned against central finite differences of the oracle's own
forward run (FP64, step h ~ 1e-4 relative: truncation ~1e-8, rounding
~1e-12), on single cells chosen to exercise every term of the reverse sweep
(bulk next to the source, CPML slab, gain cell, the objective's plane, a PEC
wall), on the pump rate, and along a random direction over all cells.  Three
regimes: a pulse-driven run with gain (Maxwell, CPML, Lorentz terms); a
noise-driven run with strong pumping and no source (the Langevin amplitude's
dependence on N2, the pump through the Crank–Nicolson propagator); a short
run from a preset strong-field state in which the field-driven population
transfer s dt is comparable to N_a (the inversion's feedback on J, the pump
through m s).  Each term of the reverse sweep was checked to matter: dropping
or flipping any one of them fails at least one of these cases.
"""
import math

import numpy as np
import pytest

from oracle.mb_oracle import MBOracle, Params, d_fwd, d_bwd, C0
from oracle.mb_adjoint import adjoint_energy_zface, energy_zface, crank_nicolson_dW
from oracle.mb_oracle import crank_nicolson, rate_matrix

DX = 20e-9
DT = 0.99 * DX / (C0 * math.sqrt(3.0))


def test_difference_transposes():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((5, 6, 7))
    y = rng.standard_normal((5, 6, 7))
    for ax in range(3):
        assert abs(np.sum(d_fwd(x, ax) * y) + np.sum(x * d_bwd(y, ax))) < 1e-12
        assert abs(np.sum(d_bwd(x, ax) * y) + np.sum(x * d_fwd(y, ax))) < 1e-12


def test_crank_nicolson_pump_derivative():
    p = Params()
    W, h = 3e12, 1e8
    dM, dm = crank_nicolson_dW(p, W, DT)
    Mp, mp = crank_nicolson(rate_matrix(p, W + h), DT)
    Mm, mm = crank_nicolson(rate_matrix(p, W - h), DT)
    np.testing.assert_allclose(dM, (Mp - Mm) / (2 * h), rtol=1e-6, atol=1e-30)
    np.testing.assert_allclose(dm, (mp - mm) / (2 * h), rtol=1e-6, atol=1e-40)


def _pulse_case():
    grid = (10, 9, 12)
    rng = np.random.default_rng(3)
    eps = np.where(rng.random(grid[::-1]) < 0.3, 8.41, 1.0)
    gain = (eps == 1.0).astype(np.uint8)
    cfg = dict(grid=grid, eps=eps, gain=gain, N_a=2e25, W_p=5e12, seed=77, steps=40,
               params=Params(npml=2),
               source=((5, 4, 5), 0, 560e-9, 1.0e-15, 0.4e-15, 5e13))
    return cfg


def _noise_case():
    grid = (8, 8, 10)
    rng = np.random.default_rng(4)
    eps = np.where(rng.random(grid[::-1]) < 0.25, 8.41, 1.0)
    gain = (eps == 1.0).astype(np.uint8)
    return dict(grid=grid, eps=eps, gain=gain, N_a=3e25, W_p=2e14, seed=1234, steps=30,
                params=Params(npml=2), source=None)


def _strong_field_case():
    """A short run from a preset state whose field-driven transfer s dt is
    comparable to N_a, so that the population terms of the reverse sweep
    (the inversion's feedback on J, the pump through m s) carry weight."""
    grid = (8, 7, 9)
    rng = np.random.default_rng(5)
    shp = grid[::-1]
    eps = np.where(rng.random(shp) < 0.3, 8.41, 1.0)
    gain = (eps == 1.0).astype(np.uint8)
    N_a = 1e23
    init = {}
    for c in "xyz":
        init["E" + c] = 1e8 * rng.standard_normal(shp)
        init["H" + c] = 1e8 / 376.73 * rng.standard_normal(shp)
        init["J" + c] = 1e12 * rng.standard_normal(shp)
        init["P" + c] = 1e12 * DT * rng.standard_normal(shp)
    frac = rng.dirichlet([4.0, 1.0, 3.0, 2.0], size=shp)
    for q in range(4):
        init[f"N{q}"] = N_a * frac[..., q] * gain
    return dict(grid=grid, eps=eps, gain=gain, N_a=N_a, W_p=1e13, seed=99, steps=6,
                params=Params(npml=1, tau10=20e-15, tau21=50e-15, tau32=20e-15), source=None,
                init=init)


def _oracle(cfg, eps=None, W_p=None):
    o = MBOracle(cfg["grid"], DX, DT, cfg["params"])
    o.set_material(cfg["eps"] if eps is None else eps, cfg["gain"], cfg["N_a"],
                   cfg["W_p"] if W_p is None else W_p)
    o.set_seed(cfg["seed"])
    if cfg["source"] is not None:
        o.add_source(*cfg["source"])
    for name, v in cfg.get("init", {}).items():
        o.set_field(name, v)
    return o


def _J(cfg, eps=None, W_p=None):
    return energy_zface(_oracle(cfg, eps, W_p), cfg["steps"])


def _cells(cfg):
    nx, ny, nz = cfg["grid"]
    g = cfg["gain"]
    gain_cell = tuple(np.argwhere(g[3:-3, 3:-3, 3:-3] != 0)[0] + 3)   # (k, j, i)
    zp = nz - cfg["params"].npml
    return {"bulk": (nz // 2, ny // 2, nx // 2 + 1), "cpml": (nz // 2, 1, nx // 2),
            "gain": gain_cell, "plane": (zp, ny // 2, nx // 2), "pec": (nz // 2, ny // 2, 0),
            "below_plane": (zp - 1, ny // 2 - 1, nx // 2)}


@pytest.mark.parametrize("case", ["pulse", "noise", "strong"])
def test_adjoint_gradient_matches_central_differences(case):
    cfg = {"pulse": _pulse_case, "noise": _noise_case, "strong": _strong_field_case}[case]()
    o = _oracle(cfg)
    res = adjoint_energy_zface(o, cfg["steps"])
    G = res["grad_eps"]
    assert res["J"] != 0.0
    scale = np.abs(G).max()
    assert scale > 0
    for name, kji in _cells(cfg).items():
        h = 1e-4 * cfg["eps"][kji]
        ep = cfg["eps"].copy()
        ep[kji] += h
        em = cfg["eps"].copy()
        em[kji] -= h
        fd = (_J(cfg, eps=ep) - _J(cfg, eps=em)) / (2 * h)
        assert abs(G[kji] - fd) <= 1e-6 * scale + 1e-7 * abs(fd), (name, G[kji], fd)
    # the pump rate
    hW = 1e-4 * cfg["W_p"]
    fdW = (_J(cfg, W_p=cfg["W_p"] + hW) - _J(cfg, W_p=cfg["W_p"] - hW)) / (2 * hW)
    assert fdW != 0.0
    assert abs(res["grad_pump"] - fdW) <= 1e-5 * abs(fdW), (res["grad_pump"], fdW)
    # a random direction over every cell
    d = np.random.default_rng(9).standard_normal(cfg["eps"].shape)
    t = 1e-5
    fdd = (_J(cfg, eps=cfg["eps"] + t * d) - _J(cfg, eps=cfg["eps"] - t * d)) / (2 * t)
    ad = float(np.sum(G * d))
    assert abs(ad - fdd) <= 1e-6 * (abs(fdd) + np.abs(G).sum() * 1e-3), (ad, fdd)


def test_objective_is_the_face_flux():
    cfg = _pulse_case()
    o = _oracle(cfg)
    res = adjoint_energy_zface(o, cfg["steps"])
    assert res["J"] == pytest.approx(o.flux[5], rel=1e-12, abs=0.0)
    assert res["J"] != 0.0


def test_gradient_of_a_linear_passive_run_scales_quadratically():
    """Passive medium (no gain): fields are linear in the source amplitude and
    J is bilinear in the fields, so J and dJ/deps scale as amp^2."""
    cfg = _pulse_case()
    cfg["N_a"] = 0.0
    r1 = adjoint_energy_zface(_oracle(cfg), cfg["steps"])
    cfg2 = dict(cfg)
    src = list(cfg["source"])
    src[-1] *= 3.0
    cfg2["source"] = tuple(src)
    r3 = adjoint_energy_zface(_oracle(cfg2), cfg["steps"])
    assert r3["J"] == pytest.approx(9.0 * r1["J"], rel=1e-10, abs=0)
    np.testing.assert_allclose(r3["grad_eps"], 9.0 * r1["grad_eps"], rtol=1e-9,
                               atol=1e-12 * np.abs(r1["grad_eps"]).max())
    assert r1["grad_pump"] == 0.0

"""GPU reverse-time adjoint (through the C ABI) against the oracle's FP64
discrete adjoint and against finite differences.

Bar: the objective J, the eps-gradient (relative L2 over all cells) and the
pump gradient within 1e-5 of the oracle's adjoint on identical inputs and
noise (the field bar of the forward step; measured errors are 1e-7 to 2e-6),
in the pulse-driven, noise-driven and strong-field regimes that pin the
oracle's adjoint, and on a grid spanning several thread blocks with ragged
tails.  The gradient is bit-identical for any checkpoint interval (the
recomputation reproduces the forward bit for bit), and the call leaves the
context exactly where mb_step would.  At the full 96^3, 4000-step workload
(checkpoints every 200 steps) the gradient is checked against central
differences of the GPU forward run itself.
"""
import math

import numpy as np
import pytest

from oracle.mb_oracle import MBOracle, Params, FIELD_NAMES
from oracle.mb_adjoint import adjoint_energy_zface
from parity_util import params_kw, rel_l2

pytestmark = pytest.mark.gpu

DX = 20e-9
DT = 0.99 * DX / (299_792_458.0 * math.sqrt(3.0))
TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_0809_1547_gb300 import build
    build.build()


def _cases():
    import test_oracle_adjoint as T
    from paper_0809_1547_gb300 import inputs
    grid = (40, 20, 24)
    eps, gain = inputs.random_small(grid, seed=3, npml=4, d_cells=5)
    big = dict(grid=grid, eps=eps.astype(np.float64), gain=gain, N_a=2e25, W_p=5e12, seed=77,
               steps=60, params=Params(npml=4),
               source=((20, 10, 12), 0, 560e-9, 1.0e-15, 0.4e-15, 5e13))
    return {"pulse": T._pulse_case(), "noise": T._noise_case(), "strong": T._strong_field_case(),
            "multi_block": big}


def _oracle(cfg):
    import test_oracle_adjoint as T
    return T._oracle(cfg)


def _gpu(cfg, eps=None, W_p=None):
    from paper_0809_1547_gb300.binding import MBSimulation, mb_default_params
    p = cfg["params"]
    pk = params_kw(npml=p.npml, tau10=p.tau10, tau21=p.tau21, tau32=p.tau32)
    g = MBSimulation(cfg["grid"], DX, DT, mb_default_params(**pk))
    g.set_material(cfg["eps"] if eps is None else eps, cfg["gain"], cfg["N_a"],
                   cfg["W_p"] if W_p is None else W_p)
    g.set_seed(cfg["seed"])
    if cfg["source"] is not None:
        g.set_source(*cfg["source"])
    for name, v in cfg.get("init", {}).items():
        if name != "N0":          # derived on the GPU (the fractions sum to N_a)
            g.set_field(name, v)
    return g


@pytest.mark.parametrize("case", ["pulse", "noise", "strong", "multi_block"])
def test_adjoint_matches_oracle_adjoint(case):
    cfg = _cases()[case]
    res = adjoint_energy_zface(_oracle(cfg), cfg["steps"])
    g = _gpu(cfg)
    J, G, gp = g.adjoint_energy_zface(cfg["steps"], 7)
    G = G.cpu().numpy().astype(np.float64)
    g.close()
    assert abs(J - res["J"]) <= TOL * abs(res["J"]), (J, res["J"])
    err = rel_l2(G, res["grad_eps"])
    assert err <= TOL, err
    assert abs(gp - res["grad_pump"]) <= TOL * abs(res["grad_pump"]), (gp, res["grad_pump"])


def test_checkpoint_interval_does_not_change_the_gradient():
    cfg = _cases()["multi_block"]
    out = []
    for K in (1, 7, 60, 1000):
        g = _gpu(cfg)
        J, G, gp = g.adjoint_energy_zface(cfg["steps"], K)
        out.append((J, G.cpu().numpy(), gp))
        g.close()
    for J, G, gp in out[1:]:
        np.testing.assert_array_equal(G, out[0][1])
        assert J == pytest.approx(out[0][0], rel=1e-12, abs=0)
        assert gp == pytest.approx(out[0][2], rel=1e-12, abs=0)


def test_adjoint_call_leaves_the_forward_state():
    cfg = _cases()["multi_block"]
    a = _gpu(cfg)
    b = _gpu(cfg)
    pa = a.add_point_probe((10, 10, 12), 16, 500e-9, 650e-9)
    pb = b.add_point_probe((10, 10, 12), 16, 500e-9, 650e-9)
    J, _, _ = a.adjoint_energy_zface(cfg["steps"], 16)
    b.step(cfg["steps"])
    assert a.n == b.n == cfg["steps"]
    for name in FIELD_NAMES:
        np.testing.assert_array_equal(a.field(name), b.field(name))
    np.testing.assert_array_equal(a.probe_spectrum(pa)[0], b.probe_spectrum(pb)[0])
    fb = b.flux()
    assert J == pytest.approx(fb[5], rel=1e-6, abs=0)     # the +z face is the default plane
    np.testing.assert_allclose(a.flux(), fb, rtol=1e-12)
    # continuing from there matches as well
    a.step(5)
    b.step(5)
    np.testing.assert_array_equal(a.field("Ez"), b.field("Ez"))
    a.close()
    b.close()


def test_autograd_function():
    import torch
    from paper_0809_1547_gb300.autograd import Realization, emitted_energy
    from paper_0809_1547_gb300.binding import mb_default_params
    cfg = _cases()["pulse"]
    r = Realization(grid=cfg["grid"], dx=DX, dt=DT, gain_mask=cfg["gain"], N_a=cfg["N_a"],
                    seed=cfg["seed"], n_steps=cfg["steps"], ckpt_every=9,
                    params=mb_default_params(**params_kw(npml=cfg["params"].npml)),
                    sources=[cfg["source"]])
    eps = torch.tensor(cfg["eps"], dtype=torch.float32, device="cuda", requires_grad=True)
    pump = torch.tensor(cfg["W_p"], dtype=torch.float64, requires_grad=True)
    J = emitted_energy(eps, pump, r)
    (3.0 * J).backward()
    res = adjoint_energy_zface(_oracle(cfg), cfg["steps"])
    assert float(J.detach()) == pytest.approx(res["J"], rel=TOL, abs=0)
    assert rel_l2(eps.grad.cpu().numpy() / 3.0, res["grad_eps"]) <= TOL
    assert float(pump.grad) / 3.0 == pytest.approx(res["grad_pump"], rel=TOL, abs=0)


def test_adjoint_argument_errors():
    from paper_0809_1547_gb300.binding import (MBError, MBSimulation, MB_ERR_ARG, MB_ERR_STATE,
                                                mb_adjoint_energy_zface, mb_default_params)
    g = MBSimulation((8, 8, 8), DX, DT, mb_default_params(npml=2))
    with pytest.raises(MBError) as e:
        mb_adjoint_energy_zface(g.handle, 4)
    assert e.value.code == MB_ERR_STATE
    g.set_material(np.ones((8, 8, 8)), np.zeros((8, 8, 8)), 0.0, 0.0)
    for n, zp in ((0, -1), (4, 0), (4, 8), (4, 99)):
        with pytest.raises(MBError) as e:
            mb_adjoint_energy_zface(g.handle, n, 2, zp)
        assert e.value.code == MB_ERR_ARG
    assert g.n == 0
    g.close()


def test_full_size_96_gradient_against_finite_differences():
    """96^3, 225 spheres (45 % fill), gain in the voids, fixed pump and noise
    seed, 4000 steps, checkpoints every 200 steps.  Central differences of the
    GPU forward run (second-order one-sided ones at eps = 1, the lower bound
    of eps): the pump (h = 1e-2 W_p, bound 1e-4), a random direction over the
    sphere cells (t = 1e-3, bound 1e-2) and one over every cell (t = 1e-4,
    bound 3e-2), and 32 seeded random cells of the CPML-free interior (h =
    1e-2 eps; bound 10 % of the difference plus 3 % of the largest sampled
    gradient).  The bounds are the finite differences' own error: 4000 noisy
    steps respond nonlinearly to larger steps, and the FP32 forward's rounding
    puts a floor of ~1e-23 J (3 % of the largest sampled gradient) under
    single-cell differences."""
    from paper_0809_1547_gb300 import inputs
    from paper_0809_1547_gb300.binding import MBSimulation, mb_default_params
    w = inputs.workload_adjoint_96()
    K = w.extra["ckpt_every"]

    def sim(eps, W):
        s = MBSimulation(w.grid, w.dx, w.dt, mb_default_params(npml=w.npml))
        s.set_material(eps, w.gain, w.N_a, W)
        s.set_seed(w.seed)
        return s

    def J_of(eps, W=w.pump):
        s = sim(eps, W)
        s.step(w.steps)
        v = s.flux()[5]
        s.close()
        return v

    s = sim(w.eps, w.pump)
    J, G, gp = s.adjoint_energy_zface(w.steps, K)
    s.close()
    G = G.cpu().numpy().astype(np.float64)
    assert J == pytest.approx(J_of(w.eps), rel=1e-6, abs=0)
    assert np.isfinite(G).all() and np.abs(G).max() > 0
    hW = 1e-2 * w.pump
    fdW = (J_of(w.eps, w.pump + hW) - J_of(w.eps, w.pump - hW)) / (2 * hW)
    assert abs(gp - fdW) <= 1e-4 * abs(fdW), (gp, fdW)
    # random directions: over the sphere cells (central, t = 1e-3) and over
    # every cell (voids only upwards, second-order one-sided, t = 1e-4)
    z = np.random.default_rng(11).standard_normal(w.eps.shape)
    ds = np.where(w.eps > 1.0, w.eps * z, 0.0)
    t = 1e-3
    fds = (J_of(w.eps + t * ds) - J_of(w.eps - t * ds)) / (2 * t)
    ads = float(np.sum(G * ds))
    assert abs(ads - fds) <= 1e-2 * abs(fds), (ads, fds)
    da = np.where(w.eps > 1.0, w.eps * z, np.abs(z))
    t = 1e-4
    fda = (-3.0 * J + 4.0 * J_of(w.eps + t * da) - J_of(w.eps + 2 * t * da)) / (2 * t)
    ada = float(np.sum(G * da))
    assert abs(ada - fda) <= 3e-2 * abs(fda), (ada, fda)
    rng = np.random.default_rng(2024)
    L = w.npml
    bad = []
    cells = [tuple(int(v) for v in rng.integers(L, w.grid[0] - L, size=3)) for _ in range(32)]
    vals = []
    for kji in cells:
        e = float(w.eps[kji])
        h = 1e-2 * e
        if e - h >= 1.0:
            ep, em = w.eps.copy(), w.eps.copy()
            ep[kji] += h
            em[kji] -= h
            fd = (J_of(ep) - J_of(em)) / (2 * h)
        else:
            e1, e2 = w.eps.copy(), w.eps.copy()
            e1[kji] += h
            e2[kji] += 2 * h
            fd = (-3.0 * J + 4.0 * J_of(e1) - J_of(e2)) / (2 * h)
        vals.append((kji, G[kji], fd))
    gmax = max(abs(v[1]) for v in vals)
    for kji, g_ad, fd in vals:
        if abs(g_ad - fd) > 0.1 * abs(fd) + 0.03 * gmax:
            bad.append((kji, g_ad, fd))
    assert not bad, bad

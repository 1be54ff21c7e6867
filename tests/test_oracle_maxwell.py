"""Pins of the oracle's Yee curl updates, PEC walls and discrete energy.

The exact discrete eigenmodes of a PEC box are written here from the
discrete Fourier symbols of the forward/backward differences, not from the
oracle's update code: with s_w = (2/dx) sin(k_w dx/2) the curl of a mode is
s x A, and a leapfrog mode oscillates at the frequency fixed by the Yee
dispersion relation (2/dt)^2 sin^2(w dt/2) = (c^2/eps_r) |s|^2.
"""
import math

import numpy as np
import pytest

from oracle.mb_oracle import MBOracle, Params, C0, EPS0, MU0

DX = 20e-9
DT = 0.99 * DX / (C0 * math.sqrt(3.0))


def _mode_fields(grid, modes, amp_dir, eps_r, n):
    """E^n and H^{n-1/2} of the exact discrete cavity mode on the Yee sites."""
    nx, ny, nz = grid
    k = [m * math.pi / (nw * DX) for m, nw in zip(modes, grid)]
    s = np.array([2.0 / DX * math.sin(kw * DX / 2.0) for kw in k])
    A = np.cross(s, np.asarray(amp_dir, dtype=float))       # s . A = 0
    A /= np.linalg.norm(A)
    omega = 2.0 / DT * math.asin(DT / 2.0 * C0 / math.sqrt(eps_r) * np.linalg.norm(s))
    B = -(DT / MU0) * np.cross(s, A) / (2.0 * math.sin(omega * DT / 2.0))
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    x_int, y_int, z_int = ii * DX, jj * DX, kk * DX
    x_h, y_h, z_h = (ii + 0.5) * DX, (jj + 0.5) * DX, (kk + 0.5) * DX
    S, Cs = np.sin, np.cos
    te = math.cos(omega * n * DT)
    th = math.sin(omega * (n - 0.5) * DT)
    E = {
        "Ex": A[0] * Cs(k[0] * x_h) * S(k[1] * y_int) * S(k[2] * z_int) * te,
        "Ey": A[1] * S(k[0] * x_int) * Cs(k[1] * y_h) * S(k[2] * z_int) * te,
        "Ez": A[2] * S(k[0] * x_int) * S(k[1] * y_int) * Cs(k[2] * z_h) * te,
    }
    H = {
        "Hx": B[0] * S(k[0] * x_int) * Cs(k[1] * y_h) * Cs(k[2] * z_h) * th,
        "Hy": B[1] * Cs(k[0] * x_h) * S(k[1] * y_int) * Cs(k[2] * z_h) * th,
        "Hz": B[2] * Cs(k[0] * x_h) * Cs(k[1] * y_h) * S(k[2] * z_int) * th,
    }
    return E, H, omega


@pytest.mark.parametrize("grid,modes,amp_dir,eps_r", [
    ((12, 10, 14), (1, 2, 1), (0.3, -0.7, 1.1), 1.0),
    ((9, 16, 11), (2, 1, 3), (1.0, 0.2, -0.4), 2.5),
    ((16, 16, 6), (3, 1, 0), (0.0, 0.0, 1.0), 8.41),     # TM_z mode (E along z)
])
def test_pec_cavity_eigenmode(grid, modes, amp_dir, eps_r):
    sim = MBOracle(grid, DX, DT, Params(npml=0))
    sim.set_material(np.full(grid[::-1], eps_r), np.zeros(grid[::-1]), 0.0, 0.0)
    E0, H0, _ = _mode_fields(grid, modes, amp_dir, eps_r, 0)
    for name, v in {**E0, **H0}.items():
        sim.set_field(name, v)
    n = 150
    sim.step(n)
    En, Hn, _ = _mode_fields(grid, modes, amp_dir, eps_r, n + 0)
    # after n steps the oracle holds E^n and H^{n-1/2}
    scaleE = max(np.abs(v).max() for v in E0.values())
    scaleH = max(np.abs(v).max() for v in H0.values()) or 1.0
    for name, v in En.items():
        np.testing.assert_allclose(sim.field(name), v, rtol=0, atol=1e-10 * scaleE)
    for name, v in Hn.items():
        np.testing.assert_allclose(sim.field(name), v, rtol=0, atol=1e-10 * max(scaleH, 1e-30))


def test_mode_frequency_matches_vacuum_plane_wave_dispersion():
    # k along x only is the 1D limit of the relation the mode test uses:
    # sin(w dt/2) = (c dt/dx) sin(k dx/2); check the helper reproduces it.
    nx = 40
    grid = (nx, 8, 8)
    k = math.pi / (nx * DX)
    w_expect = 2.0 / DT * math.asin(C0 * DT / DX * math.sin(k * DX / 2.0))
    _, _, w = _mode_fields(grid, (1, 0, 0), (0, 0, 1), 1.0, 0)
    assert abs(w - w_expect) / w_expect < 1e-14
    # and the numerical phase velocity lags c
    assert w / k < C0


def test_yee_energy_invariant_pec_box():
    """W^n = 1/2 sum eps|E^n|^2 + 1/2 sum mu0 H^{n-1/2}.H^{n+1/2} is constant."""
    grid = (10, 9, 11)
    rng = np.random.default_rng(11)
    sim = MBOracle(grid, DX, DT, Params(npml=0))
    eps = rng.uniform(1.0, 8.41, size=grid[::-1])
    sim.set_material(eps, np.zeros(grid[::-1]), 0.0, 0.0)
    for name in ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz"):
        scale = 1.0 if name[0] == "E" else 1.0 / 377.0
        sim.set_field(name, rng.standard_normal(grid[::-1]) * scale)
    # tangential E on the low walls starts at zero, as the walls impose
    sim.step(0)
    Ex, Ey, Ez = sim.E
    Ex[:, 0, :] = 0; Ex[0, :, :] = 0
    Ey[:, :, 0] = 0; Ey[0, :, :] = 0
    Ez[:, :, 0] = 0; Ez[:, 0, :] = 0
    dV = DX ** 3
    W = []
    for _ in range(60):
        E_n = [F.copy() for F in sim.E]
        H_minus = [F.copy() for F in sim.H]
        sim.step(1)
        H_plus = sim.H
        w = 0.5 * EPS0 * sum(np.sum(eps * F * F) for F in E_n) * dV
        w += 0.5 * MU0 * sum(np.sum(a * b) for a, b in zip(H_minus, H_plus)) * dV
        W.append(w)
    W = np.array(W)
    assert np.max(np.abs(W - W[0])) / abs(W[0]) < 1e-12
    # the plain energy U is NOT invariant (it oscillates), so the test has teeth
    U0 = sim.energy()
    sim.step(1)
    assert abs(sim.energy() - U0) / U0 > 1e-6


def test_courant_limit_rejected():
    with pytest.raises(ValueError):
        MBOracle((4, 4, 4), DX, 1.001 * DX / (C0 * math.sqrt(3.0)))

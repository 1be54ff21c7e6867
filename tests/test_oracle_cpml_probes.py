"""Pins of the oracle's CPML, running-DFT probes and Poynting face flux."""
import math

import numpy as np
import pytest

from oracle.mb_oracle import MBOracle, Params, C0, EPS0, MU0, cpml_profile, dft_accumulate

DX = 20e-9
DT = 0.99 * DX / (C0 * math.sqrt(3.0))
LAM_S, TAU_S = 400e-9, 0.4e-15
T0_S = 3 * TAU_S


def _pulse_run(grid, npml, src, probe, steps):
    """A broadband pulse from a soft current with x, y and z parts (so that
    every field component, Hz included, is driven); the six field components
    at a probe cell off the source's axes, per step (H scaled by eta0)."""
    sim = MBOracle(grid, DX, DT, Params(npml=npml))
    shp = grid[::-1]
    sim.set_material(np.ones(shp), np.zeros(shp), 0.0, 0.0)
    for comp, amp in ((0, 0.6e9), (1, -0.8e9), (2, 1e9)):
        sim.add_source(src, comp, LAM_S, T0_S, TAU_S, amp)
    i, j, k = probe
    eta0 = MU0 * C0
    trace = []
    for _ in range(steps):
        sim.step(1)
        trace.append([F[k, j, i] for F in sim.E] + [eta0 * F[k, j, i] for F in sim.H])
    return np.array(trace), sim


def test_cpml_coefficients_shape():
    p = Params()
    b, c = cpml_profile(40, 0.0, DX, DT, p)
    inside = np.r_[0:8, 33:40]
    assert np.all((b[inside] > 0) & (b[inside] < 1)) and np.all(c[inside] < 0)
    assert np.all(b[8:33] == 0) and np.all(c[8:33] == 0)
    # sigma grows towards the wall: |c| is largest at the wall
    assert abs(c[0]) == abs(c).max()
    bh, ch = cpml_profile(40, 0.5, DX, DT, p)
    np.testing.assert_allclose(ch[:8], ch[::-1][:8])   # symmetric about the centre


def test_cpml_reflection_against_larger_box():
    """All six components at a cell off the source's axes, 2 cells from the
    layer's inner edge, against a box large enough that no wall echo returns
    within the run: the CPML's reflection stays below 1e-3 of the peak (a
    CPML with a memory missing, a wrong grading or profiles taken half a cell
    off reflects 2-4e-2)."""
    steps = 100
    # small box: 28^3 with 8 CPML cells per face
    small, _ = _pulse_run((28, 28, 28), 8, (14, 14, 14), (17, 12, 18), steps)
    # reference: 64^3 PEC box, same source-probe offset, wall echoes arrive after ~105 steps
    ref, _ = _pulse_run((64, 64, 64), 0, (32, 32, 32), (35, 30, 36), steps)
    # the same small box without the CPML reflects strongly (the test has teeth)
    pec, _ = _pulse_run((28, 28, 28), 0, (14, 14, 14), (17, 12, 18), steps)
    peak = np.abs(ref).max()
    err_cpml = np.abs(small - ref).max() / peak
    err_pec = np.abs(pec - ref).max() / peak
    assert err_cpml < 1e-3
    assert err_pec > 100 * err_cpml


def test_point_probe_dft_of_cavity_mode():
    """A TM_z cavity mode gives E_z^n = A cos(w_m n dt): its running DFT is a geometric sum."""
    grid = (16, 16, 4)
    sim = MBOracle(grid, DX, DT, Params(npml=0))
    shp = grid[::-1]
    sim.set_material(np.ones(shp), np.zeros(shp), 0.0, 0.0)
    kk, jj, ii = np.meshgrid(np.arange(4), np.arange(16), np.arange(16), indexing="ij")
    kx = ky = math.pi / (16 * DX)
    s = 2 / DX * math.sin(kx * DX / 2)
    w_m = 2 / DT * math.asin(DT / 2 * C0 * math.sqrt(2) * s)
    Bx = -(DT / MU0) * s / (2 * math.sin(w_m * DT / 2))    # (s x z_hat)_x = s_y
    sim.set_field("Ez", np.sin(kx * ii * DX) * np.sin(ky * jj * DX))
    sim.set_field("Hx", Bx * np.sin(kx * ii * DX) * np.cos(ky * (jj + 0.5) * DX) * math.sin(-w_m * DT / 2))
    sim.set_field("Hy", -Bx * np.cos(kx * (ii + 0.5) * DX) * np.sin(ky * jj * DX) * math.sin(-w_m * DT / 2))
    ijk = (5, 9, 2)
    lam_m = 2 * math.pi * C0 / w_m
    pid = sim.add_point_probe(ijk, 7, 0.8 * lam_m, 1.2 * lam_m)
    N = 300
    sim.step(N)
    S, lams = sim.probe_spectrum(pid)
    A = math.sin(kx * ijk[0] * DX) * math.sin(ky * ijk[1] * DX)
    def G(q):   # sum_{n=1..N} exp(i q n dt)
        if abs(1 - np.exp(1j * q * DT)) < 1e-9:
            return float(N)
        return np.exp(1j * q * DT) * (1 - np.exp(1j * q * N * DT)) / (1 - np.exp(1j * q * DT))

    expect = []
    for lam in lams:
        w = 2 * math.pi * C0 / lam
        ft = A * DT / 2 * (G(w + w_m) + G(w - w_m))
        expect.append(abs(ft) ** 2)
    np.testing.assert_allclose(S, expect, rtol=1e-8)
    # the mode line sits in the middle bin
    assert int(np.argmax(S)) == 3
    # dft_accumulate on its own
    acc = dft_accumulate(np.zeros(3, complex), 2.0, np.array([1e15, 2e15, 3e15]), 1e-15, 0.5)
    np.testing.assert_allclose(acc, np.exp(1j * np.array([1.0, 2.0, 3.0])))


def _box_energy_mixed(sim, E_n, H_minus, H_plus):
    """W_V^n = 1/2 sum_V eps E^n.E^n + 1/2 sum_V mu0 H^{n-1/2}.H^{n+1/2} over the interior box."""
    L = sim.p.npml
    sl = (slice(L, sim.nz - L), slice(L, sim.ny - L), slice(L, sim.nx - L))
    uE = sum(np.sum((sim.eps_r * F * F)[sl]) for F in E_n) * EPS0
    uH = sum(np.sum((a * b)[sl]) for a, b in zip(H_minus, H_plus)) * MU0
    return 0.5 * (uE + uH) * DX ** 3


def _energy_at(sim):
    """Advance one step and return (W_V^n, flux accumulated before the step)."""
    E_n = [F.copy() for F in sim.E]
    H_minus = [F.copy() for F in sim.H]
    flux_before = sim.flux.copy()
    sim.step(1)
    return _box_energy_mixed(sim, E_n, H_minus, sim.H), flux_before


def test_face_flux_balances_interior_energy_exactly():
    """Lossless source-free interior: W_V^{n2} - W_V^{n1} = -(sum of outward face flux)."""
    grid = (30, 28, 32)
    sim = MBOracle(grid, DX, DT, Params(npml=8))
    shp = grid[::-1]
    eps = np.ones(shp)
    eps[14:18, 13:17, 15:19] = 4.0
    sim.set_material(eps, np.zeros(shp), 0.0, 0.0)
    sim.add_source((15, 14, 16), 0, LAM_S, T0_S, TAU_S, 1e9)
    sim.step(45)
    sim.sources.clear()
    W1, F1 = _energy_at(sim)
    sim.step(60)
    W2, F2 = _energy_at(sim)
    out = float(np.sum(F2 - F1))
    assert out > 0.2 * W1                      # a good part of the energy has left
    assert abs((W1 - W2) - out) < 1e-9 * W1    # exact up to round-off
    # outward flux is positive on every face once the pulse radiates away
    assert np.all(F2 - F1 > 0)


@pytest.mark.parametrize("every,stride", [(1, 1), (3, 1), (1, 2)])
def test_face_spectra_parseval(every, stride):
    """sum_n dt F(t_n) = (1/pi) int_0^inf Re(E~ x H~*) . n dw for a pulse that
    has left; a face sub-grid of every stride-th point (weighted by its
    (stride dx)^2 area) is another quadrature of the same face integral."""
    grid = (26, 26, 26)
    sim = MBOracle(grid, DX, DT, Params(npml=8))
    shp = grid[::-1]
    sim.set_material(np.ones(shp), np.zeros(shp), 0.0, 0.0)
    tau = 2e-15
    sim.add_source((13, 13, 13), 0, 532e-9, 4 * tau, tau, 1e9)
    sim.add_face_probes(stride, every, 400, 330e-9, 1100e-9)
    sim.step(560)
    total_time = float(np.sum(sim.flux))
    total_freq = 0.0
    for face in range(6):
        S, lams = sim.face_spectrum(face)
        w = 2 * math.pi * C0 / lams
        order = np.argsort(w)
        total_freq += np.trapezoid(S[order], w[order]) / math.pi
    assert total_time > 0
    assert abs(total_freq / total_time - 1) < 0.02

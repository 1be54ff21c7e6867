"""Pins of the oracle's gain medium: Lorentz recursion, Langevin force, populations.

Closed forms used here (derived from the discrete scheme, not read from the
oracle's code):
  * Lorentz recursion: eliminating J = (P^{n+1} - P^n)/dt gives
    (1+a)(P^{n+1}-P^n) - (1-a)(P^n-P^{n-1}) + (w0 dt)^2 P^n = dt^2 (xi dN E^n + F^n),
    so a harmonic drive E^n = Re(z^n), z = exp(i w dt), has the response
    P^n = Re(H(z) z^n) with H(z) = dt^2 xi dN / [(1+a)(z-1) - (1-a)(1-1/z) + (w0 dt)^2],
    and a white force of variance q^2 gives Var P = q^2 dt^4/(2 pi) int |1/D(e^{it})|^2 dt.
  * Rate equations: the steady state of dN/dt = A N with sum N = N_a is
    N0* = N_a / (1 + W_p (tau32 + tau21 + tau10)), N3* = W_p tau32 N0*,
    N2* = W_p tau21 N0*, N1* = W_p tau10 N0*; the Crank–Nicolson iterate
    approaches expm(A t) N(0) with a local error dt^3 |A^3 N| / 12.
"""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle.mb_oracle import (MBOracle, Params, C0, EPS0, MU0, HBAR, gain_constants, lorentz_update,
                              rate_matrix, crank_nicolson, population_update)

DX = 20e-9
DT = 0.99 * DX / (C0 * math.sqrt(3.0))
P0 = Params()
GC = gain_constants(P0)


def _den(z, a, w0dt):
    return (1 + a) * (z - 1) - (1 - a) * (1 - 1 / z) + w0dt ** 2


@pytest.mark.parametrize("lam", [450e-9, 590e-9, 700e-9])
def test_lorentz_recursion_harmonic_response(lam):
    w0, dw, xi = GC["w0"], GC["dw"], GC["xi"]
    a = 0.5 * dw * DT
    dN = -3e24
    w = 2 * math.pi * C0 / lam
    z = np.exp(1j * w * DT)
    H = DT ** 2 * xi * dN / _den(z, a, w0 * DT)
    J = P = 0.0
    n_steps = 3000          # transients decay like exp(-dw t / 2): e^-70 here
    for n in range(n_steps):
        E = math.cos(w * n * DT)
        J, P = lorentz_update(J, P, E, dN, 0.0, DT, w0, dw, xi)
    expect = (H * z ** n_steps).real
    assert abs(P - expect) <= 1e-9 * abs(H)


def test_lorentz_recursion_continuous_limit_is_the_lorentzian():
    """The discrete susceptibility approaches xi dN/(eps0 (w0^2 - w^2 + i w dw))."""
    w0, dw, xi = GC["w0"], GC["dw"], GC["xi"]
    a = 0.5 * dw * DT
    for w in np.linspace(0.6 * w0, 1.4 * w0, 9):
        z = np.exp(1j * w * DT)
        chi_d = DT ** 2 * xi / _den(z, a, w0 * DT)
        chi_c = xi / (w0 ** 2 - w ** 2 + 1j * w * dw)
        assert abs(chi_d - chi_c) / abs(chi_c) < 3 * (w * DT) ** 2
    # resonance at w0 and gain line-width dw (the paper's 230 nm ~ 1/t_g)
    assert abs(dw - 2 * math.pi * C0 * 230e-9 / 590e-9 ** 2) < 1e-6 * dw
    assert abs(1 / dw - 0.80e-15) < 0.01e-15


def test_lorentz_noise_stationary_variance():
    w0, dw, xi = GC["w0"], GC["dw"], GC["xi"]
    a = 0.5 * dw * DT
    theta = np.linspace(-np.pi, np.pi, 20001)[:-1]
    gain2 = np.mean(np.abs(1.0 / _den(np.exp(1j * theta), a, w0 * DT)) ** 2)
    q = 1.0
    var_expect = q ** 2 * DT ** 4 * gain2
    rng = np.random.default_rng(5)
    m = 20000
    J = np.zeros(m)
    P = np.zeros(m)
    for _ in range(600):     # > 10 damping times (2/dw = 42 steps)
        J, P = lorentz_update(J, P, 0.0, 0.0, q * rng.standard_normal(m), DT, w0, dw, xi)
    samples = []
    for _ in range(4):
        for _ in range(100):
            J, P = lorentz_update(J, P, 0.0, 0.0, q * rng.standard_normal(m), DT, w0, dw, xi)
        samples.append(np.mean(P * P))
    var = np.mean(samples)
    assert abs(var / var_expect - 1) < 0.03


def test_langevin_force_amplitude_after_one_step():
    """From rest, one step gives J = dt sigma_F zeta / (1 + a) in every gain cell."""
    grid = (16, 16, 16)
    sim = MBOracle(grid, DX, DT, Params(npml=0))
    N_a = 2e24
    sim.set_material(np.ones(grid), np.ones(grid), N_a, 1e13)
    sim.set_field("N0", np.full(grid, 0.7 * N_a))
    sim.set_field("N2", np.full(grid, 0.3 * N_a))
    sim.set_seed(0x5EED)
    sim.step(1)
    a = 0.5 * GC["dw"] * DT
    sigma = GC["a_se"] * math.sqrt((0.3 * N_a + P0.n_floor_rel * N_a) / (DX ** 3 * DT))
    sd_expect = DT * sigma / (1 + a)
    J = np.concatenate([sim.field(c).ravel() for c in ("Jx", "Jy", "Jz")])
    var = np.mean(J * J)
    n = J.size
    assert abs(var / sd_expect ** 2 - 1) < 5 * math.sqrt(2.0 / n)
    assert abs(np.mean(J)) < 5 * sd_expect / math.sqrt(n)
    # no noise without atoms in N2 beyond the floor: scale check
    assert GC["a_se"] > 0


def test_rate_steady_state_closed_form():
    p = Params(tau32=100e-15, tau21=1e-9, tau10=100e-15)
    N_a, W_p = 2e24, 1e13
    A = rate_matrix(p, W_p)
    N0 = N_a / (1 + W_p * (p.tau32 + p.tau21 + p.tau10))
    Nstar = np.array([N0, W_p * p.tau10 * N0, W_p * p.tau21 * N0, W_p * p.tau32 * N0])
    assert abs(Nstar.sum() - N_a) < 1e-12 * N_a
    np.testing.assert_allclose(A @ Nstar, 0, atol=1e-12 * W_p * N_a)
    M, _ = crank_nicolson(A, DT)
    np.testing.assert_allclose(M @ Nstar, Nstar, rtol=1e-12)
    # the iterate converges to it from N = (N_a, 0, 0, 0) (dt large to converge fast)
    M_big, _ = crank_nicolson(A, 2e-12)
    N = np.array([N_a, 0, 0, 0.0])
    for _ in range(20000):
        N = M_big @ N
    np.testing.assert_allclose(N, Nstar, rtol=1e-9)


def test_rate_crank_nicolson_matches_matrix_exponential():
    p = Params()
    N_a, W_p = 2e24, 1e13
    A = rate_matrix(p, W_p)
    M, m = crank_nicolson(A, DT)
    N = np.array([N_a, 0, 0, 0.0])
    n = 20000
    for _ in range(n):
        N = population_update(N, 0.0, M, m)
    exact = scipy.linalg.expm(A * n * DT) @ np.array([N_a, 0, 0, 0.0])
    nA = np.linalg.norm(A, 2)
    bound = n * DT ** 3 * nA ** 3 * N_a / 12 * 2
    assert np.max(np.abs(N - exact)) < bound
    assert np.max(np.abs(N - exact)) > 0      # CN is not exact: the bound is meaningful
    assert abs(N.sum() - N_a) < 1e-12 * N_a


def test_field_transfer_direction():
    """With no decay and no pump, s > 0 moves atoms from N1 to N2 at rate s."""
    p = Params(tau32=1e300, tau21=1e300, tau10=1e300)
    A = rate_matrix(p, 0.0)
    M, m = crank_nicolson(A, DT)
    N = np.array([0.0, 1e24, 0.0, 0.0])
    s = 3e33
    for _ in range(10):
        N = population_update(N, s, M, m)
    np.testing.assert_allclose(N[2], 10 * DT * s, rtol=1e-12)
    np.testing.assert_allclose(N[1], 1e24 - 10 * DT * s, rtol=1e-12)


def test_field_and_atoms_exchange_energy_exactly():
    """With decays and pump off (A ~ 0: M = I, m = dt e), the discrete Yee
    energy theorem with a current, W^{n+1} - W^n = -dt dV sum J^{n+1/2} .
    (E^n + E^{n+1})/2 for W^n = 1/2 sum eps|E^n|^2 dV + 1/2 sum mu0
    H^{n-1/2}.H^{n+1/2} dV in a PEC box, and the population update
    N2^{n+1} = N2^n + dt s make W^n + hbar w0 dV sum N2^n an invariant of the
    coupled step.  Started from zero fields and zero N2, driven by the
    Langevin currents alone, it stays zero to rounding while the field's
    energy grows from nothing."""
    grid = (10, 9, 11)
    rng = np.random.default_rng(21)
    p = Params(npml=0, tau32=1e300, tau21=1e300, tau10=1e300)
    sim = MBOracle(grid, DX, DT, p)
    gain = rng.random(grid[::-1]) < 0.5
    eps = rng.uniform(1.0, 8.41, size=grid[::-1])
    N_a = 2e25
    sim.set_material(eps, gain, N_a, 0.0)
    sim.set_seed(77)
    dV = DX ** 3
    hw = HBAR * gain_constants(p)["w0"]
    inv, W_all = [], []
    for _ in range(40):
        E_n = [F.copy() for F in sim.E]
        H_minus = [F.copy() for F in sim.H]
        atoms = hw * dV * sim.N[2].sum()
        sim.step(1)
        W = 0.5 * EPS0 * sum(np.sum(eps * F * F) for F in E_n) * dV
        W += 0.5 * MU0 * sum(np.sum(a * b) for a, b in zip(H_minus, sim.H)) * dV
        inv.append(W + atoms)
        W_all.append(W)
    scale = max(abs(w) for w in W_all)
    assert scale > 0 and W_all[-1] > 0          # the currents did put energy into the field
    assert max(abs(v) for v in inv) <= 1e-11 * scale


def _run_cavity(init_pop, steps=120):
    grid = (10, 10, 10)
    sim = MBOracle(grid, DX, DT, Params(npml=0, a_se=0.0))
    N_a = 1e26
    sim.set_material(np.ones(grid), np.ones(grid), N_a, 0.0)
    sim.N[:] = 0.0
    sim.N[init_pop] = N_a
    rng = np.random.default_rng(2)
    kk, jj, ii = np.meshgrid(*(np.arange(10),) * 3, indexing="ij")
    sim.set_field("Ez", 1e6 * np.sin(np.pi * ii / 10) * np.sin(np.pi * jj / 10))
    U0 = sim.energy()
    sim.step(steps)
    return sim, U0


def test_inverted_medium_amplifies_and_absorber_absorbs():
    gain_sim, U0 = _run_cavity(2)       # all atoms in the upper lasing level N2
    absorb_sim, _ = _run_cavity(1)      # all atoms in the lower lasing level N1
    assert gain_sim.energy() > 1.5 * U0
    assert absorb_sim.energy() < 0.9 * U0
    # energy bookkeeping direction: the absorber lifts atoms to N2
    assert absorb_sim.N[2].sum() > 0
    assert gain_sim.N[1].sum() > 0


def test_populations_conserved_in_noisy_run():
    grid = (12, 11, 10)
    sim = MBOracle(grid, DX, DT, Params(npml=3))
    rng = np.random.default_rng(9)
    gain = rng.random(grid[::-1]) < 0.6
    eps = np.where(gain, 1.0, 8.41)
    N_a = 5e24
    sim.set_material(eps, gain, N_a, 1e13)
    sim.set_seed(1234)
    sim.step(40)
    tot = sim.N.sum(axis=0)
    np.testing.assert_allclose(tot[gain], N_a, rtol=1e-13)
    assert np.all(tot[~gain] == 0)
    assert np.abs(sim.field("Jx")).max() > 0
    assert np.all(sim.field("Jx")[~gain] == 0)

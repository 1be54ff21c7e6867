"""FP64 oracle of the theory side: the bound state of the dimensionless
equation for the random-laser spectral envelope (the paper's Eq. g5)

    -phi'' + tau^2 phi + phi^3 = E phi,      phi > 0, phi -> 0 as |tau| -> inf,

and the spectral features that the paper reads off its Fourier transform
(the waist w_phi(E) and the peak p_phi(E), "Gross-Pitaevskii equation"
paragraph, Figs. 3 and 5).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``; never by the product
package, with which it shares no code.

Discretisation: tau_i = -L + i h, i = 1 .. n (h = 2L/(n+1)), phi(+-L) = 0,
second-order differences.  The discrete equation F(phi) = 0 is solved by
Newton's method (a tridiagonal system per iteration, Thomas algorithm)
started at the larger of the first-order solution near threshold,
2^{1/4} sqrt(E-1) exp(-tau^2/2) (the paper's approximation), and the
Thomas-Fermi profile sqrt(max(E - tau^2, 0)) of large E; phi = 0 also solves
the equation, so a solution that collapses to it is rejected.
Features of the converged phi (trapezoid sums on the grid):

    phi~(Omega) = int phi(tau) exp(i Omega tau) dtau        (phi even: cosine transform)
    p_phi = |phi~(0)|^2 / (4 pi^2) = (int phi)^2 / (4 pi^2)
    w_phi = sigma_Omega / (2 pi),  sigma_Omega^2 = int Omega^2 |phi~|^2 / int |phi~|^2
          = int phi'^2 / int phi^2                          (Parseval)

so that S(omega) = t_g^2 |phi~(omega t0)|^2 / (4 pi^2 gamma_S) has its peak
t_g^2 p_phi / gamma_S and the standard deviation W = w_phi / t0 in the
frequency omega / 2 pi (at threshold w_phi = 1 / (2 sqrt 2 pi)).  With
E(p) = (p - 1)/(kappa sqrt p) and t0 = t_g p^{1/4} / sqrt(kappa) (t0^2 =
t_g t_L sqrt(g0) / sqrt(alpha0 - alpha_L) in the paper's definitions),
W = w_phi sqrt(kappa) / (p^{1/4} t_g).

Pins (tests/test_oracle_gp.py): the near-threshold closed form; the discrete
identity sum(phi (-D2 phi) + tau^2 phi^2 + phi^4) = E sum(phi^2) (exact for
the discrete solution); the continuum virial identity int phi'^2 - 3 int
tau^2 phi^2 - int phi^4 / 2 + E int phi^2 = 0 (to discretisation error); the
threshold E(p_th) = 1 with p_th = 1 + kappa^2/2 + kappa sqrt(4 + kappa^2)/2.
"""
from __future__ import annotations

import math

import numpy as np


def grid(n: int, L: float):
    h = 2.0 * L / (n + 1)
    return -L + h * np.arange(1, n + 1), h


def residual(phi, tau, h, E):
    d2 = np.empty_like(phi)
    d2[1:-1] = phi[2:] - 2 * phi[1:-1] + phi[:-2]
    d2[0] = phi[1] - 2 * phi[0]
    d2[-1] = phi[-2] - 2 * phi[-1]
    return -d2 / h ** 2 + tau ** 2 * phi + phi ** 3 - E * phi


def thomas(a, b, c, d):
    """Solve the tridiagonal system with sub-diagonal a, diagonal b,
    super-diagonal c (a[0], c[-1] unused)."""
    n = len(b)
    cp = np.empty(n)
    dp = np.empty(n)
    cp[0] = c[0] / b[0]
    dp[0] = d[0] / b[0]
    for i in range(1, n):
        m = b[i] - a[i] * cp[i - 1]
        cp[i] = c[i] / m if i < n - 1 else 0.0
        dp[i] = (d[i] - a[i] * dp[i - 1]) / m
    x = np.empty(n)
    x[-1] = dp[-1]
    for i in range(n - 2, -1, -1):
        x[i] = dp[i] - cp[i] * x[i + 1]
    return x


def newton(phi, tau, h, E, tol=1e-12, max_iter=60):
    """Newton steps until the residual is below tol max(1, E) or the step
    stagnates at rounding level (|delta| <= 1e-14 max(1, max phi)); accepted
    if the final residual is below 1e-9 max(1, E)."""
    off = np.full(len(phi), -1.0 / h ** 2)
    for _ in range(max_iter):
        F = residual(phi, tau, h, E)
        if np.max(np.abs(F)) < tol * max(1.0, E):
            return phi, True
        diag = 2.0 / h ** 2 + tau ** 2 + 3.0 * phi ** 2 - E
        delta = thomas(off, diag, off, F)
        phi = phi - delta
        if np.max(np.abs(delta)) <= 1e-14 * max(1.0, phi.max()):
            break
    return phi, np.max(np.abs(residual(phi, tau, h, E))) < 1e-9 * max(1.0, E)


def near_threshold(tau, E):
    return 2.0 ** 0.25 * math.sqrt(max(E - 1.0, 0.0)) * np.exp(-tau ** 2 / 2)


def initial_guess(tau, E):
    return np.maximum(np.sqrt(np.maximum(E - tau ** 2, 0.0)), near_threshold(tau, E))


def solve(E: float, n: int = 2047, L: float | None = None):
    """phi on the grid for eigenvalue E > 1."""
    if E <= 1.0:
        raise ValueError("bound states exist for E > 1")
    L = (math.sqrt(E) + 8.0) if L is None else L
    tau, h = grid(n, L)
    phi, ok = newton(initial_guess(tau, E), tau, h, E, max_iter=100)
    if not ok or phi.max() < 0.5 * near_threshold(np.zeros(1), E)[0]:
        raise RuntimeError(f"no bound state found at E = {E}")
    return tau, h, phi


def features(tau, h, phi):
    """(w_phi, p_phi) of a solution (trapezoid sums; phi(+-L) = 0)."""
    s_phi = h * phi.sum()
    p_phi = s_phi ** 2 / (4.0 * math.pi ** 2)
    dphi = np.diff(np.concatenate(([0.0], phi, [0.0]))) / h
    sig2 = (h * np.sum(dphi ** 2)) / (h * np.sum(phi ** 2))
    return math.sqrt(sig2) / (2.0 * math.pi), p_phi


def E_of_p(p, kappa):
    return (p - 1.0) / (kappa * np.sqrt(p))


def p_threshold(kappa):
    return 1.0 + kappa ** 2 / 2.0 + kappa * math.sqrt(4.0 + kappa ** 2) / 2.0

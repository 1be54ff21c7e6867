"""FP64 oracle of the theory side: the bound state of the dimensionless
equation for the random-laser spectral envelope (the paper's Eq. g5,
"Gross-Pitaevskii equation" paragraph)

    -phi'' + tau^2 phi + phi^3 = E phi,      phi > 0, phi -> 0 as |tau| -> inf,

solved as the continuum ordinary differential equation (no grid: shooting,
or a collocation boundary-value solve at large E), and the spectral
features the paper reads off its Fourier transform (the waist w_phi(E) and
the peak p_phi(E), Figs. 3 and 5).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``; never by the product
package, with which it shares no code and no algorithm (the product solves
the equation discretised on a grid by Newton's method; this module never
discretises it).

Method.  The bound state is even with its maximum at tau = 0, so it solves

    phi'' = (tau^2 + phi^2 - E) phi,   phi'(0) = 0,   phi -> 0,   tau >= 0,

and the features need the integrals

    I0 = int phi,  I1 = int phi^2,  I2 = int phi'^2,  I3 = int tau^2 phi^2,
    I4 = int phi^4,   over [0, tau], doubled for the whole line,

which are carried as five extra components of the integrated system (so
they are as accurate as phi itself).  Two continuum methods, chosen by E:

  * SHOOTING (1 < E <= 4).  From phi(0) = a, phi'(0) = 0 the system is
    integrated outward by an adaptive eighth-order Runge-Kutta method
    (scipy's DOP853, a library step) until phi reaches 0 (a node: a is too
    small) or phi' returns to 0 with phi > 0 (phi turns up and grows without
    bound: a is too large).  The bracket [0, sqrt E] (at a = sqrt E already
    phi''(0) = 0) is bisected to rounding level.  The two final shots agree
    up to the point tau_c where the growing solution separates them; beyond
    it the tail is the equation's linear asymptotics
    phi ~ C tau^((E-1)/2) exp(-tau^2/2), matched at tau_c.  This is exact
    to rounding where the initial-value problem is well conditioned: in the
    Thomas-Fermi bulk (phi^2 ~ E - tau^2) a perturbation grows like
    exp(sqrt(2 (E - tau^2)) tau), about exp(1.1 E) across it, which FP64
    resolves only for small E.

  * BOUNDARY-VALUE SOLVE (E > 4).  The same system on [0, T], T = sqrt(E) + 8,
    with phi'(0) = 0, I_k(0) = 0 and, at T, the Robin condition of the
    decaying asymptotics phi'/phi = (E-1)/(2T) - T, solved by scipy's
    fourth-order collocation solver with an adaptive mesh (solve_bvp, a
    library step) from a smoothed Thomas-Fermi profile; the tail beyond T
    (~exp(-T^2/2)) is added from the same asymptotics.

Both methods solve the continuum equation; neither uses a fixed grid.

    phi~(Omega) = int phi(tau) exp(i Omega tau) dtau
    p_phi = |phi~(0)|^2 / (4 pi^2) = (int phi)^2 / (4 pi^2)
    w_phi = sigma_Omega / (2 pi),  sigma_Omega^2 = int Omega^2 |phi~|^2 / int |phi~|^2
          = int phi'^2 / int phi^2                                    (Parseval)

so that S(omega) = t_g^2 |phi~(omega t0)|^2 / (4 pi^2 gamma_S) has its peak
t_g^2 p_phi / gamma_S and the standard deviation W = w_phi / t0 in the
frequency omega / 2 pi (at threshold w_phi = 1 / (2 sqrt 2 pi)).  With
E(p) = (p - 1)/(kappa sqrt p) (Eq. ee) and t0 = t_g p^{1/4} / sqrt(kappa),
W = w_phi sqrt(kappa) / (p^{1/4} t_g).  Bound states exist for E > 1 (the
linear oscillator's ground state), which E(p) = 1 turns into the threshold
p_th = 1 + kappa^2/2 + kappa sqrt(4 + kappa^2)/2.

Pins (tests/test_oracle_gp.py): the paper's first-order solution near
threshold, 2^{1/4} sqrt(E - 1) exp(-tau^2/2); the two integral identities
every solution satisfies (the equation times phi, integrated; the scaling
virial); the Thomas-Fermi limit of large E; the two methods against each
other where both are accurate; the threshold E(p_th) = 1.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.integrate import quad, solve_bvp, solve_ivp

# above this E the bisection of the initial-value problem loses its digits
# (see the module docstring) and the boundary-value solve takes over
E_SHOOT_MAX = 4.0

_RTOL = 1e-13
# absolute floor relative to phi(0): far below where the growing solution
# separates the bracketing shots
_ATOL_REL = 1e-24


def _rhs(E):
    """The system (phi, phi', I0..I4)' at tau; works on scalars (one point)
    and on rows of arrays (a mesh)."""
    def f(tau, y):
        phi, dphi = y[0], y[1]
        return np.array([dphi, (tau * tau + phi * phi - E) * phi,
                         phi, phi * phi, dphi * dphi, tau * tau * phi * phi, phi ** 4])
    return f


def _node(tau, y):
    return y[0]


_node.terminal = True
_node.direction = -1


def _turn(tau, y):
    return y[1]


_turn.terminal = True
_turn.direction = 1


def _shoot(E, a, tau_max, dense=False):
    """Integrate from tau = 0 with phi = a, phi' = 0.  Returns
    (kind, solution): kind -1 = node (a too small), +1 = turns up (a too
    large), 0 = neither before tau_max."""
    if a * a >= E:
        return 1, None
    sol = solve_ivp(_rhs(E), (0.0, tau_max), [a, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0],
                    method="DOP853", rtol=_RTOL, atol=_ATOL_REL * max(a, 1e-300),
                    events=(_node, _turn), dense_output=dense)
    if sol.t_events[0].size:
        return -1, sol
    if sol.t_events[1].size:
        return 1, sol
    return 0, sol


class BoundState:
    """The even bound state of Eq. g5 at eigenvalue E as a function of tau
    (``st(tau)``), with phi(0) (``a``) and the whole-line integrals I0..I4."""

    def __init__(self, E, method, inner, tau_c, amp_c, a):
        self.E = E
        self.method = method
        self._inner = inner          # phi on [0, tau_c]
        self.tau_c = tau_c
        self._amp_c = amp_c
        self.a = a
        self.I0 = self.I1 = self.I2 = self.I3 = self.I4 = 0.0

    def tail(self, t):
        """Linear asymptotics beyond tau_c, matched to phi(tau_c)."""
        q = 0.5 * (self.E - 1.0)
        return self._amp_c * (t / self.tau_c) ** q * np.exp(-0.5 * (t * t - self.tau_c ** 2))

    def __call__(self, tau):
        t = np.abs(np.asarray(tau, dtype=np.float64))
        out = np.empty_like(t)
        inner = t <= self.tau_c
        if np.any(inner):
            out[inner] = self._inner(t[inner])
        if np.any(~inner):
            out[~inner] = self.tail(t[~inner])
        return out

    def _close(self, half_at_tau_c):
        """Whole-line integrals: the carried ones on [0, tau_c] plus the
        asymptotic tail, doubled."""
        q = 0.5 * (self.E - 1.0)
        g = self.tail

        def dg(t):
            return g(t) * (q / t - t)

        a, b = self.tau_c, self.tau_c + 40.0
        kw = dict(epsabs=0, epsrel=1e-10, limit=200)
        tails = [quad(g, a, b, **kw)[0],
                 quad(lambda t: g(t) ** 2, a, b, **kw)[0],
                 quad(lambda t: dg(t) ** 2, a, b, **kw)[0],
                 quad(lambda t: t * t * g(t) ** 2, a, b, **kw)[0],
                 quad(lambda t: g(t) ** 4, a, b, **kw)[0]]
        self.I0, self.I1, self.I2, self.I3, self.I4 = (
            2.0 * (np.asarray(half_at_tau_c, dtype=np.float64) + np.asarray(tails))).tolist()
        return self


def solve_shooting(E: float) -> BoundState:
    """Shooting on phi(0) with bisection (accurate for 1 < E <~ 5)."""
    tau_max = math.sqrt(E) + 14.0
    lo, hi = 0.0, math.sqrt(E)
    while True:
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        kind, _ = _shoot(E, mid, tau_max)
        if kind < 0:
            lo = mid
        elif kind > 0:
            hi = mid
        else:
            lo = hi = mid          # decayed below rounding undecided: resolved
            break
    if hi == lo:
        hi = math.nextafter(lo, math.inf)
    k_lo, s_lo = _shoot(E, lo, tau_max, dense=True)
    k_hi, s_hi = _shoot(E, hi, tau_max, dense=True)
    if s_lo is None or s_hi is None or k_lo > 0 or k_hi < 0:
        raise RuntimeError(f"shooting did not bracket the bound state at E = {E}")
    # stop where the two shots differ by 1e-6 of their mean
    t_end = min(s_lo.t[-1], s_hi.t[-1])
    ts = np.linspace(0.0, t_end, 20001)
    p_lo = s_lo.sol(ts)[0]
    p_hi = s_hi.sol(ts)[0]
    sep = np.abs(p_hi - p_lo) > 1e-6 * np.abs(0.5 * (p_hi + p_lo))
    ic = int(np.argmax(sep)) if np.any(sep) else len(ts) - 1
    tau_c = float(ts[max(ic - 1, 1)])
    y = 0.5 * (s_lo.sol(tau_c) + s_hi.sol(tau_c))
    if y[0] <= 0.0:
        raise RuntimeError(f"no decaying solution found at E = {E}")

    def inner(t):
        return 0.5 * (s_lo.sol(t)[0] + s_hi.sol(t)[0])

    st = BoundState(E, "shooting", inner, tau_c, float(y[0]), 0.5 * (lo + hi))
    return st._close(y[2:7])


def solve_bvp_continuum(E: float, tol: float | None = None) -> BoundState:
    """Collocation solve on [0, sqrt(E) + 8] with the asymptotic Robin
    condition at the far end (accurate for every E > 1 not close to 1)."""
    if tol is None:
        # relative residual bound of the collocation: the solution's error is
        # far smaller (~1e-11 in the features); above E ~ 200 the residual's
        # rounding floor makes 1e-7 unreachable
        tol = 1e-7 if E <= 200.0 else 1e-6
    T = math.sqrt(E) + 8.0
    q = 0.5 * (E - 1.0)
    tau = np.linspace(0.0, T, 801)
    # smoothed Thomas-Fermi start: sqrt(E - tau^2) inside, a Gaussian tail outside
    g = np.sqrt(0.5 * (E - tau ** 2 + np.sqrt((E - tau ** 2) ** 2 + 4.0)))
    g = g * np.exp(-0.5 * np.maximum(tau - math.sqrt(E), 0.0) ** 2)
    y0 = np.zeros((7, tau.size))
    y0[0] = g
    y0[1] = np.gradient(g, tau)

    def bc(ya, yb):
        return np.array([ya[1], ya[2], ya[3], ya[4], ya[5], ya[6], yb[1] - (q / T - T) * yb[0]])

    sol = None
    for t in (tol, 10 * tol, 100 * tol):
        sol = solve_bvp(_rhs(E), bc, tau, y0, tol=t, bc_tol=1e-12, max_nodes=100000)
        if sol.status == 0:
            break
    if sol is None or sol.status != 0 or sol.y[0, 0] <= 0.0:
        raise RuntimeError(f"boundary-value solve failed at E = {E}")
    yT = sol.sol(T)
    st = BoundState(E, "bvp", lambda t: sol.sol(t)[0], T, float(yT[0]), float(sol.sol(0.0)[0]))
    return st._close(yT[2:7])


def solve(E: float) -> BoundState:
    """The bound state for eigenvalue E > 1."""
    if not (E > 1.0) or not math.isfinite(E):
        raise ValueError("bound states exist for finite E > 1")
    return solve_shooting(E) if E <= E_SHOOT_MAX else solve_bvp_continuum(E)


def features(st: BoundState):
    """(w_phi, p_phi) of a bound state."""
    p_phi = st.I0 ** 2 / (4.0 * math.pi ** 2)
    sig2 = st.I2 / st.I1
    return math.sqrt(sig2) / (2.0 * math.pi), p_phi


def near_threshold(tau, E):
    """The paper's first-order solution near threshold (E -> 1+)."""
    return 2.0 ** 0.25 * math.sqrt(max(E - 1.0, 0.0)) * np.exp(-np.asarray(tau) ** 2 / 2)


def E_of_p(p, kappa):
    return (p - 1.0) / (kappa * np.sqrt(p))


def p_threshold(kappa):
    return 1.0 + kappa ** 2 / 2.0 + kappa * math.sqrt(4.0 + kappa ** 2) / 2.0

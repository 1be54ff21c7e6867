"""Plain FP64 CPU oracle of the vectorial Maxwell–Bloch FDTD step.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU legs of ``bench.py``; never by the product package, with which it
shares no code.

What it computes.  The paper ("Simulations" paragraph) solves a vectorial
Maxwell–Bloch (MB) system by finite differences in time domain: TiO2 spheres
(n = 2.9) in a gain medium that fills the voids, four-level atoms with
lambda0 = 590 nm and a 230 nm gain bandwidth (~1/t_g), a pump that is constant
in time and present only in the voids, and spontaneous emission entered as a
stochastic term.  The paper prints none of the equations; this module writes
out the standard four-level, Lorentz-oscillator MB-FDTD scheme that these
words describe (Nagra & York 1998; Chang & Taflove 2004):

    mu0 dH/dt        = -curl E
    eps0 eps_r dE/dt =  curl H - J                      (J = dP/dt)
    dJ/dt + dw_a J + w0^2 P = xi (N1 - N2) E + F        (gain cells only)
    dN/dt = A N + e (E . J) / (hbar w0),   e = (0, -1, +1, 0)

with xi = 6 pi eps0 c^3 / (w0^2 tau21), dw_a = 2 pi c dlambda / lambda0^2,
A the four-level rate matrix with pump W_p out of N0, and F a Langevin force
with variance proportional to (N2 + N_floor).

One step n -> n+1, in this order (every array is FP64, indexed [k, j, i]):
  1. H^{n+1/2} = H^{n-1/2} - dt/mu0 (curl_fwd E^n + CPML psi_H)
  2. J^{n+1/2} = [(1 - a) J^{n-1/2} + dt (xi dN^n E^n - w0^2 P^n + sigma_F zeta^n)] / (1 + a),
     a = dw_a dt / 2
  3. P^{n+1}   = P^n + dt J^{n+1/2}
  4. E^{n+1}   = E^n + dt/(eps0 eps_r) (curl_bwd H^{n+1/2} + CPML psi_E - J^{n+1/2} - J_src)
  5. N^{n+1}   = M N^n + m s,  s = (1/hbar w0) 1/2 (E^n + E^{n+1}) . J^{n+1/2}
     with M = (I - dt A/2)^-1 (I + dt A/2), m = dt (I - dt A/2)^-1 e (Crank–Nicolson)
  6. probes: running DFT of E^{n+1} at t_{n+1} (points, face sub-grids and
     whole z-planes); outward Poynting flux of the interior box, with
     (E^n + E^{n+1})/2 on each face plane and H^{n+1/2} on the adjacent
     half-plane (the pairing of the Yee curls across the plane).
Read-outs also include the energy density of a z-plane (a snapshot of the
sample's middle section, Fig. 2a) and the mode map of a plane probe (the
field of a mode under CW excitation, inset of Fig. 1).

Yee ownership: cell (i,j,k) owns Ex(i+1/2,j,k), Ey(i,j+1/2,k), Ez(i,j,k+1/2),
Hx(i,j+1/2,k+1/2), Hy(i+1/2,j,k+1/2), Hz(i+1/2,j+1/2,k); P and J sit on the E
sites; N0..N3 are per cell.  Boundaries: PEC walls at x = 0 and x = n_x dx (and
likewise in y, z): tangential E on the planes i = 0 (j = 0, k = 0) is held at
zero, fields beyond the last cell are zero.  CPML (Roden & Gedney 2000, kappa =
1, cubic sigma grading, linear alpha grading) in npml cells on each face.

Noise: one Philox4x32-10 draw (Salmon et al., SC'11) per gain cell and step,
key = (seed low word, seed high word), counter = (cell index, step, 0, 0);
u = ((x >> 9) + 1/2) 2^-23, then Box–Muller gives three normals.

Pins (tests/test_oracle_*.py): Philox known-answer vectors; Box–Muller
moments; exact discrete PEC-cavity eigenmodes (discrete dispersion relation);
the discrete Yee energy invariant; population conservation and the steady
state / matrix-exponential limits of the rate equations; the closed-form
transfer function of the Lorentz recursion; the stationary variance of the
noise-driven recursion; CPML reflection against a larger box; the running DFT
against its geometric-sum closed form; the face flux against the exact
discrete energy balance of the interior box; the plane snapshot against the
total energy, the plane DFT against point probes, the CW waveform's closed
form, a CW-driven box's mode map at the drive frequency and its quadratic
scaling (tests/test_oracle_modemap.py).
Parity unpinned: the composition of all of these in a long noisy run has no
closed form; it is pinned only through its parts.
"""
from __future__ import annotations

from dataclasses import dataclass, asdict
import math

import numpy as np

# SI constants (CODATA 2018).
C0 = 299_792_458.0
EPS0 = 8.8541878128e-12
MU0 = 1.0 / (EPS0 * C0 * C0)
ETA0 = MU0 * C0
HBAR = 1.054571817e-34
Q_E = 1.602176634e-19

# numpy axis of each Cartesian direction: arrays are indexed [k, j, i].
AX_X, AX_Y, AX_Z = 2, 1, 0


@dataclass
class Params:
    """Physical and numerical parameters of the step (SI units)."""
    lambda0: float = 590e-9       # gain centre wavelength (paper)
    dlambda: float = 230e-9       # gain bandwidth (paper), ~ 1/t_g
    tau32: float = 100e-15        # lifetimes: not given by the paper
    tau21: float = 1e-9
    tau10: float = 100e-15
    a_se: float = -1.0            # Langevin amplitude; < 0 selects the default below
    dipole_len: float = 0.1e-9    # dipole length d0/e of the default noise amplitude
    n_floor_rel: float = 1e-9     # N_floor / N_a inside the noise square root
    npml: int = 8                 # CPML cells per face
    pml_order: float = 3.0        # sigma grading exponent
    pml_sigma_factor: float = 0.8 # sigma_max = factor (order + 1) / (eta0 dx)
    pml_alpha_rel: float = 0.1    # alpha_max = 2 pi eps0 (alpha_rel c / lambda0)

    def as_dict(self):
        return asdict(self)


def gain_constants(p: Params):
    """Derived gain-medium constants: w0, dw_a, xi and the noise amplitude."""
    w0 = 2.0 * math.pi * C0 / p.lambda0
    dw = 2.0 * math.pi * C0 * p.dlambda / p.lambda0 ** 2
    xi = 6.0 * math.pi * EPS0 * C0 ** 3 / (w0 ** 2 * p.tau21)
    if p.a_se < 0:
        # Random dipoles of strength d0 = e * dipole_len driving the damped
        # oscillator: white force intensity 2 dw w0^2 d0^2 per unit density.
        a_se = w0 * (Q_E * p.dipole_len) * math.sqrt(2.0 * dw)
    else:
        a_se = p.a_se
    return {"w0": w0, "dw": dw, "xi": xi, "a_se": a_se}


# ---------------------------------------------------------------- rate equations

def rate_matrix(p: Params, W_p: float) -> np.ndarray:
    """A with dN/dt = A N for the four-level system N = (N0, N1, N2, N3).

    Pump N0 -> N3 at rate W_p, fast decay N3 -> N2 (tau32), lasing transition
    N2 -> N1 (tau21), fast decay N1 -> N0 (tau10).  Every column sums to zero.
    """
    A = np.zeros((4, 4))
    A[0, 0] = -W_p
    A[0, 1] = 1.0 / p.tau10
    A[1, 1] = -1.0 / p.tau10
    A[1, 2] = 1.0 / p.tau21
    A[2, 2] = -1.0 / p.tau21
    A[2, 3] = 1.0 / p.tau32
    A[3, 3] = -1.0 / p.tau32
    A[3, 0] = W_p
    return A


E_COUPLING = np.array([0.0, -1.0, 1.0, 0.0])   # field-driven transfer N1 -> N2


def crank_nicolson(A: np.ndarray, dt: float):
    """M = (I - dt A/2)^-1 (I + dt A/2) and m = dt (I - dt A/2)^-1 e."""
    I = np.eye(4)
    L = I - 0.5 * dt * A
    M = np.linalg.solve(L, I + 0.5 * dt * A)
    m = dt * np.linalg.solve(L, E_COUPLING)
    return M, m


# ------------------------------------------------------------------------ Philox

PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11).

    Each round multiplies words 0 and 2 by the two Philox constants and mixes
    the high halves with words 1, 3 and the key; the key is bumped by the two
    Weyl constants between rounds.  Inputs broadcast; outputs are uint32.
    """
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & _MASK32 for v in (c0, c1, c2, c3))
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    for r in range(10):
        if r > 0:
            k0 = np.uint64((int(k0) + PHILOX_W0) & 0xFFFFFFFF)
            k1 = np.uint64((int(k1) + PHILOX_W1) & 0xFFFFFFFF)
        p0 = np.uint64(PHILOX_M0) * c0      # exact: both factors < 2^32
        p1 = np.uint64(PHILOX_M1) * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return tuple(v.astype(np.uint32) for v in (c0, c1, c2, c3))


def u32_to_unit(x) -> np.ndarray:
    """u = ((x >> 9) + 1/2) * 2^-23, strictly inside (0, 1) and exact in FP32."""
    return ((np.asarray(x, dtype=np.uint32) >> np.uint32(9)).astype(np.float64) + 0.5) * 2.0 ** -23


def langevin_normals(seed: int, cell, step: int):
    """Three standard normals per cell for step ``step`` (Box–Muller, FP64)."""
    cell = np.asarray(cell, dtype=np.uint64)
    x0, x1, x2, x3 = philox4x32_10(cell, np.uint64(step), 0, 0,
                                   seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    u0, u1, u2, u3 = (u32_to_unit(v) for v in (x0, x1, x2, x3))
    r01 = np.sqrt(-2.0 * np.log(u0))
    r23 = np.sqrt(-2.0 * np.log(u2))
    return (r01 * np.cos(2.0 * np.pi * u1),
            r01 * np.sin(2.0 * np.pi * u1),
            r23 * np.cos(2.0 * np.pi * u3))


# -------------------------------------------------------------------------- CPML

def cpml_profile(n: int, half: float, dx: float, dt: float, p: Params):
    """CPML update coefficients (b, c) at positions x = i + half, i = 0..n-1.

    Roden & Gedney (2000) with kappa = 1: psi <- b psi + c dF/dw,
    b = exp(-(sigma + alpha) dt/eps0), c = sigma/(sigma + alpha) (b - 1).
    The depth into the layer is measured from the inner interface (x = npml
    or x = n - npml, in cells) towards the PEC wall; sigma grows as depth^m,
    alpha falls linearly to zero at the wall.  Outside the layers b = c = 0.
    """
    b = np.zeros(n)
    c = np.zeros(n)
    L = p.npml
    if L <= 0:
        return b, c
    x = np.arange(n, dtype=np.float64) + half
    depth = np.maximum((L - x) / L, (x - (n - L)) / L)
    depth = np.clip(depth, 0.0, 1.0)
    sigma_max = p.pml_sigma_factor * (p.pml_order + 1.0) / (ETA0 * dx)
    alpha_max = 2.0 * math.pi * EPS0 * p.pml_alpha_rel * C0 / p.lambda0
    inside = depth > 0.0
    sigma = sigma_max * depth ** p.pml_order
    alpha = alpha_max * (1.0 - depth)
    bb = np.exp(-(sigma + alpha) * dt / EPS0)
    b[inside] = bb[inside]
    c[inside] = (sigma / (sigma + alpha) * (bb - 1.0))[inside]
    return b, c


# ------------------------------------------------------------- finite differences

def d_fwd(F: np.ndarray, axis: int) -> np.ndarray:
    """F[i+1] - F[i] along ``axis``; the value beyond the last cell is zero."""
    D = -F.copy()
    lo = [slice(None)] * 3
    hi = [slice(None)] * 3
    lo[axis] = slice(0, -1)
    hi[axis] = slice(1, None)
    D[tuple(lo)] += F[tuple(hi)]
    return D


def d_bwd(F: np.ndarray, axis: int) -> np.ndarray:
    """F[i] - F[i-1] along ``axis``; the value before the first cell is zero."""
    D = F.copy()
    lo = [slice(None)] * 3
    hi = [slice(None)] * 3
    lo[axis] = slice(0, -1)
    hi[axis] = slice(1, None)
    D[tuple(hi)] -= F[tuple(lo)]
    return D


# --------------------------------------------------------------- gain sub-steps

def lorentz_update(J, P, E, dN, force, dt, w0, dw, xi):
    """Steps 2-3 for one component: returns (J^{n+1/2}, P^{n+1})."""
    a = 0.5 * dw * dt
    J_new = ((1.0 - a) * J + dt * (xi * dN * E - w0 * w0 * P + force)) / (1.0 + a)
    P_new = P + dt * J_new
    return J_new, P_new


def population_update(N, s, M, m):
    """Step 5: N^{n+1} = M N^n + m s for N of shape (4, ...)."""
    return np.tensordot(M, N, axes=(1, 0)) + m.reshape((4,) + (1,) * (N.ndim - 1)) * s


def source_waveform(t, lam, t0, tau, amp):
    """Single-cycle soft current: amp sin(w_s (t - t0)) exp(-((t - t0)/tau)^2)."""
    ws = 2.0 * math.pi * C0 / lam
    return amp * math.sin(ws * (t - t0)) * math.exp(-((t - t0) / tau) ** 2)


def source_waveform_cw(t, lam, t0, tau, amp):
    """Continuous-wave soft current switched on at t0 with a smooth rise:
    amp sin(w_s (t - t0)) (1 - exp(-((t - t0)/tau)^2)) for t >= t0, else 0."""
    if t < t0:
        return 0.0
    ws = 2.0 * math.pi * C0 / lam
    return amp * math.sin(ws * (t - t0)) * (1.0 - math.exp(-((t - t0) / tau) ** 2))


def lambda_grid(n_freq: int, lam_min: float, lam_max: float) -> np.ndarray:
    """Probe wavelengths: n_freq points uniformly spaced from lam_min to lam_max."""
    if n_freq == 1:
        return np.array([lam_min])
    return lam_min + (lam_max - lam_min) * np.arange(n_freq) / (n_freq - 1)


def dft_accumulate(acc, sample, omegas, t, weight):
    """acc_k += sample * exp(i w_k t) * weight (running DFT, FP64)."""
    return acc + sample * np.exp(1j * omegas * t) * weight


# ------------------------------------------------------------------ the step

class MBOracle:
    """One realization on an n_x x n_y x n_z Yee grid, advanced in FP64."""

    def __init__(self, grid, dx: float, dt: float, params: Params | None = None):
        nx, ny, nz = (int(v) for v in grid)
        if min(nx, ny, nz) < 1:
            raise ValueError("grid sizes must be >= 1")
        if dt <= 0 or dx <= 0 or dt > dx / (C0 * math.sqrt(3.0)):
            raise ValueError("dt must satisfy the 3D Courant limit dt <= dx/(c sqrt 3)")
        self.nx, self.ny, self.nz = nx, ny, nz
        self.shape = (nz, ny, nx)
        self.dx, self.dt = float(dx), float(dt)
        self.p = params if params is not None else Params()
        self.gc = gain_constants(self.p)
        z = lambda: np.zeros(self.shape)
        self.E = [z(), z(), z()]
        self.H = [z(), z(), z()]
        self.P = [z(), z(), z()]
        self.J = [z(), z(), z()]
        self.N = np.zeros((4,) + self.shape)
        # psi_H[(c, w)]: H component c, derivative along w (E-field differences)
        self.psi_H = {key: z() for key in (("x", "y"), ("x", "z"), ("y", "z"),
                                            ("y", "x"), ("z", "x"), ("z", "y"))}
        self.psi_E = {key: z() for key in self.psi_H}
        prof = lambda n, half, ax: tuple(
            v.reshape([n if a == ax else 1 for a in range(3)])
            for v in cpml_profile(n, half, self.dx, self.dt, self.p))
        # E-type derivative sites sit at integer positions, H-type at +1/2.
        self.be = {"x": prof(nx, 0.0, AX_X), "y": prof(ny, 0.0, AX_Y), "z": prof(nz, 0.0, AX_Z)}
        self.bh = {"x": prof(nx, 0.5, AX_X), "y": prof(ny, 0.5, AX_Y), "z": prof(nz, 0.5, AX_Z)}
        self.eps_r = np.ones(self.shape)
        self.gain = np.zeros(self.shape, dtype=bool)
        self.N_a = 0.0
        self.W_p = 0.0
        self.M, self.m = crank_nicolson(rate_matrix(self.p, 0.0), self.dt)
        self.seed = 0
        self.n = 0
        self.cell_index = np.arange(nx * ny * nz, dtype=np.uint64).reshape(self.shape)
        self.point_probes = []   # dicts: ijk, omegas, lams, acc (3, K) complex
        self.sources = []        # dicts: ijk, comp, lam, t0, tau, amp
        self.face_probes = None  # dict: stride, every, omegas, lams, faces
        self.plane_probes = []   # dicts: k, every, omegas, lams, acc (K, 3, ny, nx) complex
        self.flux = np.zeros(6)  # outward energy through x-,x+,y-,y+,z-,z+ faces

    # ------------------------------------------------------------- set-up
    def set_material(self, eps_r, gain_mask, N_a: float, W_p: float):
        """Per-cell eps_r (>= 1) and gain mask; N0 = N_a in gain cells (t = 0)."""
        eps_r = np.asarray(eps_r, dtype=np.float64).reshape(self.shape)
        gain = np.asarray(gain_mask).reshape(self.shape) != 0
        self.eps_r = eps_r.copy()
        self.gain = gain & (N_a > 0)
        self.N_a, self.W_p = float(N_a), float(W_p)
        self.M, self.m = crank_nicolson(rate_matrix(self.p, self.W_p), self.dt)
        self.N[:] = 0.0
        self.N[0][self.gain] = self.N_a
        for F in self.P + self.J:
            F[:] = 0.0

    def set_seed(self, seed: int):
        self.seed = int(seed) & 0xFFFFFFFFFFFFFFFF

    def add_point_probe(self, ijk, n_freq, lam_min, lam_max) -> int:
        lams = lambda_grid(n_freq, lam_min, lam_max)
        self.point_probes.append({"ijk": tuple(int(v) for v in ijk), "lams": lams,
                                  "omegas": 2.0 * math.pi * C0 / lams,
                                  "acc": np.zeros((3, n_freq), dtype=np.complex128)})
        return len(self.point_probes) - 1

    def add_source(self, ijk, comp, lam, t0, tau, amp):
        self.sources.append({"ijk": tuple(int(v) for v in ijk), "comp": int(comp),
                             "lam": lam, "t0": t0, "tau": tau, "amp": amp, "kind": "pulse"})

    def add_source_cw(self, ijk, comp, lam, t0, tau, amp, n_steps):
        """CW soft current (source_waveform_cw) for the n_steps steps from the
        first one whose half-step time t_{n+1/2} is >= t0; zero afterwards."""
        n0 = max(0, math.ceil(t0 / self.dt - 0.5))
        self.sources.append({"ijk": tuple(int(v) for v in ijk), "comp": int(comp),
                             "lam": lam, "t0": t0, "tau": tau, "amp": amp, "kind": "cw",
                             "n0": n0, "n1": n0 + int(n_steps)})

    def add_plane_probe(self, k, every, n_freq, lam_min, lam_max) -> int:
        """Running DFT of E on the whole plane z = k (every `every` steps)."""
        lams = lambda_grid(n_freq, lam_min, lam_max)
        self.plane_probes.append({"k": int(k), "every": int(every), "lams": lams,
                                  "omegas": 2.0 * math.pi * C0 / lams,
                                  "acc": np.zeros((n_freq, 3, self.ny, self.nx), dtype=np.complex128)})
        return len(self.plane_probes) - 1

    def add_face_probes(self, stride, every, n_freq, lam_min, lam_max):
        lams = lambda_grid(n_freq, lam_min, lam_max)
        self.face_probes = {"stride": int(stride), "every": int(every), "lams": lams,
                            "omegas": 2.0 * math.pi * C0 / lams, "faces": {}}

    # ---------------------------------------------------------- the step
    def step(self, n_steps: int = 1):
        for _ in range(n_steps):
            self._step_once()

    def _step_once(self):
        dt, dx = self.dt, self.dx
        Ex, Ey, Ez = self.E
        Hx, Hy, Hz = self.H
        be, bh, psE, psH = self.be, self.bh, self.psi_E, self.psi_H

        # 1. H^{n+1/2} = H^{n-1/2} - dt/mu0 curl E^n (forward differences) + CPML.
        dEz_dy = d_fwd(Ez, AX_Y) / dx
        dEy_dz = d_fwd(Ey, AX_Z) / dx
        dEx_dz = d_fwd(Ex, AX_Z) / dx
        dEz_dx = d_fwd(Ez, AX_X) / dx
        dEy_dx = d_fwd(Ey, AX_X) / dx
        dEx_dy = d_fwd(Ex, AX_Y) / dx
        for key, dF, w in ((("x", "y"), dEz_dy, "y"), (("x", "z"), dEy_dz, "z"),
                           (("y", "z"), dEx_dz, "z"), (("y", "x"), dEz_dx, "x"),
                           (("z", "x"), dEy_dx, "x"), (("z", "y"), dEx_dy, "y")):
            b, c = bh[w]
            psH[key] = b * psH[key] + c * dF
        Hx -= dt / MU0 * (dEz_dy - dEy_dz + psH[("x", "y")] - psH[("x", "z")])
        Hy -= dt / MU0 * (dEx_dz - dEz_dx + psH[("y", "z")] - psH[("y", "x")])
        Hz -= dt / MU0 * (dEy_dx - dEx_dy + psH[("z", "x")] - psH[("z", "y")])

        # 2-3. Lorentz polarization in the gain cells.
        E_old = [F.copy() for F in self.E]
        g = self.gain
        Jtot = [np.zeros(self.shape) for _ in range(3)]
        if g.any():
            gc = self.gc
            N1, N2 = self.N[1], self.N[2]
            dN = N1 - N2
            N_floor = self.p.n_floor_rel * self.N_a
            sigma_F = gc["a_se"] * np.sqrt((np.maximum(N2, 0.0) + N_floor) / (dx ** 3 * dt))
            zeta = langevin_normals(self.seed, self.cell_index, self.n)
            for c in range(3):
                J_new, P_new = lorentz_update(self.J[c], self.P[c], self.E[c], dN,
                                              sigma_F * zeta[c], dt, gc["w0"], gc["dw"], gc["xi"])
                self.J[c] = np.where(g, J_new, self.J[c])
                self.P[c] = np.where(g, P_new, self.P[c])
                Jtot[c] = np.where(g, self.J[c], 0.0)

        # soft current sources at t = (n + 1/2) dt
        t_half = (self.n + 0.5) * dt
        for s in self.sources:
            i, j, k = s["ijk"]
            if s["kind"] == "cw":
                if s["n0"] <= self.n < s["n1"]:
                    Jtot[s["comp"]][k, j, i] += source_waveform_cw(t_half, s["lam"], s["t0"], s["tau"],
                                                                   s["amp"])
            else:
                Jtot[s["comp"]][k, j, i] += source_waveform(t_half, s["lam"], s["t0"], s["tau"], s["amp"])

        # 4. E^{n+1} = E^n + dt/(eps0 eps_r) (curl H^{n+1/2} - J) (backward differences) + CPML.
        dHz_dy = d_bwd(Hz, AX_Y) / dx
        dHy_dz = d_bwd(Hy, AX_Z) / dx
        dHx_dz = d_bwd(Hx, AX_Z) / dx
        dHz_dx = d_bwd(Hz, AX_X) / dx
        dHy_dx = d_bwd(Hy, AX_X) / dx
        dHx_dy = d_bwd(Hx, AX_Y) / dx
        for key, dF, w in ((("x", "y"), dHz_dy, "y"), (("x", "z"), dHy_dz, "z"),
                           (("y", "z"), dHx_dz, "z"), (("y", "x"), dHz_dx, "x"),
                           (("z", "x"), dHy_dx, "x"), (("z", "y"), dHx_dy, "y")):
            b, c = be[w]
            psE[key] = b * psE[key] + c * dF
        ce = dt / (EPS0 * self.eps_r)
        Ex += ce * (dHz_dy - dHy_dz + psE[("x", "y")] - psE[("x", "z")] - Jtot[0])
        Ey += ce * (dHx_dz - dHz_dx + psE[("y", "z")] - psE[("y", "x")] - Jtot[1])
        Ez += ce * (dHy_dx - dHx_dy + psE[("z", "x")] - psE[("z", "y")] - Jtot[2])
        # PEC walls: tangential E on the planes i = 0, j = 0, k = 0.
        Ex[:, 0, :] = 0.0
        Ex[0, :, :] = 0.0
        Ey[:, :, 0] = 0.0
        Ey[0, :, :] = 0.0
        Ez[:, :, 0] = 0.0
        Ez[:, 0, :] = 0.0

        # 5. populations (Crank–Nicolson), driven by s = 1/2 (E^n + E^{n+1}) . J / (hbar w0).
        if g.any():
            EJ = sum(0.5 * (E_old[c] + self.E[c]) * self.J[c] for c in range(3))
            s = EJ / (HBAR * self.gc["w0"])
            N_new = population_update(self.N, s, self.M, self.m)
            self.N = np.where(g[None], N_new, self.N)

        self.n += 1
        self._probes(E_old)

    # ------------------------------------------------------------- probes
    def _probes(self, E_old):
        t = self.n * self.dt
        for pr in self.point_probes:
            i, j, k = pr["ijk"]
            for c in range(3):
                pr["acc"][c] = dft_accumulate(pr["acc"][c], self.E[c][k, j, i], pr["omegas"], t, self.dt)
        for pp in self.plane_probes:
            if self.n % pp["every"] == 0:
                ph = np.exp(1j * pp["omegas"] * t) * (pp["every"] * self.dt)       # E^{n+1} at t_{n+1}
                for c in range(3):
                    pp["acc"][:, c] += self.E[c][pp["k"]][None, :, :] * ph[:, None, None]
        E_mid = [0.5 * (a + b) for a, b in zip(E_old, self.E)]
        self.flux += self.dt * np.array(self.face_fluxes(E_mid))
        fp = self.face_probes
        if fp is not None and self.n % fp["every"] == 0:
            w = fp["omegas"]
            ph_E = np.exp(1j * w * t) * (fp["every"] * self.dt)                 # E^{n+1} at t_{n+1}
            ph_H = np.exp(1j * w * (t - 0.5 * self.dt)) * (fp["every"] * self.dt)  # H^{n+1/2}
            for face in range(6):
                Ea, Eb, Ha, Hb = self.face_fields(face, fp["stride"], self.E)
                acc = fp["faces"].setdefault(face, np.zeros((4,) + Ea.shape + (len(w),),
                                                             dtype=np.complex128))
                for q, (F, ph) in enumerate(((Ea, ph_E), (Eb, ph_E), (Ha, ph_H), (Hb, ph_H))):
                    acc[q] += F[..., None] * ph

    def _interior(self, n):
        L = self.p.npml
        return (L, n - L) if n - 2 * L > 0 else (0, n)

    def face_plane(self, axis_name: str, high: bool) -> int:
        n = {"x": self.nx, "y": self.ny, "z": self.nz}[axis_name]
        lo, hi = self._interior(n)
        return hi if high else lo

    def face_fields(self, face: int, stride: int, E):
        """Tangential (E_a, E_b) on a face plane p and (H_a, H_b) on the half-plane p - 1/2.

        (a, b, normal) is right-handed.  The six faces bound the interior box
        [npml, n - npml)^3: the low plane p = npml holds the box's first E
        layer and the H layer just outside it; the high plane p = n - npml
        holds the first E layer outside the box and the box's last H layer.
        With E = (E^n + E^{n+1})/2 and H = H^{n+1/2} this pairing is exactly
        the coupling the Yee curls make across the plane, so the box's
        discrete energy changes by -dt times the summed outward flux.
        Transverse extent: the box's rectangle, every ``stride``-th point.
        Sites outside the grid hold zero fields.
        """
        axis_name = "xyz"[face // 2]
        high = face % 2 == 1
        p = self.face_plane(axis_name, high)
        Ex, Ey, Ez = E
        Hx, Hy, Hz = self.H
        (x0, x1), (y0, y1), (z0, z1) = (self._interior(self.nx), self._interior(self.ny),
                                        self._interior(self.nz))
        sx, sy, sz = slice(x0, x1, stride), slice(y0, y1, stride), slice(z0, z1, stride)
        if axis_name == "x":
            n, pick = self.nx, (lambda F, q: F[sz, sy, q])
            comps = (Ey, Ez, Hy, Hz)
        elif axis_name == "y":
            n, pick = self.ny, (lambda F, q: F[sz, q, sx])
            comps = (Ez, Ex, Hz, Hx)
        else:
            n, pick = self.nz, (lambda F, q: F[q, sy, sx])
            comps = (Ex, Ey, Hx, Hy)
        zero = np.zeros(pick(Ex, 0).shape)
        Ea = pick(comps[0], p) if p < n else zero
        Eb = pick(comps[1], p) if p < n else zero
        Ha = pick(comps[2], p - 1) if p >= 1 else zero
        Hb = pick(comps[3], p - 1) if p >= 1 else zero
        return Ea, Eb, Ha, Hb

    def face_fluxes(self, E_mid):
        """Outward Poynting flux (W) through the six faces of the interior box."""
        out = []
        dA = self.dx * self.dx
        for face in range(6):
            Ea, Eb, Ha, Hb = self.face_fields(face, 1, E_mid)
            F = float(np.sum(Ea * Hb - Eb * Ha)) * dA
            out.append(F if face % 2 == 1 else -F)
        return out

    # ------------------------------------------------------------ read-out
    def probe_spectrum(self, probe_id: int):
        pr = self.point_probes[probe_id]
        return np.sum(np.abs(pr["acc"]) ** 2, axis=0), pr["lams"].copy()

    def face_spectrum(self, face: int):
        """Outward Poynting spectral density summed over the face sub-grid."""
        fp = self.face_probes
        acc = fp["faces"].get(face)
        K = len(fp["omegas"])
        if acc is None:
            return np.zeros(K), fp["lams"].copy()
        Ea, Eb, Ha, Hb = acc
        S = np.real(Ea * np.conj(Hb) - Eb * np.conj(Ha))
        S = S.reshape(-1, K).sum(axis=0) * (fp["stride"] * self.dx) ** 2
        return (S if face % 2 == 1 else -S), fp["lams"].copy()

    def plane_mode_map(self, probe_id: int, bin_: int) -> np.ndarray:
        """Sum over components of |DFT of E|^2 on the probe's plane, (ny, nx)."""
        acc = self.plane_probes[probe_id]["acc"][bin_]
        return np.sum(np.abs(acc) ** 2, axis=0)

    def plane_energy_density(self, k: int) -> np.ndarray:
        """Energy density (J/m^3) of the cells of plane z = k with the stored
        fields: 1/2 (eps0 eps_r |E|^2 + mu0 |H|^2), the per-cell terms of energy()."""
        uE = sum(F[k] * F[k] for F in self.E) * EPS0 * self.eps_r[k]
        uH = sum(F[k] * F[k] for F in self.H) * MU0
        return 0.5 * (uE + uH)

    def energy(self) -> float:
        """U = 1/2 sum (eps0 eps_r |E|^2 + mu0 |H|^2) dx^3 with the stored fields."""
        uE = sum(np.sum(self.eps_r * F * F) for F in self.E) * EPS0
        uH = sum(np.sum(F * F) for F in self.H) * MU0
        return 0.5 * (uE + uH) * self.dx ** 3

    def field(self, name: str) -> np.ndarray:
        """Named field: Ex Ey Ez Hx Hy Hz Px Py Pz Jx Jy Jz N0 N1 N2 N3."""
        group, c = name[0], name[1:]
        if group == "N":
            return self.N[int(c)]
        idx = "xyz".index(c)
        return {"E": self.E, "H": self.H, "P": self.P, "J": self.J}[group][idx]

    def set_field(self, name: str, values):
        values = np.asarray(values, dtype=np.float64).reshape(self.shape)
        group, c = name[0], name[1:]
        if group == "N":
            self.N[int(c)] = values.copy()
            return
        idx = "xyz".index(c)
        {"E": self.E, "H": self.H, "P": self.P, "J": self.J}[group][idx] = values.copy()


FIELD_NAMES = ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz", "Px", "Py", "Pz",
               "Jx", "Jy", "Jz", "N0", "N1", "N2", "N3")

"""FP64 discrete adjoint of the oracle's Maxwell–Bloch step.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` (and the CPU legs of
``bench.py``); never by the product package, with which it shares no code.

Objective.  The energy that crosses the plane z = p dx in +z during n steps,
over the transverse rectangle of the interior box (the CPML-free region):

    J = sum_n dt dx^2 sum_{i,j} [ Ex_mid(i,j,p) Hy(i,j,p-1) - Ey_mid(i,j,p) Hx(i,j,p-1) ]

with E_mid = (E^n + E^{n+1})/2 and H = H^{n+1/2}: the same discrete Poynting
pairing as the oracle's face flux (for p = n_z - npml it is exactly the
accumulated flux through the box's +z face).  The paper reports emission
observed through such probe planes ("Simulations" paragraph, spectra of
Figs. 1-2); the gradient of this energy with respect to the permittivity map
and the pump rate is the differentiable read-out built on the same step.

Method.  The step x^{n+1} = F(x^n; eps, W_p) (MBOracle._step_once) is
differentiated as a program: the reverse sweep runs n = N-1 .. 0 and maps the
adjoint of x^{n+1} to that of x^n by the transposed Jacobian of each sub-step,
taken in the reverse of the forward order (populations, E update, Lorentz
update, H update), with the objective's partial derivatives added at each
step.  The forward states are all kept (small grids only).  Transposes of the
differences: d_fwd^T = -d_bwd and d_bwd^T = -d_fwd (zero beyond the grid).
Parameter derivatives: d(ce)/d eps = -ce/eps for ce = dt/(eps0 eps_r);
the Crank–Nicolson propagator M = L^-1 R, m = dt L^-1 e with L = I - (dt/2)A,
R = I + (dt/2)A has dM/dW = (dt/2) L^-1 A_W (I + M) and dm/dW = (dt/2) L^-1
A_W m, A_W = dA/dW_p.

Pins (tests/test_oracle_adjoint.py): the difference transposes by inner
products; the objective against the oracle's own face flux; the gradient
against central finite differences of the forward objective (single cells in
the bulk, in the CPML and on gain cells; the pump; a random direction over all
cells).
"""
from __future__ import annotations

import numpy as np

from .mb_oracle import (AX_X, AX_Y, AX_Z, EPS0, HBAR, MU0, crank_nicolson, d_bwd, d_fwd,
                        langevin_normals, rate_matrix)

# (component, derivative axis) keys of the CPML memories, with the sign of
# the memory in that component's curl: curl_x = d_y F_z - d_z F_y + psi_xy - psi_xz, ...
_PSI_SIGN = {("x", "y"): 1.0, ("x", "z"): -1.0, ("y", "z"): 1.0, ("y", "x"): -1.0,
             ("z", "x"): 1.0, ("z", "y"): -1.0}
_AXIS = {"x": AX_X, "y": AX_Y, "z": AX_Z}
_COMP = {"x": 0, "y": 1, "z": 2}


def _other(key):
    """The field component whose derivative the memory (c, w) holds: the
    curl's c-component differentiates along w the component that is neither c
    nor w."""
    c, w = key
    return ({"x", "y", "z"} - {c, w}).pop()


def rate_matrix_dW() -> np.ndarray:
    """dA/dW_p of the four-level rate matrix (pump N0 -> N3)."""
    A = np.zeros((4, 4))
    A[0, 0] = -1.0
    A[3, 0] = 1.0
    return A


def crank_nicolson_dW(p, W_p: float, dt: float):
    """(dM/dW_p, dm/dW_p) of the Crank–Nicolson propagator."""
    A = rate_matrix(p, W_p)
    M, m = crank_nicolson(A, dt)
    L = np.eye(4) - 0.5 * dt * A
    AW = rate_matrix_dW()
    dM = 0.5 * dt * np.linalg.solve(L, AW @ (np.eye(4) + M))
    dm = 0.5 * dt * np.linalg.solve(L, AW @ m)
    return dM, dm


def default_z_plane(o) -> int:
    return o.face_plane("z", True)


def _rect(o):
    (x0, x1), (y0, y1) = o._interior(o.nx), o._interior(o.ny)
    return slice(y0, y1), slice(x0, x1)


def _snapshot(o):
    return {"E": [F.copy() for F in o.E], "H": [F.copy() for F in o.H],
            "P": [F.copy() for F in o.P], "J": [F.copy() for F in o.J],
            "N": o.N.copy(), "n": o.n}


def plane_flux(o, E0, E1, H1, p: int) -> float:
    """Energy crossing plane p in +z during one step (J): dt dx^2 sum(mx Hy - my Hx)."""
    if not (1 <= p < o.nz):
        raise ValueError("z plane must satisfy 1 <= p < n_z")
    sy, sx = _rect(o)
    mx = 0.5 * (E0[0][p, sy, sx] + E1[0][p, sy, sx])
    my = 0.5 * (E0[1][p, sy, sx] + E1[1][p, sy, sx])
    return o.dt * o.dx * o.dx * float(np.sum(mx * H1[1][p - 1, sy, sx] - my * H1[0][p - 1, sy, sx]))


def energy_zface(o, n_steps: int, z_plane: int | None = None) -> float:
    """Advance the oracle n_steps and return the objective J of that window."""
    p = default_z_plane(o) if z_plane is None else int(z_plane)
    J = 0.0
    for _ in range(n_steps):
        E0 = [F.copy() for F in o.E]
        o.step(1)
        J += plane_flux(o, E0, o.E, o.H, p)
    return J


def adjoint_energy_zface(o, n_steps: int, z_plane: int | None = None):
    """Advance the oracle n_steps; return {"J", "grad_eps", "grad_pump"}.

    grad_eps[k, j, i] = dJ/d eps_r of that cell (J per unit eps_r),
    grad_pump = dJ/dW_p (J s).  Noise and sources are held fixed (the same
    Philox stream for every eps and W_p).
    """
    p = default_z_plane(o) if z_plane is None else int(z_plane)
    dt, dx = o.dt, o.dx
    gc = o.gc
    g = o.gain
    gf = g.astype(np.float64)
    shape = o.shape
    states = [_snapshot(o)]
    J = 0.0
    for _ in range(n_steps):
        o.step(1)
        states.append(_snapshot(o))
        J += plane_flux(o, states[-2]["E"], states[-1]["E"], states[-1]["H"], p)

    # constants of the step
    a = 0.5 * gc["dw"] * dt
    cJ = (1.0 - a) / (1.0 + a)           # J^{n+1/2} per J^{n-1/2}
    cF = dt / (1.0 + a)                  # J^{n+1/2} per unit of the bracket
    w0 = gc["w0"]
    ce = dt / (EPS0 * o.eps_r)
    M, m = o.M, o.m
    dM, dm = crank_nicolson_dW(o.p, o.W_p, dt)
    N_floor = o.p.n_floor_rel * o.N_a
    mask = [np.ones(shape) for _ in range(3)]   # PEC: tangential E on i=0, j=0, k=0
    mask[0][:, 0, :] = 0.0
    mask[0][0, :, :] = 0.0
    mask[1][:, :, 0] = 0.0
    mask[1][0, :, :] = 0.0
    mask[2][:, :, 0] = 0.0
    mask[2][:, 0, :] = 0.0
    sy, sx = _rect(o)

    z = lambda: np.zeros(shape)
    lE, lH, lP, lJ = [z(), z(), z()], [z(), z(), z()], [z(), z(), z()], [z(), z(), z()]
    lN = np.zeros((4,) + shape)
    lpsE = {key: z() for key in _PSI_SIGN}
    lpsH = {key: z() for key in _PSI_SIGN}
    grad_eps = z()
    grad_W = 0.0

    for n in range(n_steps - 1, -1, -1):
        s0, s1 = states[n], states[n + 1]
        E0, E1, H1, J1, N0 = s0["E"], s1["E"], s1["H"], s1["J"], s0["N"]
        lE0 = [z(), z(), z()]
        lE1 = [F.copy() for F in lE]
        lH1 = [F.copy() for F in lH]

        # objective of this step
        w = dt * dx * dx
        lE1[0][p, sy, sx] += 0.5 * w * H1[1][p - 1, sy, sx]
        lE1[1][p, sy, sx] -= 0.5 * w * H1[0][p - 1, sy, sx]
        lE0[0][p, sy, sx] += 0.5 * w * H1[1][p - 1, sy, sx]
        lE0[1][p, sy, sx] -= 0.5 * w * H1[0][p - 1, sy, sx]
        lH1[1][p - 1, sy, sx] += w * 0.5 * (E0[0][p, sy, sx] + E1[0][p, sy, sx])
        lH1[0][p - 1, sy, sx] -= w * 0.5 * (E0[1][p, sy, sx] + E1[1][p, sy, sx])

        # 5. populations: N^{n+1} = M N^n + m s in gain cells
        lJ1 = [F.copy() for F in lJ]
        if g.any():
            EJ = sum(0.5 * (E0[c] + E1[c]) * J1[c] for c in range(3))
            s = EJ / (HBAR * w0)
            ls = np.tensordot(m, lN, axes=(0, 0)) * gf
            dN = np.tensordot(dM, N0, axes=(1, 0)) + dm.reshape(4, 1, 1, 1) * s
            grad_W += float(np.sum(lN * dN * gf[None]))
            lN = np.where(g[None], np.tensordot(M.T, lN, axes=(1, 0)), lN)
            for c in range(3):
                lE1[c] += ls * 0.5 * J1[c] / (HBAR * w0)
                lE0[c] += ls * 0.5 * J1[c] / (HBAR * w0)
                lJ1[c] += ls * 0.5 * (E0[c] + E1[c]) / (HBAR * w0)

        # 4. E^{n+1} = mask (E^n + ce (curl_bwd H^{n+1/2} + psi_E - J_tot))
        lEt = [mask[c] * lE1[c] for c in range(3)]
        grad_eps -= sum(lEt[c] * (E1[c] - E0[c]) for c in range(3)) / o.eps_r
        u = [ce * lEt[c] for c in range(3)]
        for c in range(3):
            lE0[c] += lEt[c]
            lJ1[c] -= gf * u[c]
        # coefficient of each backward difference d_w F (F = the third
        # component) in the update: u directly, and through psi_E
        for key, sign in _PSI_SIGN.items():
            c, wax = key
            tot = lpsE[key] + sign * u[_COMP[c]]
            b, cc = o.be[wax]
            lpsE[key] = b * tot
            coef = sign * u[_COMP[c]] + cc * tot
            F = _COMP[_other(key)]
            lH1[F] += -d_fwd(coef, _AXIS[wax]) / dx

        # 2-3. Lorentz polarization (gain cells): P^{n+1} = P^n + dt J^{n+1/2},
        # J^{n+1/2} = cJ J^{n-1/2} + cF (xi dN E^n - w0^2 P^n + sigma_F(N2) zeta)
        if g.any():
            N1, N2 = N0[1], N0[2]
            dNn = N1 - N2
            root = np.sqrt((np.maximum(N2, 0.0) + N_floor) / (dx ** 3 * dt))
            dsig = np.where(N2 > 0.0, gc["a_se"] * 0.5 / (root * dx ** 3 * dt), 0.0)
            zeta = langevin_normals(o.seed, o.cell_index, s0["n"])
            lJt = [lJ1[c] + dt * lP[c] for c in range(3)]
            for c in range(3):
                lE0[c] += gf * cF * gc["xi"] * dNn * lJt[c]
            ldN = gf * cF * gc["xi"] * sum(E0[c] * lJt[c] for c in range(3))
            lN[1] += ldN
            lN[2] -= ldN
            lN[2] += gf * cF * dsig * sum(zeta[c] * lJt[c] for c in range(3))
            for c in range(3):
                lP[c] = np.where(g, lP[c] - cF * w0 * w0 * lJt[c], lP[c])
                lJ[c] = np.where(g, cJ * lJt[c], lJ1[c])
        else:
            lJ = lJ1

        # 1. H^{n+1/2} = H^{n-1/2} - dt/mu0 (curl_fwd E^n + psi_H)
        v = [-dt / MU0 * lH1[c] for c in range(3)]
        for key, sign in _PSI_SIGN.items():
            c, wax = key
            tot = lpsH[key] + sign * v[_COMP[c]]
            b, cc = o.bh[wax]
            lpsH[key] = b * tot
            coef = sign * v[_COMP[c]] + cc * tot
            F = _COMP[_other(key)]
            lE0[F] += -d_bwd(coef, _AXIS[wax]) / dx
        lH = lH1
        lE = lE0

    return {"J": J, "grad_eps": grad_eps, "grad_pump": grad_W}

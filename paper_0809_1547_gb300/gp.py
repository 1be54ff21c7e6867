"""Theory curves of the random-laser spectrum versus pump (the paper's
"Gross-Pitaevskii equation" paragraph, Figs. 3 and 5).

The envelope equation -phi'' + tau^2 phi + phi^3 = E phi is solved on the
GPU (``mb_gp_features``) for the nonlinear eigenvalue
    E(p) = (p - 1) / (kappa sqrt(p)),
where p is the pump in units of the threshold gain of the high-Q modes and
kappa = (t_g / t_L) sqrt(alpha0/alpha_L - 1).  Its Fourier transform gives
the normalised waist w_phi and peak p_phi, hence the linewidth and the peak
of the spectrum:
    W t_g = w_phi sqrt(kappa) / p^{1/4},      S_p gamma_S / t_g^2 = p_phi.
Lasing needs E > 1, i.e. p above
    p_th = 1 + kappa^2 / 2 + kappa sqrt(4 + kappa^2) / 2.
"""
from __future__ import annotations

import math

import numpy as np

from .binding import mb_gp_features


def E_of_p(p, kappa: float):
    p = np.asarray(p, dtype=np.float64)
    return (p - 1.0) / (kappa * np.sqrt(p))


def p_threshold(kappa: float) -> float:
    return 1.0 + 0.5 * kappa * kappa + 0.5 * kappa * math.sqrt(4.0 + kappa * kappa)


def spectral_features(E, n_grid: int = 2047):
    """(w_phi, p_phi) for eigenvalues E > 1 (GPU, FP64)."""
    return mb_gp_features(E, n_grid)


def theory_curves(p, kappa: float, n_grid: int = 2047) -> dict:
    """Linewidth W t_g and peak S_p gamma_S / t_g^2 versus pump p (> p_th)."""
    p = np.asarray(p, dtype=np.float64)
    if np.any(p <= p_threshold(kappa)):
        raise ValueError("every pump must exceed the threshold p_th(kappa)")
    E = E_of_p(p, kappa)
    w, pk = spectral_features(E, n_grid)
    return {"p": p, "E": E, "W_tg": w * math.sqrt(kappa) / p ** 0.25, "S_p": pk,
            "p_th": p_threshold(kappa)}

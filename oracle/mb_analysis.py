"""Spectral statistics of a pump sweep, written out as their definitions.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``; never by the product
package, with which it shares no code.

The paper characterises random lasing by the emission peak and the linewidth
of the spectrum versus the pump: the linewidth as a standard deviation of the
spectrum (experiment, "Experimental results" paragraph, Fig. 4b) and by a
Gaussian fit (the Maxwell–Bloch simulations shown in Fig. 5b).  For a
spectrum S_k sampled on angular frequencies w_k:

    peak:        k* = argmax S_k, (w_{k*}, S_{k*})
    centroid:    wbar = sum S_k w_k / sum S_k
    std width:   sigma = sqrt(sum S_k (w_k - wbar)^2 / sum S_k)
    Gaussian:    the least-squares parabola ln S = a + b w + c w^2 through the
                 samples with S_k >= frac * S_{k*}; sigma_G = sqrt(-1/(2c)),
                 centre -b/(2c) (undefined when c >= 0 or fewer than 3 samples)
    threshold:   the lowest pump level whose mean std width is at most half
                 the mean std width at the lowest level (gain narrowing), or
                 None when no level narrows that far.
    emission threshold: with E_q the mean emitted energy (sum of S) at the
                 q-th level L_q (ascending), the lowest L_q from which the
                 log-log slope ln(E_{q+1}/E_q) / ln(L_{q+1}/L_q) exceeds 2,
                 or None: spontaneous emission grows in proportion to the
                 number of atoms (slope ~1), stimulated emission above
                 threshold makes the growth super-linear.

Pins (tests/test_oracle_analysis.py): a sampled Gaussian gives back its
centre and width; a flat spectrum's std width is that of a uniform
distribution; a two-line spectrum's std width is half the line spacing; a
synthetic S-curve gives back its kink, and power laws up to slope 2 have
no emission threshold.
"""
from __future__ import annotations

import math

import numpy as np

C0 = 299_792_458.0


def omegas_of(lams) -> np.ndarray:
    return 2.0 * math.pi * C0 / np.asarray(lams, dtype=np.float64)


def peak(S, w):
    k = int(np.argmax(S))
    return float(w[k]), float(S[k])


def std_width(S, w) -> float:
    S = np.asarray(S, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    tot = S.sum()
    mean = (S * w).sum() / tot
    return math.sqrt((S * (w - mean) ** 2).sum() / tot)


def gaussian_fit(S, w, frac: float = 0.1):
    """(centre, sigma) of the least-squares Gaussian near the peak, or (None, None)."""
    S = np.asarray(S, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    keep = S >= frac * S.max()
    if keep.sum() < 3:
        return None, None
    x = w[keep]
    y = np.log(S[keep])
    x0 = x.mean()
    # normal equations of y = a + b (x - x0) + c (x - x0)^2
    X = np.stack([np.ones_like(x), x - x0, (x - x0) ** 2], axis=1)
    a, b, c = np.linalg.solve(X.T @ X, X.T @ y)
    if c >= 0:
        return None, None
    return float(x0 - b / (2.0 * c)), float(math.sqrt(-1.0 / (2.0 * c)))


def sweep_table(levels, spectra, w):
    """Per pump level (sorted): mean peak frequency, mean std width, mean
    Gaussian width (over instances where the fit exists), and the threshold
    level.  `levels[i]` is the pump of spectrum `spectra[i]`."""
    levels = np.asarray(levels, dtype=np.float64)
    rows = []
    for L in sorted(set(levels.tolist())):
        idx = [i for i in range(len(levels)) if levels[i] == L]
        pk = [peak(spectra[i], w)[0] for i in idx]
        sd = [std_width(spectra[i], w) for i in idx]
        gf = [gaussian_fit(spectra[i], w)[1] for i in idx]
        gf = [g for g in gf if g is not None]
        em = [float(np.sum(spectra[i])) for i in idx]
        rows.append({"level": L, "peak_w": float(np.mean(pk)), "std_w": float(np.mean(sd)),
                     "gauss_w": float(np.mean(gf)) if gf else None, "n": len(idx),
                     "emitted": float(np.mean(em))})
    thr = None
    for r in rows:
        if r["std_w"] <= 0.5 * rows[0]["std_w"]:
            thr = r["level"]
            break
    return rows, thr


def emission_threshold(levels, emitted, slope: float = 2.0):
    """The lowest level L_q (levels ascending) from which the emitted energy
    grows faster than L^slope to the next level, or None."""
    for q in range(len(levels) - 1):
        g = math.log(emitted[q + 1] / emitted[q]) / math.log(levels[q + 1] / levels[q])
        if g > slope:
            return float(levels[q])
    return None

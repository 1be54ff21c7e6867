"""Pump sweep over a batched ensemble: emission peak, linewidth and threshold
versus the atomic density N_a (the simulation side of the paper's Fig. 5b,
"Experimental results" paragraph: linewidth as a standard deviation and by a
Gaussian fit of the spectrum).

Every realization of the ensemble (N_a levels x disorder seeds) runs in one
MBBatch; each carries a centre point probe whose running DFT (on the GPU)
gives its spectrum.  The statistics of the spectra are host-side
reductions of a few hundred numbers per realization:

    peak       the bin of largest S
    std width  sqrt(sum S (w - wbar)^2 / sum S), wbar the S-weighted mean
    Gaussian   a parabola fitted to ln S over the bins with S >= 0.1 max S:
               sigma = sqrt(-1 / (2 c)) for the quadratic coefficient c < 0
    threshold  the lowest N_a whose mean std width is at most half of the
               lowest level's (gain narrowing)
    emission   the lowest N_a from which the mean emitted energy grows faster
    threshold  than N_a^2 to the next level (spontaneous emission grows as
               N_a, stimulated emission above threshold faster)

    python -m paper_0809_1547_gb300.sweep --steps 8000 --out sweep.json

`--window-from S` restarts the probes at step S, so the spectra are those of
the emission after S (the spontaneous background of the first steps left
out).
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

C0 = 299_792_458.0
LAM_MIN, LAM_MAX, N_FREQ = 475e-9, 705e-9, 128


def spectral_stats(S: np.ndarray, lam: np.ndarray, frac: float = 0.1) -> dict:
    """Statistics of spectra S (instances x bins) on wavelengths lam (bins)."""
    S = np.atleast_2d(np.asarray(S, dtype=np.float64))
    w = 2.0 * math.pi * C0 / np.asarray(lam, dtype=np.float64)
    kpk = np.argmax(S, axis=1)
    tot = S.sum(axis=1)
    wbar = (S @ w) / tot
    var = (S * (w[None, :] - wbar[:, None]) ** 2).sum(axis=1) / tot
    gauss = np.full(S.shape[0], np.nan)
    for q in range(S.shape[0]):
        sel = S[q] >= frac * S[q, kpk[q]]
        if sel.sum() >= 3:
            ws = w[sel]
            c2, _, _ = np.polyfit(ws - ws.mean(), np.log(S[q, sel]), 2)
            if c2 < 0:
                gauss[q] = math.sqrt(-0.5 / c2)
    return {"peak_w": w[kpk], "peak_lam": np.asarray(lam)[kpk], "peak_S": S[np.arange(S.shape[0]), kpk],
            "std_w": np.sqrt(var), "gauss_w": gauss, "total": tot}


def summarize(levels, stats: dict) -> tuple[list, float | None]:
    """Per N_a level (ascending): means over the realizations at that level."""
    levels = np.asarray(levels, dtype=np.float64)
    rows = []
    for L in np.unique(levels):
        m = levels == L
        g = stats["gauss_w"][m]
        g = g[np.isfinite(g)]
        rows.append({"N_a": float(L), "n": int(m.sum()),
                     "peak_lam_nm": float(np.mean(stats["peak_lam"][m]) * 1e9),
                     "peak_w": float(np.mean(stats["peak_w"][m])),
                     "std_w": float(np.mean(stats["std_w"][m])),
                     "std_w_spread": float(np.std(stats["std_w"][m])),
                     "gauss_w": float(np.mean(g)) if g.size else None,
                     "emitted": float(np.mean(stats["total"][m]))})
    base = rows[0]["std_w"]
    thr = next((r["N_a"] for r in rows if r["std_w"] <= 0.5 * base), None)
    return rows, thr


def emission_threshold(rows, slope: float = 2.0):
    """The lowest N_a (rows ascending, as summarize returns them) from which
    the log-log slope of the mean emitted energy to the next level exceeds
    `slope`, or None."""
    L = np.array([r["N_a"] for r in rows])
    E = np.array([r["emitted"] for r in rows])
    g = np.log(E[1:] / E[:-1]) / np.log(L[1:] / L[:-1])
    hit = np.nonzero(g > slope)[0]
    return float(L[hit[0]]) if hit.size else None


def run_pump_sweep(workloads, steps: int, stream=None, autotune: bool = True, record=(),
                   window_from: int = 0):
    """Advance every workload of the ensemble `steps` steps in one MBBatch
    and return (levels, spectra, lam, seconds).  With `record` (ascending
    step counts below `steps`), also the spectra at each of those counts:
    then returns (levels, spectra, lam, seconds, [(step, spectra), ...]).
    With window_from > 0 the probes restart at that step (mb_reset_probes),
    so the spectra read later cover the window [window_from, step) only."""
    from .binding import MBBatch, mb_default_params
    b = MBBatch([w.grid for w in workloads], workloads[0].dx, workloads[0].dt,
                mb_default_params(npml=workloads[0].npml), stream=stream)

    def read():
        out, lam_ = [], None
        for inst in b.instances:
            S, lam_ = inst.probe_spectrum(0)
            out.append(S)
        return np.array(out), lam_

    snaps = []
    try:
        for q, w in enumerate(workloads):
            b.set_instance(q, w.eps, w.gain, w.N_a, w.pump, w.seed)
            b.instances[q].add_point_probe(tuple(v // 2 for v in w.grid), N_FREQ, LAM_MIN, LAM_MAX)
        if autotune:
            b.autotune()
        t0 = time.perf_counter()
        done = 0
        rec = {int(v) for v in record if 0 < int(v) < steps}
        marks = sorted(rec |
                       ({int(window_from)} if 0 < window_from < steps else set()))
        for r in marks:
            b.step(r - done)
            b.synchronize()
            done = r
            if r in rec:
                snaps.append((r, read()[0]))
            if r == window_from:
                for inst in b.instances:
                    inst.reset_probes()
        b.step(steps - done)
        b.synchronize()
        secs = time.perf_counter() - t0
        spectra, lam = read()
    finally:
        b.close()
    levels = [w.N_a for w in workloads]
    if record:
        return levels, spectra, lam, secs, snaps
    return levels, spectra, lam, secs


def main():
    from . import inputs
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--n-pump", type=int, default=16)
    ap.add_argument("--n-seed", type=int, default=5)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--na-min", type=float, default=5e23, help="lowest N_a level (m^-3)")
    ap.add_argument("--na-max", type=float, default=2e25, help="highest N_a level (m^-3)")
    ap.add_argument("--pump", type=float, default=0.0,
                    help="pump rate W_p (1/s) of every realization (default: the workload's)")
    ap.add_argument("--top-levels", type=int, default=0,
                    help="keep only the highest N_a levels (all seeds of each)")
    ap.add_argument("--record", default="",
                    help="comma-separated step counts at which the statistics are also taken "
                         "(spectra accumulated from step 0)")
    ap.add_argument("--window-from", type=int, default=0,
                    help="restart the probes at this step: the spectra cover the later steps only")
    ap.add_argument("--out", default="")
    args = ap.parse_args()
    ws = inputs.workload_batch(n_pump=args.n_pump, n_seed=args.n_seed, N_a_lo=args.na_min,
                               N_a_hi=args.na_max)
    if args.pump > 0:
        for w in ws:
            w.pump = args.pump
    if args.top_levels > 0:
        keep = sorted({w.N_a for w in ws})[-args.top_levels:]
        ws = [w for w in ws if w.N_a in keep]
    record = [int(v) for v in args.record.split(",") if v.strip()]
    res = run_pump_sweep(ws, args.steps, record=record, window_from=args.window_from)
    levels, spectra, lam, secs = res[:4]
    snaps = res[4] if record else []
    stats = spectral_stats(spectra, lam)
    rows, thr = summarize(levels, stats)
    cells = sum(int(np.prod(w.grid)) for w in ws)
    dt = ws[0].dt
    out = {"instances": len(ws), "steps": args.steps, "t_ps": args.steps * dt * 1e12,
           "spectra_from_step": args.window_from,
           "pump_W_p": ws[0].pump, "seconds": secs,
           "mcell_updates_per_s": cells * args.steps / secs / 1e6, "threshold_N_a": thr,
           "emission_threshold_N_a": emission_threshold(rows),
           "levels": rows,
           "history": []}
    for st, S in snaps:
        r_, thr_ = summarize(levels, spectral_stats(S, lam))
        out["history"].append({"step": st, "t_ps": st * dt * 1e12, "threshold_N_a": thr_,
                               "emission_threshold_N_a": emission_threshold(r_), "levels": r_})
    text = json.dumps(out, indent=1)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text)
    print(text)


if __name__ == "__main__":
    main()

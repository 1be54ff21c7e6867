"""The paper-scale single realization end to end ("Simulations" paragraph,
Figs. 1-2): a 320^3 packing of ~8000 TiO2 spheres, first its passive
response to a single-cycle 532 nm pulse at the centre, then an active run
(gain in the voids, N_a above threshold, Langevin noise, no source) of 20000
steps with DFT probes on the six faces of the interior box.

Read-outs, all on the GPU path (the host only reduces a few hundred numbers):

    passive   the field energy U(t) every `every` steps (its decay after the
              pulse leaves the source region: the sample's slowest leak), the
              energy through the six faces, the centre probe's spectrum and
              the faces' outward spectral energy summed
    active    U(t) and the emitted energy (six faces) every `every` steps, the
              six faces' outward spectral energy summed: emission peak,
              std width and Gaussian width (spectral_stats), total

    python -m paper_0809_1547_gb300.sample_run --steps 20000 --out sample.json
"""
from __future__ import annotations

import argparse
import copy
import json
import math
import time

import numpy as np

from .sweep import spectral_stats
from .workloads import FACE_EVERY, FACE_STRIDE, LAM_MAX, LAM_MIN, N_FREQ, setup_simulation


def _faces_total(sim):
    S, lam = None, None
    for face in range(6):
        Sf, lam = sim.face_spectrum(face)
        S = np.asarray(Sf, dtype=np.float64) if S is None else S + Sf
    return S, np.asarray(lam)


def _stats(S, lam):
    st = spectral_stats(np.clip(S, 0.0, None)[None, :], lam)
    return {"peak_nm": float(st["peak_lam"][0] * 1e9), "std_w": float(st["std_w"][0]),
            "gauss_w": None if not np.isfinite(st["gauss_w"][0]) else float(st["gauss_w"][0]),
            "total": float(st["total"][0])}


def _run(sim, steps, every):
    """Steps in blocks of `every`, with (step, t_ps, U, emitted) after each."""
    rows = []
    done = 0
    t0 = time.perf_counter()
    while done < steps:
        n = min(every, steps - done)
        sim.step(n)
        done += n
        U, fl = sim.energy()
        rows.append({"step": done, "t_ps": done * sim.dt * 1e12, "U_J": float(U),
                     "emitted_J": float(np.sum(fl))})
    sim.synchronize()
    return rows, time.perf_counter() - t0


def run_sample(w, steps: int = 20000, passive_steps: int = 10000, every: int = 1000, stream=None):
    out = {"workload": w.name, "grid": list(w.grid), "spheres": int(w.n_spheres),
           "fill": float(w.fill), "dt_s": w.dt, "N_a": w.N_a, "W_p": w.pump}
    mid = tuple(v // 2 for v in w.grid)
    # passive: the single-cycle pulse (tau 1 fs, centred at 4 fs) at the centre
    wp = copy.copy(w)
    wp.N_a = 0.0
    sim = setup_simulation(wp, autotune=True, stream=stream)
    sim.set_source(mid, 2, 532e-9, 4e-15, 1e-15, 1e9)
    rows, secs = _run(sim, passive_steps, every)
    Sc, lam = sim.probe_spectrum(0)
    Sf, lamf = _faces_total(sim)
    peak = max(r["U_J"] for r in rows)
    late = [r for r in rows if r["t_ps"] > 0.1 and r["U_J"] > 0]
    tau = None
    if len(late) >= 2:
        a, b = late[0], late[-1]
        if b["U_J"] < a["U_J"]:
            tau = (b["t_ps"] - a["t_ps"]) / math.log(a["U_J"] / b["U_J"])
    out["passive"] = {"steps": passive_steps, "seconds": secs, "history": rows,
                      "U_peak_J": peak, "U_decay_time_ps": tau,
                      "centre": _stats(np.asarray(Sc), np.asarray(lam)), "faces": _stats(Sf, lamf),
                      "faces_S": Sf.tolist(), "lam_nm": (lamf * 1e9).tolist()}
    sim.close()
    # active: gain on, Langevin noise, no source
    sim = setup_simulation(w, autotune=True, stream=stream)
    rows, secs = _run(sim, steps, every)
    Sc, lam = sim.probe_spectrum(0)
    Sf, lamf = _faces_total(sim)
    out["active"] = {"steps": steps, "t_ps": steps * w.dt * 1e12, "seconds": secs,
                     "mcell_updates_per_s": w.ncell * steps / secs / 1e6, "history": rows,
                     "centre": _stats(np.asarray(Sc), np.asarray(lam)), "faces": _stats(Sf, lamf),
                     "faces_S": Sf.tolist(), "lam_nm": (lamf * 1e9).tolist(),
                     "probes": {"face_stride": FACE_STRIDE, "face_every": FACE_EVERY, "bins": N_FREQ,
                                "lam_nm": [LAM_MIN * 1e9, LAM_MAX * 1e9]}}
    sim.close()
    return out


def main():
    from . import inputs
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--grid", type=int, default=320)
    ap.add_argument("--steps", type=int, default=20000, help="active run steps")
    ap.add_argument("--passive-steps", type=int, default=10000)
    ap.add_argument("--every", type=int, default=1000, help="read-out interval (steps)")
    ap.add_argument("--out", default="")
    args = ap.parse_args()
    w = inputs.workload_paper(args.grid)
    out = run_sample(w, args.steps, args.passive_steps, args.every)
    text = json.dumps(out, indent=1)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text)
    print(json.dumps({k: out[k] for k in ("workload", "grid", "spheres", "fill")}))
    for part in ("passive", "active"):
        p = out[part]
        print(part, json.dumps({k: p[k] for k in p if k not in ("history", "faces_S", "lam_nm")}))


if __name__ == "__main__":
    main()

"""Host logic of the paper-scale run (sample_run) on the CPU: a stand-in
simulation whose energy decays as exp(-t / 0.2 ps) after the pulse and whose
face spectra are a known Gaussian line; the read-outs must give that decay
time, the line's peak and its width."""
import math
from types import SimpleNamespace

import numpy as np

from paper_0809_1547_gb300 import sample_run

C0 = 299_792_458.0


class _FakeSim:
    def __init__(self, w, tau_ps=0.2, lam0=560e-9, sig_w=1.5e14):
        self.dt = w.dt
        self.n = 0
        self.tau_ps = tau_ps
        self.lam = np.linspace(475e-9, 705e-9, 128)
        w_ = 2 * math.pi * C0 / self.lam
        w0 = 2 * math.pi * C0 / lam0
        self.line = np.exp(-0.5 * ((w_ - w0) / sig_w) ** 2)

    def set_source(self, *a):
        pass

    def step(self, n):
        self.n += n

    def energy(self):
        t = self.n * self.dt * 1e12
        return 1e-18 * math.exp(-t / self.tau_ps), np.full(6, 1e-20)

    def probe_spectrum(self, pid):
        return self.line * 2.0, self.lam

    def face_spectrum(self, face):
        return self.line * (face + 1), self.lam

    def synchronize(self):
        pass

    def close(self):
        pass


def test_sample_run_reductions(monkeypatch):
    w = SimpleNamespace(name="fake", grid=(8, 8, 8), n_spheres=3, fill=0.4, dt=3.8e-17, N_a=5e24,
                        pump=1e13, ncell=512)
    monkeypatch.setattr(sample_run, "setup_simulation", lambda w_, autotune=True, stream=None: _FakeSim(w_))
    out = sample_run.run_sample(w, steps=4000, passive_steps=10000, every=1000)
    p, a = out["passive"], out["active"]
    assert len(p["history"]) == 10 and len(a["history"]) == 4
    assert p["history"][-1]["step"] == 10000 and a["history"][-1]["step"] == 4000
    assert abs(p["U_decay_time_ps"] - 0.2) < 1e-9
    for part in (p, a):
        assert abs(part["faces"]["peak_nm"] - 560.0) < 2.0          # within a bin of the line
        assert abs(part["faces"]["gauss_w"] / 1.5e14 - 1.0) < 0.02   # the line's width
        assert abs(sum(part["faces_S"]) - 21 * float(np.sum(_FakeSim(w).line))) < 1e-9 * sum(part["faces_S"])

"""Helpers for running the CUDA path and the oracle on identical inputs."""
from __future__ import annotations

import math

import numpy as np

from oracle.mb_oracle import MBOracle, Params, FIELD_NAMES

DX = 20e-9
DT = 0.99 * DX / (299_792_458.0 * math.sqrt(3.0))

# Per-field tolerance after the run: relative L2 of (gpu - oracle) / oracle.
# 1e-5 is the bound stated for the FP32 step against the FP64 oracle.
REL_L2_TOL = 1e-5


def params_kw(**kw):
    base = dict(lambda0=590e-9, dlambda=230e-9, tau32=100e-15, tau21=1e-9, tau10=100e-15,
                a_se=-1.0, dipole_len=0.1e-9, n_floor_rel=1e-9, npml=8, pml_order=3.0,
                pml_sigma_factor=0.8, pml_alpha_rel=0.1)
    base.update(kw)
    return base


def make_pair(grid, eps, gain, N_a, pump, seed, pkw, dt=DT, dx=DX):
    """An oracle and a GPU simulation set up identically (fields zero)."""
    from paper_0809_1547_gb300.binding import MBSimulation, mb_default_params
    o = MBOracle(grid, dx, dt, Params(**pkw))
    o.set_material(eps, gain, N_a, pump)
    o.set_seed(seed)
    g = MBSimulation(grid, dx, dt, mb_default_params(**pkw))
    g.set_material(eps, gain, N_a, pump)
    g.set_seed(seed)
    return o, g


def rel_l2(gpu, ref):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref)
    num = np.linalg.norm(gpu - ref)
    if den == 0.0:
        return 0.0 if num == 0.0 else math.inf
    return num / den


def field_errors(o, g, names=FIELD_NAMES):
    return {name: rel_l2(g.field(name), o.field(name)) for name in names}


def assert_fields_match(o, g, tol=REL_L2_TOL, names=FIELD_NAMES):
    errs = field_errors(o, g, names)
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, f"fields beyond rel-L2 {tol}: {bad}"
    return errs

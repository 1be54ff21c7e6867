"""Thin ctypes binding of the C ABI in ``include/mb_fdtd.h``.

Argument marshalling only: every step of the computation runs in the CUDA
library ``libmbfdtd.so``.  The functions carry the C names (``mb_create``,
``mb_step``, ...); :class:`MBSimulation` wraps one context.  If the library
has not been built, or cannot be loaded, every call raises
:class:`MBLibraryError`; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmbfdtd.so")

MB_OK, MB_ERR_ARG, MB_ERR_COURANT, MB_ERR_OOM, MB_ERR_MATERIALS = 0, -1, -2, -3, -4
MB_ERR_TIMEOUT, MB_ERR_NONFINITE, MB_ERR_CUDA, MB_ERR_STATE = -5, -6, -7, -8
MB_BATCH_PERSISTENT, MB_BATCH_CONCURRENT = 0, 1
ERROR_NAMES = {MB_ERR_ARG: "MB_ERR_ARG", MB_ERR_COURANT: "MB_ERR_COURANT", MB_ERR_OOM: "MB_ERR_OOM",
               MB_ERR_MATERIALS: "MB_ERR_MATERIALS", MB_ERR_TIMEOUT: "MB_ERR_TIMEOUT",
               MB_ERR_NONFINITE: "MB_ERR_NONFINITE", MB_ERR_CUDA: "MB_ERR_CUDA",
               MB_ERR_STATE: "MB_ERR_STATE"}

FIELDS = ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz", "Px", "Py", "Pz",
          "Jx", "Jy", "Jz", "N0", "N1", "N2", "N3")
FIELD_ID = {name: i for i, name in enumerate(FIELDS)}


class MBLibraryError(RuntimeError):
    """The CUDA library is missing or failed to load."""


class MBError(RuntimeError):
    """A C-ABI call returned an error code."""

    def __init__(self, code, msg):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


class mb_params(C.Structure):
    _fields_ = [("lambda0", C.c_double), ("dlambda", C.c_double), ("tau32", C.c_double),
                ("tau21", C.c_double), ("tau10", C.c_double), ("a_se", C.c_double),
                ("dipole_len", C.c_double), ("n_floor_rel", C.c_double), ("npml", C.c_int),
                ("pml_order", C.c_double), ("pml_sigma_factor", C.c_double),
                ("pml_alpha_rel", C.c_double), ("n_ref", C.c_double)]


# (name, restype, argtypes) of every exported function
_P = C.c_void_p
_SIGS = [
    ("mb_default_params", None, [C.POINTER(mb_params)]),
    ("mb_last_error", C.c_char_p, [_P]),
    ("mb_create", C.c_int, [C.POINTER(_P), C.POINTER(C.c_int), C.c_double, C.c_double,
                            C.POINTER(mb_params), _P]),
    ("mb_destroy", C.c_int, [_P]),
    ("mb_create_slab", C.c_int, [C.POINTER(_P), C.POINTER(C.c_int), C.c_int, C.c_int, C.c_double,
                                 C.c_double, C.POINTER(mb_params), _P]),
    ("mb_slab_info", C.c_int, [_P, C.POINTER(C.c_int)]),
    ("mb_halo_bytes", C.c_int, [_P, C.POINTER(C.c_size_t)]),
    ("mb_halo_pack", C.c_int, [_P, C.c_int, _P]),
    ("mb_halo_unpack", C.c_int, [_P, C.c_int, _P]),
    ("mb_set_material", C.c_int, [_P, _P, _P, C.c_double, C.c_double]),
    ("mb_set_seed", C.c_int, [_P, C.c_uint64]),
    ("mb_add_point_probe", C.c_int, [_P, C.POINTER(C.c_int), C.c_int, C.c_double, C.c_double,
                                     C.POINTER(C.c_int)]),
    ("mb_add_face_probes", C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double]),
    ("mb_set_source", C.c_int, [_P, C.POINTER(C.c_int), C.c_int, C.c_double, C.c_double,
                                C.c_double, C.c_double]),
    ("mb_set_source_cw", C.c_int, [_P, C.POINTER(C.c_int), C.c_int, C.c_double, C.c_double,
                                   C.c_double, C.c_double, C.c_int]),
    ("mb_add_plane_probe", C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                     C.POINTER(C.c_int)]),
    ("mb_plane_mode_map", C.c_int, [_P, C.c_int, C.c_int, _P]),
    ("mb_plane_energy_density", C.c_int, [_P, C.c_int, _P]),
    ("mb_step", C.c_int, [_P, C.c_int]),
    ("mb_step_timed", C.c_int, [_P, C.c_int, _P]),
    ("mb_flux", C.c_int, [_P, _P]),
    ("mb_synchronize", C.c_int, [_P]),
    ("mb_join_probes", C.c_int, [_P]),
    ("mb_reset_probes", C.c_int, [_P]),
    ("mb_get_step", C.c_int, [_P, C.POINTER(C.c_int64)]),
    ("mb_probe_spectrum", C.c_int, [_P, C.c_int, _P, _P]),
    ("mb_face_spectrum", C.c_int, [_P, C.c_int, _P, _P]),
    ("mb_energy", C.c_int, [_P, C.POINTER(C.c_double), _P]),
    ("mb_get_field", C.c_int, [_P, C.c_int, _P]),
    ("mb_get_cpml", C.c_int, [_P, C.c_int, _P, C.POINTER(C.c_size_t)]),
    ("mb_gain_list", C.c_int, [_P, _P, C.POINTER(C.c_int64)]),
    ("mb_get_material", C.c_int, [_P, _P]),
    ("mb_set_field", C.c_int, [_P, C.c_int, _P]),
    ("mb_get_field_device", C.c_int, [_P, C.c_int, _P, C.POINTER(C.c_double)]),
    ("mb_save_state", C.c_int, [_P, _P, C.POINTER(C.c_size_t)]),
    ("mb_load_state", C.c_int, [_P, _P, C.c_size_t]),
    ("mb_autotune", C.c_int, [_P]),
    ("mb_get_tuning", C.c_int, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    ("mb_set_tuning", C.c_int, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    ("mb_flux_async", C.c_int, [_P, _P]),
    ("mb_debug_fail_alloc", None, [C.c_int]),
    ("mb_get_single_pass", C.c_int, [_P, C.POINTER(C.c_int)]),
    ("mb_set_single_pass", C.c_int, [_P, C.POINTER(C.c_int)]),
    ("mb_launch_stats", C.c_int, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int64)]),
    ("mb_device_bytes", C.c_int, [_P, C.POINTER(C.c_size_t)]),
    ("mb_philox4x32_10", C.c_int, [_P, _P, _P, C.c_int]),
    ("mb_host_tables", C.c_int, [_P, C.c_double, C.c_double, _P, C.c_double, C.c_double, _P, _P,
                                 C.POINTER(C.c_double)]),
    ("mb_material_map", C.c_int, [_P, _P, C.c_int64, C.c_int, C.c_int, _P, _P, C.POINTER(C.c_int64),
                                  _P, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    ("mb_energy_sum_noalloc", C.c_int, [_P, _P, _P, _P, _P, _P, _P, C.c_int64, _P, _P]),
    ("mb_batch_create", C.c_int, [C.POINTER(_P), C.c_int, C.POINTER(C.c_int), C.c_double,
                                  C.c_double, C.POINTER(mb_params), _P]),
    ("mb_batch_destroy", C.c_int, [_P]),
    ("mb_batch_set_instance", C.c_int, [_P, C.c_int, _P, _P, C.c_double, C.c_double,
                                        C.c_uint64]),
    ("mb_batch_instance", C.c_int, [_P, C.c_int, C.POINTER(_P)]),
    ("mb_batch_step", C.c_int, [_P, C.c_int]),
    ("mb_batch_synchronize", C.c_int, [_P]),
    ("mb_batch_autotune", C.c_int, [_P]),
    ("mb_batch_get_tuning", C.c_int, [_P, C.POINTER(C.c_int)]),
    ("mb_batch_set_mode", C.c_int, [_P, C.c_int]),
    ("mb_batch_get_mode", C.c_int, [_P, C.POINTER(C.c_int)]),
    ("mb_gp_features", C.c_int, [_P, C.c_int, C.c_int, _P, _P, _P]),
    ("mb_selftest_bounded_waits", C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_int)]),
    ("mb_adjoint_energy_zface", C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P,
                                          C.POINTER(C.c_double), C.POINTER(C.c_double)]),
]

_lib = None


def load_library(path: str | None = None):
    """Load ``libmbfdtd.so`` (raises MBLibraryError when it is absent)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise MBLibraryError(f"{p} not found: build it with paper_0809_1547_gb300.build.build()")
    try:
        lib = C.CDLL(p)
    except OSError as e:
        raise MBLibraryError(f"cannot load {p}: {e}") from e
    for name, res, args in _SIGS:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def exported_names():
    return [s[0] for s in _SIGS]


def _check(code, ctx=None):
    if code != MB_OK:
        lib = load_library()
        msg = lib.mb_last_error(ctx)
        raise MBError(code, msg.decode() if msg else "")


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def mb_default_params(**overrides) -> mb_params:
    p = mb_params()
    load_library().mb_default_params(C.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def mb_create(grid, dx, dt, params: mb_params | None = None, stream: int | None = None):
    lib = load_library()
    h = C.c_void_p()
    g = (C.c_int * 3)(*[int(v) for v in grid])
    _check(lib.mb_create(C.byref(h), g, float(dx), float(dt),
                         C.byref(params) if params is not None else None,
                         C.c_void_p(stream) if stream else None))
    return h


def mb_destroy(h):
    if h:
        _check(load_library().mb_destroy(h))


def mb_create_slab(grid, z_begin, z_end, dx, dt, params: mb_params | None = None,
                   stream: int | None = None):
    lib = load_library()
    h = C.c_void_p()
    g = (C.c_int * 3)(*[int(v) for v in grid])
    _check(lib.mb_create_slab(C.byref(h), g, int(z_begin), int(z_end), float(dx), float(dt),
                              C.byref(params) if params is not None else None,
                              C.c_void_p(stream) if stream else None))
    return h


def mb_slab_info(h):
    """(whole grid's n_z, whole-grid plane of local plane 0, first own local
    plane, one past the last own local plane)."""
    out = (C.c_int * 4)()
    _check(load_library().mb_slab_info(h, out), h)
    return tuple(out)


def mb_halo_bytes(h) -> int:
    b = C.c_size_t()
    _check(load_library().mb_halo_bytes(h, C.byref(b)), h)
    return b.value


def mb_halo_pack(h, side: int, dev_ptr: int):
    _check(load_library().mb_halo_pack(h, int(side), C.c_void_p(dev_ptr)), h)


def mb_halo_unpack(h, side: int, dev_ptr: int):
    _check(load_library().mb_halo_unpack(h, int(side), C.c_void_p(dev_ptr)), h)


def mb_set_material(h, eps_map, gain_mask, N_a, pump):
    eps = np.ascontiguousarray(eps_map, dtype=np.float32)
    gm = np.ascontiguousarray(gain_mask, dtype=np.uint8)
    _check(load_library().mb_set_material(h, _ptr(eps), _ptr(gm), float(N_a), float(pump)), h)


def mb_set_seed(h, seed):
    _check(load_library().mb_set_seed(h, C.c_uint64(int(seed) & 0xFFFFFFFFFFFFFFFF)), h)


def mb_add_point_probe(h, ijk, n_freq, lam_min, lam_max) -> int:
    pid = C.c_int()
    _check(load_library().mb_add_point_probe(h, (C.c_int * 3)(*ijk), int(n_freq), float(lam_min),
                                             float(lam_max), C.byref(pid)), h)
    return pid.value


def mb_add_face_probes(h, stride, every, n_freq, lam_min, lam_max):
    _check(load_library().mb_add_face_probes(h, int(stride), int(every), int(n_freq),
                                             float(lam_min), float(lam_max)), h)


def mb_set_source(h, ijk, comp, lam, t0, tau, amp):
    _check(load_library().mb_set_source(h, (C.c_int * 3)(*ijk), int(comp), float(lam), float(t0),
                                        float(tau), float(amp)), h)


def mb_set_source_cw(h, ijk, comp, lam, t0, tau, amp, n_steps):
    _check(load_library().mb_set_source_cw(h, (C.c_int * 3)(*ijk), int(comp), float(lam), float(t0),
                                           float(tau), float(amp), int(n_steps)), h)


def mb_add_plane_probe(h, k, every, n_freq, lam_min, lam_max) -> int:
    pid = C.c_int()
    _check(load_library().mb_add_plane_probe(h, int(k), int(every), int(n_freq), float(lam_min),
                                             float(lam_max), C.byref(pid)), h)
    return pid.value


def mb_plane_mode_map(h, probe_id, bin_, shape):
    out = np.zeros(int(np.prod(shape)))
    _check(load_library().mb_plane_mode_map(h, int(probe_id), int(bin_), _ptr(out)), h)
    return out.reshape(shape)


def mb_plane_energy_density(h, k, shape):
    out = np.zeros(int(np.prod(shape)))
    _check(load_library().mb_plane_energy_density(h, int(k), _ptr(out)), h)
    return out.reshape(shape)


def mb_step(h, n):
    _check(load_library().mb_step(h, int(n)), h)


def mb_step_timed(h, n):
    """Advance n steps with per-pass CUDA-event timing: returns ms summed per
    pass (H, E, point DFT, face DFT)."""
    ms = np.zeros(4)
    _check(load_library().mb_step_timed(h, int(n), _ptr(ms)), h)
    return ms


def mb_flux(h):
    fl = np.zeros(6)
    _check(load_library().mb_flux(h, _ptr(fl)), h)
    return fl


def mb_flux_async(h, out_ptr: int):
    """Queue the read of the six face energies into the 6-double host buffer
    at out_ptr (pinned memory); valid once the stream has passed this call."""
    _check(load_library().mb_flux_async(h, C.c_void_p(out_ptr)), h)


def mb_debug_fail_alloc(n: int):
    """Test hook: make the n-th device allocation from now on fail (n < 0: off)."""
    load_library().mb_debug_fail_alloc(int(n))


def mb_host_tables(grid, dx, dt, params: mb_params | None = None, N_a=0.0, pump=0.0):
    """Host-only diagnostic: ({axis: (bE, cE, bH, cH)}, gain coefficients
    dict, E0) exactly as a context with these arguments steps with them."""
    g = (C.c_int * 3)(*[int(v) for v in grid])
    cp = np.empty(4 * sum(int(v) for v in grid), np.float32)
    gn = np.empty(20, np.float32)
    E0 = C.c_double()
    _check(load_library().mb_host_tables(g, float(dx), float(dt), C.byref(params) if params else None,
                                         float(N_a), float(pump), _ptr(cp), _ptr(gn), C.byref(E0)))
    out, o = {}, 0
    for w, n in zip("xyz", grid):
        n = int(n)
        out[w] = tuple(cp[o + q * n:o + (q + 1) * n].copy() for q in range(4))
        o += 4 * n
    gain = {"cJ1": gn[0], "cJE": gn[1], "cJP": gn[2], "cJN": gn[3], "nfloor": gn[4], "g": gn[5:8].copy(),
            "G": gn[8:17].reshape(3, 3).copy(), "mk": gn[17:20].copy()}
    return out, gain, E0.value


def mb_material_map(eps_map, gain_mask, gain_on=True, max_threads=16):
    """Host-only diagnostic: (material bytes, gain-cell indices, distinct
    eps_r values in id order, dense flag) as mb_set_material builds them."""
    eps = np.ascontiguousarray(eps_map, dtype=np.float32).reshape(-1)
    gm = np.ascontiguousarray(gain_mask, dtype=np.uint8).reshape(-1)
    if eps.size != gm.size or eps.size < 1:
        raise ValueError("eps_map and gain_mask must have the same, non-zero size")
    mat = np.empty(eps.size, np.uint8)
    glist = np.empty(eps.size, np.uint32)
    lut = np.empty(128, np.float32)
    ng, nv, dense = C.c_int64(), C.c_int(), C.c_int()
    _check(load_library().mb_material_map(_ptr(eps), _ptr(gm), eps.size, int(bool(gain_on)),
                                          int(max_threads), _ptr(mat), _ptr(glist), C.byref(ng),
                                          _ptr(lut), C.byref(nv), C.byref(dense)))
    return mat, glist[:ng.value].copy(), lut[:nv.value].copy(), bool(dense.value)


def mb_synchronize(h):
    _check(load_library().mb_synchronize(h), h)


def mb_join_probes(h):
    """Order the context's stream after probe launches mb_step left running
    on its second stream (no host wait)."""
    _check(load_library().mb_join_probes(h), h)


def mb_reset_probes(h):
    """Zero every probe's running DFT sums: later spectra cover the steps
    taken after this call (a time window)."""
    _check(load_library().mb_reset_probes(h), h)


def mb_get_step(h) -> int:
    n = C.c_int64()
    _check(load_library().mb_get_step(h, C.byref(n)), h)
    return n.value


def mb_probe_spectrum(h, probe_id, n_freq):
    S = np.zeros(n_freq)
    lam = np.zeros(n_freq)
    _check(load_library().mb_probe_spectrum(h, int(probe_id), _ptr(S), _ptr(lam)), h)
    return S, lam


def mb_face_spectrum(h, face, n_freq):
    S = np.zeros(n_freq)
    lam = np.zeros(n_freq)
    _check(load_library().mb_face_spectrum(h, int(face), _ptr(S), _ptr(lam)), h)
    return S, lam


def mb_energy(h):
    U = C.c_double()
    fl = np.zeros(6)
    _check(load_library().mb_energy(h, C.byref(U), _ptr(fl)), h)
    return U.value, fl


def mb_gain_list(h):
    """The context's gain-cell list (uint32 cell indices, increasing)."""
    lib = load_library()
    n = C.c_int64()
    _check(lib.mb_gain_list(h, None, C.byref(n)), h)
    out = np.zeros(n.value, dtype=np.uint32)
    if n.value:
        _check(lib.mb_gain_list(h, _ptr(out), C.byref(n)), h)
    return out


def mb_get_material(h, shape):
    """The context's material bytes [k, j, i] (uint8; bit 7: gain cell)."""
    out = np.zeros(int(np.prod(shape)), dtype=np.uint8)
    _check(load_library().mb_get_material(h, _ptr(out)), h)
    return out.reshape(shape)


def mb_get_cpml(h, axis: int):
    """CPML memories of the slabs along `axis` (SI, FP64), shaped (4, ...) by
    the layout of mb_get_cpml: x (4, n_z, n_y, 2L), y (4, n_z, 2L, n_x),
    z (4, zn, n_y, n_x); None without CPML."""
    lib = load_library()
    n = C.c_size_t()
    _check(lib.mb_get_cpml(h, int(axis), None, C.byref(n)), h)
    if n.value == 0:
        return None
    out = np.zeros(n.value, dtype=np.float64)
    _check(lib.mb_get_cpml(h, int(axis), _ptr(out), C.byref(n)), h)
    return out


def mb_get_field(h, which, shape):
    out = np.zeros(int(np.prod(shape)), dtype=np.float32)
    wid = FIELD_ID[which] if isinstance(which, str) else int(which)
    _check(load_library().mb_get_field(h, wid, _ptr(out)), h)
    return out.reshape(shape)


def mb_set_field(h, which, values):
    v = np.ascontiguousarray(values, dtype=np.float32)
    wid = FIELD_ID[which] if isinstance(which, str) else int(which)
    _check(load_library().mb_set_field(h, wid, _ptr(v)), h)


def mb_get_field_device(h, which, dev_ptr: int) -> float:
    scale = C.c_double()
    wid = FIELD_ID[which] if isinstance(which, str) else int(which)
    _check(load_library().mb_get_field_device(h, wid, C.c_void_p(dev_ptr), C.byref(scale)), h)
    return scale.value


def mb_save_state(h) -> bytes:
    lib = load_library()
    n = C.c_size_t()
    _check(lib.mb_save_state(h, None, C.byref(n)), h)
    buf = (C.c_char * n.value)()
    _check(lib.mb_save_state(h, buf, C.byref(n)), h)
    return bytes(buf)


def mb_load_state(h, blob: bytes):
    buf = C.create_string_buffer(blob, len(blob))
    _check(load_library().mb_load_state(h, buf, len(blob)), h)


def mb_autotune(h):
    _check(load_library().mb_autotune(h), h)


def mb_get_tuning(h):
    """((variant, bx, by, bz), (variant, bx, by, bz)) of the H and E passes."""
    bh = (C.c_int * 4)()
    be = (C.c_int * 4)()
    _check(load_library().mb_get_tuning(h, bh, be), h)
    return tuple(bh), tuple(be)


def mb_set_tuning(h, tune_h, tune_e):
    _check(load_library().mb_set_tuning(h, (C.c_int * 4)(*tune_h), (C.c_int * 4)(*tune_e)), h)


def mb_get_single_pass(h):
    """(on, bx, by, kz) of the single-pass step."""
    t = (C.c_int * 4)()
    _check(load_library().mb_get_single_pass(h, t), h)
    return tuple(t)


def mb_set_single_pass(h, tune):
    _check(load_library().mb_set_single_pass(h, (C.c_int * 4)(*tune)), h)


def mb_launch_stats(h):
    per = C.c_int()
    tot = C.c_int64()
    _check(load_library().mb_launch_stats(h, C.byref(per), C.byref(tot)), h)
    return per.value, tot.value


def mb_device_bytes(h) -> int:
    n = C.c_size_t()
    _check(load_library().mb_device_bytes(h, C.byref(n)), h)
    return n.value


def mb_philox4x32_10(ctr, key):
    """Device Philox4x32-10 on counters ctr (n, 4) uint32 with key (2,): returns (n, 4)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, dtype=np.uint32).reshape(2)
    out = np.zeros_like(c)
    _check(load_library().mb_philox4x32_10(_ptr(c), _ptr(k), _ptr(out), c.shape[0]))
    return out


def mb_energy_sum_noalloc(ex, ey, ez, hx, hy, hz, eps_r, ncell, out, stream=0):
    """Energy sum from caller-owned device arrays without any allocation (see
    include/mb_fdtd.h); arguments are device addresses (ints), eps_r may be 0."""
    _check(load_library().mb_energy_sum_noalloc(
        C.c_void_p(ex), C.c_void_p(ey), C.c_void_p(ez), C.c_void_p(hx), C.c_void_p(hy),
        C.c_void_p(hz), C.c_void_p(eps_r) if eps_r else None, int(ncell), C.c_void_p(out),
        C.c_void_p(stream) if stream else None))


def mb_batch_create(grids, dx, dt, params: mb_params | None = None, stream: int | None = None):
    lib = load_library()
    h = C.c_void_p()
    flat = [int(v) for g in grids for v in g]
    g = (C.c_int * len(flat))(*flat)
    _check(lib.mb_batch_create(C.byref(h), len(grids), g, float(dx), float(dt),
                               C.byref(params) if params is not None else None,
                               C.c_void_p(stream) if stream else None))
    return h


def mb_batch_destroy(h):
    if h:
        _check(load_library().mb_batch_destroy(h))


def mb_batch_set_instance(h, b, eps_map, gain_mask, N_a, pump, seed):
    eps = np.ascontiguousarray(eps_map, dtype=np.float32)
    gm = np.ascontiguousarray(gain_mask, dtype=np.uint8)
    _check(load_library().mb_batch_set_instance(h, int(b), _ptr(eps), _ptr(gm), float(N_a),
                                                float(pump),
                                                C.c_uint64(int(seed) & 0xFFFFFFFFFFFFFFFF)))


def mb_batch_instance(h, b):
    ctx = C.c_void_p()
    _check(load_library().mb_batch_instance(h, int(b), C.byref(ctx)))
    return ctx


def mb_batch_step(h, n):
    _check(load_library().mb_batch_step(h, int(n)))


def mb_batch_synchronize(h):
    _check(load_library().mb_batch_synchronize(h))


def mb_batch_autotune(h):
    _check(load_library().mb_batch_autotune(h))


def mb_batch_get_tuning(h):
    """(bx, by, kz) of the persistent kernel."""
    t = (C.c_int * 3)()
    _check(load_library().mb_batch_get_tuning(h, t))
    return tuple(t)


def mb_batch_set_mode(h, mode: int):
    """MB_BATCH_PERSISTENT (one persistent launch per step call) or
    MB_BATCH_CONCURRENT (the members' own launches on concurrent streams)."""
    _check(load_library().mb_batch_set_mode(h, int(mode)))


def mb_batch_get_mode(h) -> int:
    m = C.c_int()
    _check(load_library().mb_batch_get_mode(h, C.byref(m)))
    return int(m.value)


def mb_adjoint_energy_zface(h, n_steps, ckpt_every=200, z_plane=-1, d_grad_eps: int = 0):
    """(J, dJ/dW_p); dJ/deps_r written to the device array at d_grad_eps (if non-zero)."""
    gp = C.c_double()
    J = C.c_double()
    _check(load_library().mb_adjoint_energy_zface(h, int(n_steps), int(ckpt_every), int(z_plane),
                                                  C.c_void_p(d_grad_eps) if d_grad_eps else None,
                                                  C.byref(gp), C.byref(J)), h)
    return J.value, gp.value


def mb_selftest_bounded_waits(which, limit=4096):
    """Blocks whose bounded wait gave up on an event that never comes
    (which 0: grid barrier, 1: mbarrier)."""
    n = C.c_int()
    _check(load_library().mb_selftest_bounded_waits(int(which), int(limit), C.byref(n)))
    return n.value


def mb_gp_features(E, n_grid=2047, want_phi=False):
    """(w_phi, p_phi[, phi]) of the bound states for the eigenvalues E (> 1)."""
    Ev = np.ascontiguousarray(np.atleast_1d(E), dtype=np.float64)
    w = np.zeros(len(Ev))
    p = np.zeros(len(Ev))
    phi = np.zeros((len(Ev), int(n_grid))) if want_phi else None
    _check(load_library().mb_gp_features(_ptr(Ev), len(Ev), int(n_grid), _ptr(w), _ptr(p),
                                         _ptr(phi) if want_phi else None))
    return (w, p, phi) if want_phi else (w, p)


class MBSimulation:
    """One Maxwell–Bloch FDTD realization on the GPU (owns one C context).

    ``grid`` is (n_x, n_y, n_z); host arrays passed to it are indexed
    [k, j, i] (x fastest), like the fields it returns.
    """

    def __init__(self, grid, dx, dt, params: mb_params | None = None, stream=None, _handle=None):
        self.grid = tuple(int(v) for v in grid)
        self.shape = self.grid[::-1]
        self.dx, self.dt = float(dx), float(dt)
        self.probe_nfreq = {}
        self.face_nfreq = 0
        self._owned = _handle is None
        if _handle is not None:   # a context owned by an MBBatch
            self._h = _handle
            return
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream().cuda_stream or None
            except Exception:
                stream = None
        self._h = mb_create(self.grid, dx, dt, params, stream)

    def close(self):
        if getattr(self, "_h", None):
            if self._owned:
                mb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    def set_material(self, eps_r, gain_mask, N_a, pump):
        mb_set_material(self._h, np.asarray(eps_r).reshape(-1), np.asarray(gain_mask).reshape(-1),
                        N_a, pump)

    def set_seed(self, seed):
        mb_set_seed(self._h, seed)

    def add_point_probe(self, ijk, n_freq, lam_min, lam_max):
        pid = mb_add_point_probe(self._h, ijk, n_freq, lam_min, lam_max)
        self.probe_nfreq[pid] = int(n_freq)
        return pid

    def add_face_probes(self, stride, every, n_freq, lam_min, lam_max):
        mb_add_face_probes(self._h, stride, every, n_freq, lam_min, lam_max)
        self.face_nfreq = int(n_freq)

    def set_source(self, ijk, comp, lam, t0, tau, amp):
        mb_set_source(self._h, ijk, comp, lam, t0, tau, amp)

    def set_source_cw(self, ijk, comp, lam, t0, tau, amp, n_steps):
        mb_set_source_cw(self._h, ijk, comp, lam, t0, tau, amp, n_steps)

    def add_plane_probe(self, k, every, n_freq, lam_min, lam_max):
        return mb_add_plane_probe(self._h, k, every, n_freq, lam_min, lam_max)

    def plane_mode_map(self, probe_id, bin_):
        """(n_y, n_x) mode map of a plane probe at one frequency bin."""
        return mb_plane_mode_map(self._h, probe_id, bin_, self.shape[1:])

    def plane_energy_density(self, k):
        """(n_y, n_x) energy density (J/m^3) of the plane z = k."""
        return mb_plane_energy_density(self._h, k, self.shape[1:])

    def step(self, n=1):
        mb_step(self._h, n)

    def step_timed(self, n):
        return mb_step_timed(self._h, n)

    def flux(self):
        return mb_flux(self._h)

    def flux_async(self, out):
        """Queue the read of the six face energies (J) into `out`, a pinned
        torch CPU tensor of 6 float64 (complete once the simulation's stream
        passes this point, e.g. after an event recorded on it)."""
        import torch
        if not (isinstance(out, torch.Tensor) and out.dtype == torch.float64 and out.numel() >= 6
                and out.device.type == "cpu" and out.is_contiguous()):
            raise ValueError("out must be a contiguous CPU float64 tensor of 6 values")
        mb_flux_async(self._h, out.data_ptr())

    def synchronize(self):
        mb_synchronize(self._h)

    def join_probes(self):
        """Make the simulation's stream wait for the probe DFTs that step()
        left running beside later steps (enqueued only)."""
        mb_join_probes(self._h)

    def reset_probes(self):
        """Start the probes' spectra afresh: they cover the steps taken from
        here on (mb_reset_probes)."""
        mb_reset_probes(self._h)

    @property
    def n(self):
        return mb_get_step(self._h)

    def probe_spectrum(self, probe_id):
        return mb_probe_spectrum(self._h, probe_id, self.probe_nfreq[probe_id])

    def face_spectrum(self, face):
        return mb_face_spectrum(self._h, face, self.face_nfreq)

    def energy(self):
        return mb_energy(self._h)

    def field(self, name):
        return mb_get_field(self._h, name, self.shape)

    def gain_list(self):
        """The gain cells the two-pass step's Lorentz blocks run over."""
        return mb_gain_list(self._h)

    def material(self):
        """The material bytes [k, j, i] mb_set_material built on the device."""
        return mb_get_material(self._h, self.grid[::-1])

    def cpml(self, axis: int):
        """CPML memories along `axis` (SI), shaped (4, ...) as in mb_get_cpml:
        x (4, n_z, n_y, 2L), y (4, n_z, 2L, n_x), z (4, zn, n_y, n_x)."""
        v = mb_get_cpml(self._h, axis)
        if v is None:
            return None
        nx, ny, nz = self.grid
        per = v.size // 4
        if axis == 0:
            return v.reshape(4, nz, ny, per // (nz * ny))
        if axis == 1:
            return v.reshape(4, nz, per // (nz * nx), nx)
        return v.reshape(4, per // (ny * nx), ny, nx)

    def set_field(self, name, values):
        mb_set_field(self._h, name, np.asarray(values).reshape(-1))

    def field_device(self, name):
        """(tensor, scale): the field copied into a torch CUDA tensor in the
        device's scaled units, and the factor that turns it into SI."""
        import torch
        t = torch.empty(self.shape, dtype=torch.float32, device="cuda")
        scale = mb_get_field_device(self._h, name, t.data_ptr())
        return t, scale

    def save_state(self) -> bytes:
        return mb_save_state(self._h)

    def load_state(self, blob: bytes):
        mb_load_state(self._h, blob)

    def autotune(self):
        mb_autotune(self._h)

    def launch_stats(self):
        return mb_launch_stats(self._h)

    def tuning(self):
        return mb_get_tuning(self._h)

    def set_tuning(self, tune_h, tune_e):
        mb_set_tuning(self._h, tune_h, tune_e)

    def single_pass(self):
        """(on, bx, by, kz) of the single-pass step."""
        return mb_get_single_pass(self._h)

    def set_single_pass(self, tune):
        """tune = (on, bx, by, kz); on = 0 returns to the two passes."""
        mb_set_single_pass(self._h, tune)

    def device_bytes(self):
        return mb_device_bytes(self._h)

    def adjoint_energy_zface(self, n_steps, ckpt_every=200, z_plane=-1):
        """Advance n_steps; return (J, grad_eps as a torch CUDA tensor shaped
        like the grid [k, j, i], dJ/dW_p)."""
        import torch
        g = torch.empty(self.shape, dtype=torch.float32, device="cuda")
        J, gp = mb_adjoint_energy_zface(self._h, n_steps, ckpt_every, z_plane, g.data_ptr())
        return J, g, gp


class MBBatch:
    """An ensemble of realizations on grids of any sizes, advanced together by
    one persistent launch per :meth:`step`, or by the members' own launches
    on concurrent streams (:meth:`set_mode`; :meth:`autotune` keeps the
    faster) (``mb_batch_*`` in the C ABI).
    ``instances[b]`` is an :class:`MBSimulation` view of member b: set its
    probes and sources and read it out as usual, but step it only through the
    batch."""

    def __init__(self, grids, dx, dt, params: mb_params | None = None, stream=None):
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream().cuda_stream or None
            except Exception:
                stream = None
        self.grids = [tuple(int(v) for v in g) for g in grids]
        self._h = mb_batch_create(self.grids, dx, dt, params, stream)
        self.instances = [MBSimulation(g, dx, dt, _handle=mb_batch_instance(self._h, b))
                          for b, g in enumerate(self.grids)]

    def __len__(self):
        return len(self.instances)

    def close(self):
        if getattr(self, "_h", None):
            for s in self.instances:
                s.close()
            mb_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_instance(self, b, eps_r, gain_mask, N_a, pump, seed):
        mb_batch_set_instance(self._h, b, np.asarray(eps_r).reshape(-1),
                              np.asarray(gain_mask).reshape(-1), N_a, pump, seed)

    def step(self, n=1):
        mb_batch_step(self._h, n)

    def synchronize(self):
        mb_batch_synchronize(self._h)

    def autotune(self):
        mb_batch_autotune(self._h)

    def tuning(self):
        return mb_batch_get_tuning(self._h)

    @property
    def mode(self):
        return mb_batch_get_mode(self._h)

    def set_mode(self, mode):
        mb_batch_set_mode(self._h, mode)

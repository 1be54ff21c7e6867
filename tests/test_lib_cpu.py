"""Host-side checks of the C ABI that need no GPU: build, load, exports, argument validation."""
import ctypes as C
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_0809_1547_gb300 import build
    from paper_0809_1547_gb300.binding import load_library
    build.build()
    return load_library()


def _declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(inc, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(mb_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("mb_create", "mb_set_material", "mb_step", "mb_probe_spectrum", "mb_energy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_0809_1547_gb300.binding import exported_names
    declared = _declared_functions()
    for name in declared:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    assert declared <= set(exported_names()) | {"mb_default_params"}


def test_default_params_agree_with_the_oracle(lib):
    from paper_0809_1547_gb300.binding import mb_default_params
    from oracle.mb_oracle import Params
    p = mb_default_params()
    o = Params()
    for f in ("lambda0", "dlambda", "tau32", "tau21", "tau10", "a_se", "dipole_len", "n_floor_rel",
              "npml", "pml_order", "pml_sigma_factor", "pml_alpha_rel"):
        assert getattr(p, f) == getattr(o, f), f


def test_argument_validation_without_gpu(lib):
    from paper_0809_1547_gb300.binding import MB_ERR_ARG, MB_ERR_COURANT
    h = C.c_void_p()
    dx = 20e-9
    dt_ok = 0.99 * dx / (299792458.0 * math.sqrt(3.0))
    assert lib.mb_create(C.byref(h), (C.c_int * 3)(0, 4, 4), dx, dt_ok, None, None) == MB_ERR_ARG
    assert lib.mb_create(C.byref(h), (C.c_int * 3)(4, 4, 4), dx, 1.01 * dt_ok / 0.99, None, None) == MB_ERR_COURANT
    assert lib.mb_create(C.byref(h), (C.c_int * 3)(4, 4, 4), -dx, dt_ok, None, None) == MB_ERR_ARG
    assert lib.mb_create(None, (C.c_int * 3)(4, 4, 4), dx, dt_ok, None, None) == MB_ERR_ARG
    assert h.value is None
    assert b"Courant" in lib.mb_last_error(None) or b"null" in lib.mb_last_error(None)
    assert lib.mb_step(None, 1) == MB_ERR_ARG
    assert lib.mb_destroy(None) == 0


def test_create_without_a_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_0809_1547_gb300.binding import MB_ERR_CUDA, MB_ERR_OOM
    h = C.c_void_p()
    dx = 20e-9
    dt = 0.99 * dx / (299792458.0 * math.sqrt(3.0))
    rc = lib.mb_create(C.byref(h), (C.c_int * 3)(4, 4, 4), dx, dt, None, None)
    assert rc in (MB_ERR_CUDA, MB_ERR_OOM)
    assert h.value is None


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_0809_1547_gb300.binding import load_library, MBLibraryError
    with pytest.raises(MBLibraryError):
        load_library(str(tmp_path / "missing.so"))

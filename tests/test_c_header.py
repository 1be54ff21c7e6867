"""The boundary header is plain C: a C99 translation unit that includes it
and calls its entry points compiles warning-free with gcc, and links against
the library (CPU; nothing runs)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SOURCE = r"""
#include <stdint.h>
#include <stdio.h>
#include "mb_fdtd.h"

int run(void) {
    mb_params p;
    mb_ctx* ctx = NULL;
    const int grid[3] = {64, 48, 40};
    const int probe[3] = {32, 24, 20};
    int pid = -1;
    double S[16], lam[16], U = 0.0, flux[6];
    mb_default_params(&p);
    if (mb_create(&ctx, grid, 20e-9, 3.8e-17, &p, NULL) != MB_OK) {
        printf("%s\n", mb_last_error(NULL));
        return 1;
    }
    if (mb_add_point_probe(ctx, probe, 16, 475e-9, 705e-9, &pid) != MB_OK ||
        mb_step(ctx, 10) != MB_OK || mb_probe_spectrum(ctx, pid, S, lam) != MB_OK ||
        mb_energy(ctx, &U, flux) != MB_OK) {
        printf("%s\n", mb_last_error(ctx));
        mb_destroy(ctx);
        return 1;
    }
    mb_destroy(ctx);
    return 0;
}
"""


def test_header_compiles_as_c99_and_links(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    src = tmp_path / "use.c"
    src.write_text(SOURCE)
    obj = tmp_path / "use.o"
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-c",
                        "-I", os.path.join(ROOT, "include"), str(src), "-o", str(obj)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lib_dir = os.path.join(ROOT, "paper_0809_1547_gb300")
    if not os.path.exists(os.path.join(lib_dir, "libmbfdtd.so")):
        pytest.skip("library not built")
    so = tmp_path / "libuse.so"
    r = subprocess.run([gcc, "-shared", str(obj), "-o", str(so), "-L", lib_dir, "-lmbfdtd"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr

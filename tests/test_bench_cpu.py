"""Host-side pieces of the benchmark (CPU): the per-cell byte counts the
roofline divides by, and the reading of the committed ncu summaries."""
import json
import os

import numpy as np
import pytest

import bench
from paper_0809_1547_gb300 import inputs


class _W:
    def __init__(self, grid, npml, gain_frac, N_a=1.0):
        self.grid = grid
        self.npml = npml
        self.N_a = N_a
        rng = np.random.default_rng(0)
        self.gain = (rng.random(grid[::-1]) < gain_frac).astype(np.uint8)


def test_byte_counts_reduce_to_the_stencil_minimum():
    w = _W((16, 16, 16), 0, 0.0)
    ab = bench.algorithmic_bytes(w)
    assert ab["single_pass_launch"] == 49.0          # E, H read + write, material byte
    assert ab["step_two_pass_minimum"] == 73.0       # E, H read twice over two passes
    assert ab["step_reference"] == 73.0
    assert ab["h_launch"] + ab["e_launch"] == 73.0


def test_byte_counts_grow_with_gain_and_cpml():
    w = _W((40, 40, 40), 4, 0.5)
    ab = bench.algorithmic_bytes(w)
    g, f = ab["gain_fraction"], ab["slab_fraction_sum"]
    assert f == pytest.approx(3 * 8 / 40)
    assert 0.45 < g < 0.55
    assert ab["single_pass_launch"] == pytest.approx(49 + 32 * f + 72 * g)
    assert ab["step_reference"] == pytest.approx(73 + 64 * f + 80 * g)
    # the single pass saves exactly one read of E and H (24 B/cell)
    assert ab["step_two_pass_minimum"] - ab["single_pass_launch"] == pytest.approx(24.0)
    # gain off: no gain bytes
    assert bench.algorithmic_bytes(_W((40, 40, 40), 4, 0.5, N_a=0.0))["gain_fraction"] == 0.0


def test_committed_traffic_summary_is_read_only_for_matching_sources():
    summary = os.path.join(bench.PROFILE_DIR, "k_step_fused_traffic_mb320_active.md")
    text = open(summary).read()
    assert "kernel_source_hash:" in text and "bytes_per_launch_full_size:" in text
    value = bench.traffic_from_profile("k_step_fused")
    recorded = text.split("kernel_source_hash:")[1].split()[0]
    stated = float(text.split("bytes_per_launch_full_size:")[1].split()[0])
    # a full 320^3 launch moves between 100 and 130 B per cell
    assert 100 * 320 ** 3 < stated < 130 * 320 ** 3
    if recorded == bench.kernel_source_hash():
        assert value == pytest.approx(stated, rel=1e-6, abs=0)
    else:
        assert value is None
    assert bench.traffic_from_profile("no_such_kernel") is None


def test_paper_workload_byte_count_at_320():
    w = inputs.workload_paper_320()
    ab = bench.algorithmic_bytes(w)
    assert ab["single_pass_launch"] == pytest.approx(85.3, abs=0.5)
    assert ab["step_reference"] == pytest.approx(117.6, abs=0.5)


def test_reference_arm_prints_one_valid_line():
    """`bench.py --impl reference` (the oracle timed on the host cores, the
    arm run beside ours) prints one JSON line with our metric, unit and
    direction, impl = reference, its cpu_baseline and an e2e without copies."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3", "--ref-budget", "8", "--ref-cores", "2"],
                       capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and "unavailable" not in d
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] >= 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}

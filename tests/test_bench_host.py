"""Host logic of bench.py (no GPU): the per-kernel byte model behind the
roofline figure, and the reference arm's JSON line."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _info(sizes, t=8, a=(2, 2, 2)):
    return {"t": t, "a": list(a), "sizes": sizes}


def test_byte_model_of_the_256_workload():
    """2x2x2 subdomains of 128^3, t = 8: layer fractions 2tS/N = 1/8 per axis."""
    fr = bench.layer_fractions(_info([[128, 128]] * 3))
    assert fr["fused2"]
    assert fr["L01"] == pytest.approx(0.25) and fr["L"] == pytest.approx(0.375)
    assert fr["sh"] == pytest.approx(1 - 0.875 ** 3) and fr["g01"] == pytest.approx(1 - 0.875 ** 2)
    per = {k: bench.kernel_bytes_per_voxel(k, fr) for k in
           ("corr_x", "rows_first", "strided_fwd", "mid_axis0", "strided_inv", "rows_last", "corr_e", "shell_update")}
    assert per["rows_last"] == 32 and per["strided_fwd"] == per["mid_axis0"] == 16
    assert per["corr_x"] == pytest.approx(4.0) and per["corr_e"] == pytest.approx(4.0)
    assert per["rows_first"] == pytest.approx(24 + 8 * fr["g01"])
    assert sum(per.values()) == pytest.approx(126.3, abs=0.05)


def test_byte_model_without_fused_axis2_corrections():
    """An axis-2 edge with a prime factor above 7: the correction launches on x
    cover axis 2 and the first pass reads E x on every layer voxel."""
    fr = bench.layer_fractions(_info([[123, 123]] * 3))
    assert not fr["fused2"]
    assert bench.kernel_bytes_per_voxel("corr_x", fr) == pytest.approx(2 * fr["L"] * 8)
    assert bench.kernel_bytes_per_voxel("rows_first", fr) == pytest.approx(24 + 8 * fr["sh"])


def test_uncorrected_axes_have_no_layers():
    fr = bench.layer_fractions(_info([[64], [64], [64]], a=(0, 0, 0)))
    assert fr["L"] == 0 and fr["sh"] == 0 and fr["g01"] == 0


@pytest.mark.slow
def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0

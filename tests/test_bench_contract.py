"""The benchmark's reference arm (the oracle, timed on the host) prints one JSON line with
the keys of the measurement contract; it runs without a GPU."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("integrator", ["euler", "heun"])
def test_reference_arm_json_line(integrator):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "1", "--integrator", integrator], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("stochastic 256x128x512")
    assert d["config"]["integrator"] == integrator


def test_projection_flop_counts():
    """2 (r_1 + r_2) per element for the two first contractions, 2 sum r_n for the paper's
    O(r d S) count; the rate uses the kernel time in ms."""
    sys.path.insert(0, ROOT)
    import bench
    fl = bench.projection_flops([512, 256, 12], [16, 16, 12])
    S = 512 * 256 * 12
    assert fl["first_contractions"] == 64 * S and fl["paper_2rd"] == 88 * S
    acts = [(0, (16, 16, 12)), (1, (14, 16, 10))]
    f = bench.flops_fields([512, 256, 12], acts, 0.5)
    assert f["mean_ranks"] == [15.0, 16.0, 11.0]
    assert abs(f["tflops_first_contractions"] - 2 * 31 * S / 0.5e-3 / 1e12) < 1e-12

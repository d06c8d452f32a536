"""Host-side checks of bench.py (no GPU): the reference arm prints one JSON line with the
contract's keys, and the algorithmic operation and transcendental counts follow their closed
forms on a small batch."""
import json
import os
import subprocess
import sys

import numpy as np

from paper_2406_01821_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1",
                          "--cpu-sample", "2048"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert "workload" in d["config"]


def test_operation_counts_closed_forms():
    import bench
    b = synth.from_lists([[(0, [(0, -1, synth.GT, 1.0, 0.0, 0.5), (1, 2, synth.LT, 0.3, -0.7, 0.0)]),
                           (1, [(2, -1, synth.LT, -1.0, 0.0, 0.1)])]], [1])
    N = 100
    # 2 thresholds x 1 op + 1 pair x 3 ops per sample; 2 rules x 3 word ops per 32 samples (4 words)
    assert bench.hard_algorithmic_ops(b, N) == N * (2 + 3) + 3 * 2 * 4
    # 3 transcendentals per condition and sample, 11 per rule and sample
    assert bench.soft_transcendentals(b, N) == N * (3 * 3 + 11 * 2)
    assert np.isclose(bench.hard_algorithmic_ops(b, 32) / 32, 5 + 6 / 32)


def test_skip_list_matches_whole_leg_names():
    import bench
    assert bench.parse_skip("serving") == {"serving"}
    assert "evolution" not in bench.parse_skip("soft_evolution, serving")
    assert bench.parse_skip("soft,evolution,") == {"soft", "evolution"}
    assert bench.parse_skip("") == set()

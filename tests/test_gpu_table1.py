"""The synthetic Table 1 sweep (bench.py --workload table1) end to end on a
few rooms: every method and spacing gets an MAE, and the ordering the paper
reports at its extremes holds (FCC with K = 8 far below K = 1; GCC with r = 2
no worse than r = 1 by more than sampling noise)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_table1_sweep_runs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--workload", "table1", "--rooms", "3"],
                       capture_output=True, text=True, cwd=ROOT, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert len(d["d_m"]) == 11
    for name, v in d["mae_deg"].items():
        assert len(v) == 11 and all(0.0 <= x <= 180.0 for x in v), name
    k1 = sum(d["mae_deg"]["FCC K=1"]) / 11
    k8 = sum(d["mae_deg"]["FCC K=8"]) / 11
    assert k8 < 0.5 * k1
    assert set(d["paper_mae_deg"]) == set(d["mae_deg"])

"""Host-side pieces that need no GPU: the served form's arrival process and admission size,
and the reference (oracle) arm of bench.py, whose JSON line the contract fixes."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_poisson_arrivals():
    from paper_2003_12726_gb300.serve import poisson_arrivals
    t = poisson_arrivals(20000, 20.0, seed=3)
    assert np.all(np.diff(t) >= 0) and t[0] > 0
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 20.0) < 0.05 / 20.0             # mean gap 1/rate
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05            # exponential: CV = 1
    assert np.array_equal(t, poisson_arrivals(20000, 20.0, seed=3))


def test_admission_size_covers_the_workspace():
    import paper_2003_12726_gb300 as px
    from paper_2003_12726_gb300.serve import estimate_bytes
    dims, win = (100, 256, 256, 320, 320), (8, 8)
    for form in (px.FORM_FP32, px.FORM_BF16, px.FORM_TF32):
        ws = px.workspace_size(px.Dims(*dims), px.Options(win[0], win[1], True, form))
        est = estimate_bytes(dims, win, form)
        assert est > ws + 4 * 100 * 256 * 256                    # workspace + frames at least
    assert estimate_bytes((200,) + dims[1:], win, 0) > estimate_bytes(dims, win, 0)


@pytest.mark.timeout(600)
def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1", "--workload", "small"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"

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


def test_full_loop_entry_of_the_bench_line():
    """The full-iteration entry of the default bench line, built from a time_form result:
    per-group averages, FP64/ALU/HBM rooflines with the work the groups are defined by, and
    a JSON-serialisable result."""
    from types import SimpleNamespace
    sys.path.insert(0, ROOT)
    import bench
    s = SimpleNamespace(frames=np.zeros((4, 8, 16), np.float32), ref_shape=(12, 20),
                        M=np.ones((8, 16), np.uint8), window=(2, 2))
    r = {"ktimes": {"omap_scatter": (5, 1.0), "integrate": (5, 20.0), "update_translations": (5, 2.0),
                    "calc_error": (5, 3.0), "filter_map": (5, 0.5), "prepare": (5, 0.05), "upm_exact": (0, 0.0)},
         "ms_per_step": 5.5, "launches": 60, "sweep": {"pairs": 25, "ms": 1.0},
         "extra": {"tw": (1, 1), "filter_r": 4, "integ_steps": 200}, "t_wall": (0.0, 1.0)}
    pk = {"hbm_gbs": 6662.9, "bf16_tflops": 1942.8}
    e = bench.full_loop_entry(r, s, 1.0, "bf16", pk, "measured", 152, 2070.0)
    assert e["dominant_kernel"] == "integrate" and e["kernel_ms"]["integrate"] == 4.0
    assert "upm_exact" not in e["kernel_ms"] and "prepare" not in e["kernel_rooflines"]
    roof = e["kernel_rooflines"]
    assert roof["integrate"]["bound"] == "fp64" and roof["filter_map"]["bound"] == "fp64"
    assert roof["update_translations"]["bound"] == "alu" and roof["calc_error"]["bound"] == "hbm"
    # integrate: 17 flop per good pixel and step over the average launch time
    want = 17.0 * 8 * 16 * 200 / 1e12 / (4.0e-3)
    assert abs(roof["integrate"]["achieved"] - want) < 1e-12 * max(want, 1.0)
    fp64_peak = 152 * 2 * 2 * 2070.0e6 / 1e12
    assert abs(roof["integrate"]["peak"] - fp64_peak) < 1e-12
    # update_translations: 12 flop per pixel, frame and shift of the 3 x 3 window
    want = 12.0 * 4 * 8 * 16 * 9 / 1e12 / (0.4e-3)
    assert abs(roof["update_translations"]["achieved"] - want) < 1e-9 * want
    assert e["translation_window"] == [1, 1] and e["integrate_steps"] == 200
    json.dumps(e)


def test_integrate_central_stencil_identity():
    """The identity behind the integration kernel's fast path: where a pixel's equations along
    an axis are central at p - e, p and p + e, and neither the pixel two behind is second-order
    forward nor the one two ahead second-order backward, (G^T G x)[p] on that axis is
    (2 x[p] - x[p - 2e] - x[p + 2e]) / 4. Checked against G^T G built as a dense matrix from
    the stencil rule (section "Update pixel mapping", the integrate option) on a masked grid."""
    rng = np.random.default_rng(12726 + 907)
    ny, nx = 19, 27
    M = (rng.random((ny, nx)) > 0.04).astype(np.uint8)
    M[4:7, 9:] = 0

    def code(i, j, a):
        L, pos = (ny, i) if a == 0 else (nx, j)

        def good(k):
            t = pos + k
            if t < 0 or t >= L:
                return False
            return bool(M[t, j] if a == 0 else M[i, t])
        if not good(0):
            return 0
        if good(1) and good(-1):
            return 1
        if good(1) and good(2):
            return 2
        if good(-1) and good(-2):
            return 3
        return 4 if good(1) else (5 if good(-1) else 0)

    taps = {1: [(1, .5), (-1, -.5)], 2: [(0, -1.5), (1, 2.), (2, -.5)], 3: [(0, 1.5), (-1, -2.), (-2, .5)],
            4: [(1, 1.), (0, -1.)], 5: [(0, 1.), (-1, -1.)]}
    rows = []
    for a in range(2):
        for i in range(ny):
            for j in range(nx):
                c = code(i, j, a)
                if c:
                    row = np.zeros(ny * nx)
                    for off, cf in taps[c]:
                        row[(i + off) * nx + j if a == 0 else i * nx + j + off] += cf
                    rows.append(row)
    G = np.array(rows)
    x = rng.normal(size=ny * nx)
    q = (G.T @ (G @ x)).reshape(ny, nx)
    X = x.reshape(ny, nx)
    n_fast = 0
    for i in range(ny):
        for j in range(nx):
            def fast(a):
                cc = lambda k: code(i + k, j, a) if a == 0 else code(i, j + k, a)
                return cc(0) == 1 and cc(-1) == 1 and cc(1) == 1 and cc(-2) != 2 and cc(2) != 3
            if fast(0) and fast(1):
                n_fast += 1
                v = X[i, j] - 0.25 * (X[i - 2, j] + X[i + 2, j] + X[i, j - 2] + X[i, j + 2])
                assert abs(v - q[i, j]) < 1e-12
    assert n_fast > 50

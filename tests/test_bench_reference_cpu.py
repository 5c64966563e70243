"""The benchmark's reference arm (the float64 oracle on the host) keeps the
JSON contract the harness reads: one line with the metric, value, unit,
timing, the CPU-baseline object and the end-to-end object.  Runs on the CPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run(
        [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "3", "--warmup", "3"],
        capture_output=True, text=True, timeout=600, cwd=ROOT,
    )
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "config"):
        assert key in line, key
    assert line["steps"] == 3 and line["warmup"] == 3 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    # the same config keys and values as the GPU arm's line at the same N
    sys.path.insert(0, ROOT)
    import bench

    assert line["config"] == bench.step_config(1)


def test_accuracy_report_of_the_headline_step():
    """bench.accuracy on results with known errors: the oracle's own values give
    zero error and bit-exact copies; a relative slip of 1e-6 in z shows as
    full_rel = 1e-6 and full_eps = 1e-6 / kappa; a slip in C shows in
    partial_c_rel; a non-finite z is reported as null (the line stays JSON)."""
    import sys

    import numpy as np

    import oracle as O
    from paper_2109_00626_gb300 import inputs as G

    sys.path.insert(0, ROOT)
    import bench

    x, y = G.order10_r64(0, np.float32)
    x64 = [c.astype(np.float64) for c in x]
    y64 = [c.astype(np.float64) for c in y]
    z = O.contract_full(x64, y64)
    zc, _ = O.partial_chain(x64, y64, bench.MASK)
    a = bench.accuracy(x, y, z, zc)
    assert a["full_eps"] == 0.0 and a["partial_c_rel"] == 0.0 and a["partial_copies_exact"]
    b = bench.accuracy(x, y, z * (1 + 1e-6), zc)
    assert abs(b["full_rel"] - 1e-6) < 1e-12 and abs(b["full_eps"] * b["kappa"] - 1e-6) < 1e-12
    zc2 = [c.copy() for c in zc]
    zc2[3] = zc2[3] * (1 + 1e-4)
    c = bench.accuracy(x, y, z, zc2)
    assert 0.5e-4 < c["partial_c_rel"] <= 1e-4 * (1 + 1e-9)
    zc2[0] = zc2[0] + 1.0
    assert not bench.accuracy(x, y, z, zc2)["partial_copies_exact"]
    d = bench.accuracy(x, y, float("nan"), zc)
    assert d["full_eps"] is None and d["full_rel"] is None


def test_tensor_core_accuracy_report():
    """bench.tc_accuracy: the oracle's own z gives zero end-to-end error and, for
    the bf16 form, the (small) effect of rounding the cores; a relative slip of
    1e-6 shows as rel = 1e-6; the stated bounds are the rounding-error model's
    (relative to |z*|: about 3 % for bf16 on this kappa ~ 1e12 pair, and about
    5e-4 for x3)."""
    import math
    import sys

    import numpy as np

    import oracle as O
    from paper_2109_00626_gb300 import inputs as G

    sys.path.insert(0, ROOT)
    import bench

    x, y = G.order16_r256(0)
    z = O.contract_full([c.astype(np.float64) for c in x], [c.astype(np.float64) for c in y])
    m, e = math.frexp(z)
    rep = bench.tc_accuracy({"native": (m, e), "bf16x3": (m * (1 + 1e-6), e)})
    assert rep["native"]["eps_vs_fp32_cores"] == 0.0
    assert 0.0 < rep["native"]["eps_vs_bf16_cores"] < 1e-10
    assert abs(rep["bf16x3"]["rel_vs_fp32_cores"] - 1e-6) < 1e-12
    from oracle import error_model as M

    x64 = [c.astype(np.float64) for c in x]
    y64 = [c.astype(np.float64) for c in y]
    assert rep["bf16x3"]["bound_rel"] == M.tc_bound(x64, y64, "bf16x3", z) / abs(z)
    assert 1e-5 < rep["bf16x3"]["bound_rel"] < 1e-3 and 1e-3 < rep["native"]["bound_rel"] < 0.2

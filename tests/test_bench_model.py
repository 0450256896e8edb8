"""The benchmark's roofline byte and flop models (CPU).

The byte model of the product's passes is what `roofline.achieved` divides by
the measured pass time, so it is pinned here to its closed form: per RHS,
3 (2N + 8 Nbox) complex elements for the 3-pass schedule and 3 (2N + 24 Nbox)
for the 5-pass one when P = 2 N per axis, plus the 6 M Fourier-space tensor
components read once per batch -- which for the 64x48x32 ellipsoid on its
128x96x64 grid with 2 RHS is about 40 MB and 78 MB per RHS in complex64.
"""
import math

import pytest

import bench
from paper_1002_1505_gb300 import workloads as W


def _sizes(w):
    from oracle import targets as o_targets
    t = o_targets.make_target(w.shape, w.shpar)
    return t.n, tuple(int(v) for v in t.box)


@pytest.mark.parametrize("passes", [3, 5])
def test_byte_model_closed_form(passes):
    n, box = 51488, (64, 48, 32)
    pad = (128, 96, 64)
    nbox = box[0] * box[1] * box[2]
    m = pad[0] * pad[1] * pad[2]
    for nrhs in (1, 2, 128):
        per_launch, names = bench.algorithmic_bytes(passes, n, box, pad, nrhs, 8)
        assert len(per_launch) == len(names) == passes
        per_rhs = sum(per_launch) / nrhs
        k = 8 if passes == 3 else 24
        assert per_rhs == pytest.approx(8 * (3 * (2 * n + k * nbox) + 6 * m / nrhs), rel=1e-15)
    # the ellipsoid bench workload, 2 RHS, complex64: ~40 MB (3-pass) / ~78 MB (5-pass) per RHS
    per_rhs = sum(bench.algorithmic_bytes(passes, n, box, pad, 2, 8)[0]) / 2
    assert per_rhs / 1e6 == pytest.approx(40.2 if passes == 3 else 78.0, abs=0.1)


def test_byte_model_complex128_doubles():
    a64 = bench.algorithmic_bytes(5, 1000, (10, 12, 14), (20, 24, 28), 3, 8)[0]
    a128 = bench.algorithmic_bytes(5, 1000, (10, 12, 14), (20, 24, 28), 3, 16)[0]
    assert [2 * v for v in a64] == a128


def test_flop_model_counts_each_transform_once_per_direction():
    box, pad, nrhs = (64, 48, 32), (128, 96, 64), 2
    f3 = bench.algorithmic_flops(3, box, pad, nrhs)
    f5 = bench.algorithmic_flops(5, box, pad, nrhs)
    assert sum(f3) == pytest.approx(sum(f5), rel=1e-15)  # same work, different pass split
    fft = lambda L: 5 * L * math.log2(L)
    x = 3 * box[1] * box[2] * fft(pad[0])
    y = 3 * box[2] * pad[0] * fft(pad[1])
    z = 3 * pad[0] * pad[1] * fft(pad[2])
    assert sum(f3) == pytest.approx(nrhs * (2 * x + 2 * y + 2 * z + 66 * pad[0] * pad[1] * pad[2]), rel=1e-15)


def test_bench_workloads_match_their_documented_sizes():
    # the sizes the bench line and the profiles quote
    assert _sizes(W.ELLIPSOID64) == (51488, (64, 48, 32))
    assert _sizes(W.PRISM48)[0] == 110592


def _run_bench(args, env_extra=None):
    import json
    import os
    import subprocess
    import sys
    env = dict(os.environ)
    env.update(env_extra or {})
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = subprocess.run([sys.executable, os.path.join(root, "bench.py")] + args, capture_output=True, text=True,
                         env=env, timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    return [json.loads(ln) for ln in lines]


@pytest.mark.parametrize("ws", [1, 2])
def test_reference_arm_line_and_config(ws):
    """`bench.py --impl reference` (the oracle on the host cores) prints one line with the contract's
    keys on rank 0, nothing on the other ranks, and the same config object the GPU arm prints for
    the same workload and world size (its sites and box from the library's host-only set-up)."""
    from paper_1002_1505_gb300 import dda as D
    w = W.SPHERE12
    env = {"WORLD_SIZE": str(ws), "RANK": "0", "LOCAL_RANK": "0"}
    out = _run_bench(["--impl", "reference", "--workload", "sphere12", "--gpus", str(ws), "--steps", "2",
                      "--warmup", "3"], env)
    assert len(out) == 1
    line = out[0]
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "matvecs/s"
    assert line["n_gpus"] == ws and line["steps"] == 2 and line["warmup"] == 3 and line["higher_is_better"]
    assert line["value"] > 0 and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": "matvecs/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    ctx = D.Context(-1)
    n, box = ctx.dda_setup_shape(w.shape, w.shpar)
    pad = w.pad if w.pad else tuple(2 * v for v in box)
    assert line["config"] == bench.workload_config(w, n, box, pad, ws)
    if ws > 1:
        env["RANK"] = "1"
        assert _run_bench(["--impl", "reference", "--workload", "sphere12", "--gpus", str(ws), "--steps", "2"],
                          env) == []

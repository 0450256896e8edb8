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

"""Writes tests/golden/hexprism160_q.txt: efficiencies of the 160 x 128 hexagonal prism
(1,694,720 dipoles, m = 1.33 + 0.001i, x = 20, padded grid 256 x 256 x 320) for the first
seeded orientation and both incident polarizations, from the FP64 oracle alone.

The oracle's BiCGstab (van der Vorst 1992) with its zero-padded FFT product (Goodman, Draine &
Flatau 1991; pinned to the direct O(N^2) sum in the oracle's own tests) is run to a true relative
residual of 1e-8, then the oracle's Q_ext, Q_abs, Q_sca, Q_pha (Draine 1988, the efficiencies the
guide reports) are written.  Run from the repository root:

    python tests/golden/make_hexprism160_q.py

It takes tens of minutes on a few cores (each FP64 product transforms three 21M-point grids).
Only `oracle/` and the input description `paper_1002_1505_gb300/workloads.py` are used.
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import dda as odda  # noqa: E402
from paper_1002_1505_gb300 import workloads as W  # noqa: E402

TOL = 1e-8


def main():
    w = W.HEXPRISM160
    t0 = time.time()
    prob = odda.build_problem(w.shape, w.shpar, w.m, w.x, w.prescription, w.orientations[:1], e01_lf=w.e01,
                              iorth=2, pad=w.pad)
    ps, iters = odda.solve(prob, "bicgstab", tol=TOL, workers=-1, maxit=3000)
    q = odda.cross_sections(prob, ps)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "hexprism160_q.txt")
    with open(out, "w") as fh:
        fh.write("# Efficiencies of the hexagonal prism 160 x 128 (SHPAR 160 128 6), m = 1.33 + 0.001i, x = 20,\n")
        fh.write("# GKDLDR, padded grid 256 x 256 x 320, first seeded orientation of its workload, e01 = y_LF,\n")
        fh.write("# both polarizations (RHS 0 and 1).  Written by tests/golden/make_hexprism160_q.py from the\n")
        fh.write(f"# FP64 oracle only: BiCGstab with the FFT product to |E - A P|/|E| <= {TOL:g}\n")
        fh.write(f"# (iterations {iters[0]}, {iters[1]}; {time.time() - t0:.0f} s).\n")
        fh.write("# key value\n")
        fh.write(f"N {prob.target.n}\n")
        fh.write(f"kd {prob.kd:.17g}\n")
        for b in range(2):
            for key in ("Qext", "Qabs", "Qsca", "Qpha"):
                fh.write(f"{key}_{b} {q[b][key]:.17g}\n")
    print(open(out).read())


if __name__ == "__main__":
    main()

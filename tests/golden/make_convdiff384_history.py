"""Writes convdiff_pe10_384_alpha092_hist40.txt: the oracle's relres history
of 40 FP64 SIP iterations (alpha 0.92) on the 384^3 convection-diffusion block
with median cell Peclet number 10 (seed 4542).  Calls only the oracle and the
seeded input generator."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1303_4538_gb300 import workloads as W  # noqa: E402

if __name__ == "__main__":
    blk = W.convdiff_pe10_384cube()
    F = oracle.factor(blk.nx, blk.ny, blk.nz, blk.coefs, 0.92)
    x, it, rel, hist = oracle.solve(blk.nx, blk.ny, blk.nz, blk.coefs, F, blk.b, rtol=-1.0, max_iters=40)
    with open(os.path.join(HERE, "convdiff_pe10_384_alpha092_hist40.txt"), "w") as f:
        f.write("# relres(x_n), n = 0..40: oracle FP64 SIP, alpha 0.92, convdiff_pe10_384cube (seed 4542)\n")
        f.write("# written by tests/golden/make_convdiff384_history.py\n")
        for v in hist:
            f.write(f"{v:.17e}\n")

"""Writes the oracle regression fixtures in this folder.  Calls only oracle/ and
the seeded input generator; run from the repository root:

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2003_07504_gb300 import synth  # noqa: E402


def main():
    # Algorithm 1, one channel, 12 x 10, lam=1, p=0.8, eps=1e-4, N=4 (the paper's fixed N, c = c0).
    f = synth.voronoi_texture(12, 10, 1, K=4, A=0.05, Tmin=3, Tmax=5, sigma=0.02, seed=4242)[0]
    u = O.ils_channel(f.astype(np.float64), 1.0, 0.8, 1e-4, 4)
    with open(os.path.join(HERE, "ils_12x10_lam1_p08_N4.txt"), "w") as fh:
        fh.write("# Algorithm 1 (Sec. 3.2), lam=1 p=0.8 eps=1e-4 N=4 c=c0; written by make_golden.py from oracle/\n")
        fh.write("# line 1: f (120 values, row-major, float32 exactly representable); line 2: u^4 (float64)\n")
        fh.write(" ".join(repr(float(v)) for v in f.reshape(-1)) + "\n")
        fh.write(" ".join(repr(float(v)) for v in u.reshape(-1)) + "\n")


if __name__ == "__main__":
    main()

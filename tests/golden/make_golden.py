"""Writes tests/golden/lattice_density.txt.  Calls only oracle/.

Uniform cubic lattice of spacing s in a periodic box, equal masses m = s^3 (mean density 1), h = 1.2 s.  Every
particle sees the same neighbourhood, so rho = m * sum over lattice vectors k of W(|k| s, h).  With support
2h = 2.4 s only the shells |k|^2 in {0,1,2,3,4,5} contribute; their multiplicities (lattice vectors of that
squared length in Z^3) are 1, 6, 12, 8, 6, 24, 57 vectors in all.  The shell sum below evaluates the oracle's
kernel at the six shell radii; the density test then checks that the oracle's all-pairs, minimum-image density
sum reproduces it for every particle of a 16^3 and a 64^3 lattice.

Run:  python tests/golden/make_golden.py
"""
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402

SHELLS = [(0, 1), (1, 6), (2, 12), (3, 8), (4, 6), (5, 24)]


def shell_sum(hfac):
    s = 1.0
    r = np.array([math.sqrt(k2) * s for k2, _ in SHELLS])
    w = oracle.w(r, np.full(r.size, hfac * s))
    return float(sum(mult * wk for (_, mult), wk in zip(SHELLS, w))) * s ** 3


def main():
    val = shell_sum(1.2)
    with open(os.path.join(HERE, "lattice_density.txt"), "w") as fh:
        fh.write("# rho of a uniform periodic lattice, mean density 1, h = 1.2 spacing, cubic spline (support 2h)\n")
        fh.write("# = sum over the 57 lattice vectors with |k| < 2.4 of s^3 W(|k| s, 1.2 s); written by make_golden.py\n")
        fh.write("# shells |k|^2:multiplicity = " + " ".join(f"{k2}:{m}" for k2, m in SHELLS) + "\n")
        fh.write(f"hfac 1.2\nrho {val:.17g}\n")
    print(val)


if __name__ == "__main__":
    main()

"""Writes the stored expected values under tests/golden/ that are too slow to
recompute in the CPU test-suite.  Calls only the FP64 oracle (oracle/).

  python tests/golden/make_golden.py

example21_uniform20_g0.9_phi_quadrant.txt
    Scalar flux of Example 2.1 (Sec. 2) with the linear kernel g = 0.9
    (eq. anisotropic kernel, mirror-averaged in zeta), 2D uniform set N = 20
    (1600 ordinates), diamond difference 100 x 100, SI to 1e-12.  The field is
    symmetric under x -> 1-x and y -> 1-y, so only the lower-left 50 x 50
    quadrant is stored ([j][i], i = 0..49 fastest).
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
import rom_workloads as W  # noqa: E402


def main():
    p = W.example_2_1(g=0.9)
    r = O.solve_xy(p.I, p.J, p.bounds, p.sigma_t, p.sigma_s, p.q, [O.quad_uniform_xy(20)],
                   kernel="linear", g=0.9, tol=1e-12)
    phi = r["phi"][0]
    quad = phi[:50, :50]
    path = os.path.join(HERE, "example21_uniform20_g0.9_phi_quadrant.txt")
    with open(path, "w") as f:
        f.write("# Example 2.1, g = 0.9 linear kernel (mirror-averaged), uniform N = 20, DD 100x100,\n")
        f.write("# SI tol 1e-12; lower-left 50x50 quadrant of phi, rows j = 0..49, written by\n")
        f.write("# tests/golden/make_golden.py from the FP64 oracle.\n")
        for row in quad:
            f.write(" ".join(f"{v:.15e}" for v in row) + "\n")
    print("wrote", path, "iters", r["iters"][0])


if __name__ == "__main__":
    main()

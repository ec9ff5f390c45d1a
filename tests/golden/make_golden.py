"""Writes tests/golden/lattice_cubic_eta1.2348.txt from the oracle's kernel.

The value is the root s = h/d of sum_k w(|k| / (gamma_K s)) = (gamma_K eta)^3
over the vectors k of a perfect cubic lattice (Sec. 3.1.1, eq. "partition").
It calls only the oracle (and scipy's root finder)."""
import os
import sys

import numpy as np
from scipy.optimize import brentq

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
import oracle  # noqa: E402

ETA = 1.2348


def main():
    k = np.arange(-4, 5)
    K = np.array(np.meshgrid(k, k, k, indexing="ij")).reshape(3, -1).T
    r = np.sqrt((K ** 2).sum(1))
    g = oracle.GAMMA_K
    s = brentq(lambda s: sum(oracle.w(ri / (g * s)) for ri in r) - (g * ETA) ** 3, 1.0, 1.6,
               xtol=1e-15, rtol=1e-15)
    n = int((r < g * s).sum())
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lattice_cubic_eta1.2348.txt")
    with open(out, "w") as f:
        f.write("# Perfect cubic lattice, cubic-spline kernel (Dehnen & Aly 2012 form, "
                "gamma_K = 1.825742),\n# eta = 1.2348: smoothing length from eq. \"partition\" "
                "(Sec. 3.1.1) solved over the\n# lattice sum.  Written by "
                "tests/golden/make_golden.py (calls only oracle/).\n")
        f.write(f"h_over_d = {s!r}\nn_ngb = {n}\n")


if __name__ == "__main__":
    main()

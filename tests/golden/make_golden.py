"""Write the exact-solution fixtures in this folder.

The paper prints no worked numeric example, so each fixture is the exact solution of a
small FP64 system computed in rational arithmetic by ``oracle.exact`` (the only module
this script calls), rounded once to FP64.  Values are stored as hex floats so the files
round-trip bit for bit.  Re-run with ``python tests/golden/make_golden.py``.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.exact import residual_exact, solve_exact  # noqa: E402

CASES = [
    # name, (t_-1, t_0, t_1), N, seed, distribution
    ("sym_4", (-1.0, 4.0, -1.0), 9, 11, "uniform"),
    ("nonsym_25", (-1.2, 2.5, -0.8), 12, 12, "normal"),
    ("weak_2001", (-1.0, 2.001, -1.0), 16, 13, "uniform"),
    ("equality_dominance", (-1.2, 2.0, -0.8), 10, 14, "uniform"),
    ("mixed_sign", (0.7, 2.5, -1.1), 11, 15, "normal"),
    ("lower_bidiag", (-1.0, 2.0, 0.0), 8, 16, "uniform"),
    ("laplacian", (-1.0, 2.0, -1.0), 13, 17, "uniform"),
    ("two_rows", (-0.5, 3.0, 0.25), 2, 18, "uniform"),
]


def main():
    for name, t, N, seed, dist in CASES:
        rng = np.random.default_rng(seed)
        F = rng.uniform(-1.0, 1.0, N) if dist == "uniform" else rng.standard_normal(N)
        x = solve_exact(t, F)
        assert all(r == 0 for r in residual_exact(t, x, F))
        with open(os.path.join(HERE, name + ".txt"), "w") as fh:
            fh.write("# exact solution of T x = F, T = tridiag{t_-1, t_0, t_1}, rational arithmetic,\n")
            fh.write("# rounded once to FP64 (written by tests/golden/make_golden.py via oracle.exact)\n")
            fh.write("t " + " ".join(float(v).hex() for v in t) + "\n")
            fh.write("F " + " ".join(float(v).hex() for v in F) + "\n")
            fh.write("x " + " ".join(float(v).hex() for v in x) + "\n")


if __name__ == "__main__":
    main()

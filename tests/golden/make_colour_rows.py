"""Write the first row C_{id, tau} of the adjoint colour matrix, Eq. (2.17),
for n = 4..9 gluons, computed by the oracle's explicit SU(3) contraction
(oracle/bg_oracle.cpp: colour_coefficient).  Orderings tau of the labels
2..n-1 are in lexicographic order.  Calls only oracle/.

    python tests/golden/make_colour_rows.py [n ...]

n = 4..8 take seconds to a minute; n = 9 (5040 entries of 8^9 terms) about two
hours on 8 cores.
"""
import math
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
from oracle import oracle as O  # noqa: E402


def main(ns):
    for n in ns:
        t0 = time.time()
        row = O.colour_row_explicit(n)
        path = O.golden_row_path(n)
        with open(path, "w") as f:
            f.write(f"# first row C[id, tau] of the adjoint colour matrix (Eq. 2.17), n = {n} gluons\n")
            f.write(f"# {math.factorial(n - 2)} entries, tau in lexicographic order over labels 2..{n - 1}\n")
            f.write("# written by tests/golden/make_colour_rows.py (oracle explicit SU(3) contraction)\n")
            for v in row:
                f.write(f"{v:.17g}\n")
        print(f"n={n}: {len(row)} entries in {time.time() - t0:.1f} s -> {path}")


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or [4, 5, 6, 7, 8])

"""Write lebesgue_curves.txt: the Lebesgue constants Lambda = ||beta||_1 of the
extrapolation weights against the history size M (Sec. 6.6, the figure of the
Lebesgue constants), for naive extrapolation EXTRAP(M-1, M), the stabilised
least-squares EXTRAP(floor(sqrt(M)), M) and the sparse SPEXTRAP(floor(sqrt(M)), M).
The paper's figure data is not available; this regenerates the curves from the
oracle alone.

    python tests/golden/make_lebesgue_curves.py
"""
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import extrap as ex  # noqa: E402


def rows(Ms=range(1, 17)):
    for M in Ms:
        m = int(math.isqrt(M))
        if m > M - 1:
            m = M - 1
        yield (M, m, ex.lebesgue_constant(ex.naive_coeffs(M)), ex.lebesgue_constant(ex.lsq_coeffs(M, m)),
               ex.lebesgue_constant(ex.sparse_coeffs(M, m)))


def main():
    path = os.path.join(HERE, "lebesgue_curves.txt")
    with open(path, "w") as f:
        f.write("# Lebesgue constants of the extrapolation weights vs history size M (Sec. 6.6).\n")
        f.write("# Written by tests/golden/make_lebesgue_curves.py from oracle/extrap.py only.\n")
        f.write("# format: M m naive_EXTRAP(M-1,M) EXTRAP(m,M) SPEXTRAP(m,M)   (m = floor(sqrt(M)))\n")
        for M, m, a, b, c in rows():
            f.write("%d %d %.17g %.17g %.17g\n" % (M, m, a, b, c))
    print(path)


if __name__ == "__main__":
    main()

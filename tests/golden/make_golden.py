"""Regenerate tests/golden/poisson_S.txt from the Poisson identity.

Uses only the closed form H = L sqrt(alpha/pi) sum_n exp(-alpha L^2 n^2); the
oracle is not called.  Run: python tests/golden/make_golden.py
"""
import math
import os


def S_poisson(L, alpha, nmax=50):
    H = L * math.sqrt(alpha / math.pi) * sum(
        math.exp(-alpha * L * L * n * n) for n in range(-nmax, nmax + 1))
    return H ** 3 - 1.0


HEADER = """\
# Normaliser S = sum_{m != 0} exp(-pi^2 |m|^2 / (alpha L^2)) of the RBE sampling
# density (the paper's Q, Sec. 2.2, Eq. 12), alpha = 0.62.
# Closed form by the Poisson (theta-function) identity:
#   H = sum_m exp(-a m^2) = L sqrt(alpha/pi) sum_n exp(-alpha L^2 n^2),  S = H^3 - 1.
# Written by tests/golden/make_golden.py from that closed form (the oracle is
# not called); columns: N  L  S
"""

if __name__ == "__main__":
    rows = [(1000, 17.1)] + [(n, (n / 0.2) ** (1 / 3)) for n in (100000, 1000000, 10000000)]
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "poisson_S.txt")
    with open(out, "w") as f:
        f.write(HEADER)
        for n, L in rows:
            f.write("%d %r %.6f\n" % (n, L, S_poisson(L, 0.62)))

"""Writes the stored expected values under tests/golden/ from oracle/ only.

supports_L1024_lam2.txt: the kernel supports of Sec. 2.2,
[floor(lam^-(1+j) L), ceil(lam^(1-j) L)], and J_max = ceil(log_lam L), for
L = 1024, lam = 2 -- the paper's formulas evaluated by the oracle.
Run: python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402


def main():
    L, lam = 1024, 2.0
    J = O.j_max(L, lam)
    with open(os.path.join(HERE, "supports_L1024_lam2.txt"), "w") as fh:
        fh.write("# Sec. 2.2: J_max = ceil(log_lam L); supp kappa^j = [floor(lam^-(1+j) L), ceil(lam^(1-j) L)]\n")
        fh.write(f"# L={L} lam={lam}\nJmax {J}\n")
        for j in range(J + 1):
            lo, hi = O.support(j, L, lam)
            fh.write(f"{j} {lo} {hi}\n")


if __name__ == "__main__":
    main()

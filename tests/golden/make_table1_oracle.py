"""Writes table1_oracle.txt: mu = 1 / sigma_M(P_N U P_M) of the oracle's U for
every cell of Table 1 (Sec. 4), beside the printed value, and whether the two
agree to the printed precision (|difference| <= 5e-4).

1D: M = 2^7, N = 2^(7+q).  2D: M = 2^5 x 2^5; P_N U P_M is then a Kronecker
product of two 1D sections, so its smallest singular value is the square of
the 1D one at M = 2^5.  Calls only oracle/.  Run from the repository root:
    python tests/golden/make_table1_oracle.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import dense, tables, wavelets as W  # noqa: E402

ROWS = [("DB2", 2, False), ("DB3", 3, False), ("DB4", 4, False), ("DB5", 5, False), ("DB6", 6, False),
        ("sym2", 2, True), ("sym3", 3, True), ("sym4", 4, True), ("sym5", 5, True), ("sym6", 6, True)]


def printed():
    out = {}
    for line in open(os.path.join(HERE, "table1.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, dim, *vals = line.split()
        out[(name, int(dim))] = [float(v) for v in vals]
    return out


def mu(R, q, p, symlet):
    pp = tables.Sym(p) if symlet else p
    U = dense.U1d_scaling(R, q, pp, W.VMP)
    return 1.0 / np.linalg.svd(U, compute_uv=False)[-1]


def main():
    tab = printed()
    lines = ["# Oracle mu = 1 / sigma_M(P_N U P_M) for every cell of Table 1 (Sec. 4), VMP boundary.",
             "# Written by tests/golden/make_table1_oracle.py (calls only oracle/).",
             "# columns: wavelet dim q oracle printed difference agrees(|difference| <= 5e-4)"]
    for dim in (1, 2):
        for name, p, sym in ROWS:
            for q in (1, 2, 3, 4):
                v = mu(7, q, p, sym) if dim == 1 else mu(5, q, p, sym) ** 2
                pr = tab[(name, dim)][q - 1]
                d = v - pr
                lines.append(f"{name} {dim} {q} {v:.6f} {pr:.3f} {d:+.6f} {int(abs(d) <= 5e-4)}")
    with open(os.path.join(HERE, "table1_oracle.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()

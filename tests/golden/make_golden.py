"""Writes gram_small_oracle.txt: the FP64 oracle on the small Gram workload
(8 x 8 pairs of 32-point paths, d = 3, dyadic order 1; the scheme of Sec. 3.1,
eq. explicit_finite_diff) and on its 8 straight-line pairs, at dyadic orders
0 to 3.  Calls only oracle/ and the seeded input generators.

    python tests/golden/make_golden.py

Regenerate it only with a change to the oracle's arithmetic, and name in that
commit the passage of the paper that justifies the change."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2006_14794_gb300 import inputs  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "gram_small_oracle.txt")


def main():
    w = inputs.gram_small()
    lines = ["# FP64 oracle (scheme of Sec. 3.1, eq. explicit_finite_diff), inputs.gram_small():",
             "# 'gram i j k' = k(X_i, Y_j) at dyadic order 1;",
             "# 'line b lam k' = k of straight-line pair b at dyadic order lam (0..3).",
             "# Written by tests/golden/make_golden.py."]
    G = oracle.gram(w["X"], w["Y"], w["dyadic_order"])
    for i in range(G.shape[0]):
        for j in range(G.shape[1]):
            lines.append("gram %d %d %.17g" % (i, j, G[i, j]))
    for lam in range(4):
        k = oracle.pairs(w["lines_x"], w["lines_y"], lam)
        for b, v in enumerate(k):
            lines.append("line %d %d %.17g" % (b, lam, v))
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()

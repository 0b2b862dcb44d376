"""Writes the golden fixtures of this folder from the oracle alone.

alg1_trace.txt -- Algorithm 1 (k = 1, B = 2, levels of width 2) on five
hand-picked integer candidates in an already-rotated 4-d space.  Every entry
can be checked by hand from Eq. 3: the heap is seeded with candidate 0
(distance 50), so d_k = 50; a candidate is pruned at the first level whose
LB exceeds d_k.

Run:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
import oracle  # noqa: E402

TQ = np.array([3.0, 0.0, 4.0, 0.0])
TX = np.array([[0.0, 0.0, 0.0, 5.0],     # 0: seeds the heap, dist 50
               [3.0, 0.0, 4.0, 1.0],     # 1: dist 1 -> new best
               [-9.0, 0.0, 0.0, 0.0],    # 2: LB^1 = 144 - 0 > 50 -> pruned at l=1
               [3.0, 0.0, -4.0, 0.0],    # 3: LB^1 = 0, LB^2 = 64 > 50 -> l=2
               [3.0, 1.0, 4.0, 0.0]])    # 4: dist 1, ties candidate 1
M = [2, 2]


def main():
    m = oracle.level_thresholds(4, M)
    ids, dists, rho = oracle.refine(TQ, TX, np.arange(5), m, k=1, B=2)
    LB, UB, _, _ = oracle.bounds(TQ, TX, m)
    with open(os.path.join(HERE, "alg1_trace.txt"), "w") as f:
        f.write("# Algorithm 1 / Eq. 3 trace, written by make_golden.py\n")
        f.write("# candidate  LB^0 LB^1 LB^2  UB^0 UB^1 UB^2  rho\n")
        for i in range(5):
            f.write(f"{i} " + " ".join(f"{v:.6f}" for v in LB[i]) + " " +
                    " ".join(f"{v:.6f}" for v in UB[i]) + f" {rho[i]}\n")
        f.write(f"topk {ids[0]} {dists[0]:.6f}\n")


if __name__ == "__main__":
    main()

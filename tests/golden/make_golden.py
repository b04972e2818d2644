"""Write the stored expected values under tests/golden/ from the oracle alone.

Every value written here comes from ``oracle/`` (the CPU oracle); nothing is
taken from the CUDA path.

  leja_points_oracle_1000.txt  the first 1000 greedy Leja points on [-2, 2]
                               (Sec. 2.1 of arXiv 2310.08344), %.17g per line.

Run:  python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402


def main():
    xi = oracle.leja_points_compute(1000)
    path = os.path.join(HERE, "leja_points_oracle_1000.txt")
    np.savetxt(path, xi, fmt="%.17g")
    print("wrote", path)


if __name__ == "__main__":
    main()

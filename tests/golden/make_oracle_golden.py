"""Write the stored oracle values of the 2000-point workload (tests/golden/).

Calls only `oracle/` (and the seeded input generator): the 10 smallest
eigenvalues of L_sym = I - D^{-1/2} W D^{-1/2} (Sec. 2) for n = 2000 points
uniform in [-1/4, 1/4]^3 (seed 1), sigma = 0.1, and the degrees of the first
16 points.  The CPU test `test_oracle_reproduces_stored_values` checks that
the oracle still gives these numbers, so a change to its arithmetic shows.

    python tests/golden/make_oracle_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import eigen, graph  # noqa: E402
from paper_2007_05239_gb300 import workloads  # noqa: E402

OUT = os.path.join(HERE, "oracle_single_n2000_d3.txt")


def main():
    X = workloads.uniform_cube(2000, 3, seed=1)
    lam, _ = eigen.lsym_eigs(X, 0.1, 10)
    deg = graph.degrees(X, 0.1)[:16]
    with open(OUT, "w") as f:
        f.write("# Oracle values for n = 2000 points uniform in [-1/4, 1/4]^3 (seed 1), Gaussian sigma = 0.1,\n")
        f.write("# written by tests/golden/make_oracle_golden.py (oracle/ only).\n")
        f.write("# eigenvalue i: the i-th smallest eigenvalue of L_sym (Sec. 2); degree j: D_jj = sum_{k != j} W_jk.\n")
        for i, v in enumerate(lam):
            f.write(f"eigenvalue {i} {v:.17e}\n")
        for j, v in enumerate(deg):
            f.write(f"degree {j} {v:.17e}\n")
    print(OUT)


if __name__ == "__main__":
    main()

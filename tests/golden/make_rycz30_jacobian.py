"""Writes rycz30_jacobian.txt: the FP64 oracle's <Z_0 Z_29> and its full
Jacobian (600 entries) for the 30-qubit RY + CZ-brick workload (20 layers,
seeded angles, a seeded 5-qubit dense block after every fifth layer), by the
oracle's adjoint method (phi, lambda and mu: three 16 GiB vectors).  Calls
only oracle/ and the seeded workload generator; about 50 GiB of host memory
and one to two hours of CPU time.

    python tests/golden/make_rycz30_jacobian.py
"""

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from workloads import ry_cz_brick  # noqa: E402


def main():
    c, p = ry_cz_brick(30, 20)
    t0 = time.time()
    E, J = oracle.adjoint_jacobian(c, p)
    dt = time.time() - t0
    with open(os.path.join(HERE, "rycz30_jacobian.txt"), "w") as f:
        f.write("# ry_cz_brick(30, 20) (seeded angles, four 5-qubit dense blocks), observable Z_0 Z_29:\n")
        f.write("# first value <Z_0 Z_29>, then d<Z_0 Z_29>/d params[k] for k = 0..599, FP64 oracle adjoint method\n")
        f.write(f"# written by tests/golden/make_rycz30_jacobian.py ({oracle.num_threads()} threads, {dt:.0f} s)\n")
        f.write(f"{float(E[0])!r}\n")
        for v in np.asarray(J[0]):
            f.write(f"{float(v)!r}\n")
    print(float(E[0]), dt)


if __name__ == "__main__":
    main()

"""Writes rycz30_expval.txt: the FP64 oracle's <Z_0 Z_29> for the 30-qubit
RY + CZ-brick workload (20 layers, seeded angles, a seeded 5-qubit dense
block after every fifth layer).  Calls only oracle/ and the
seeded workload generator; needs two 16 GiB vectors of host memory and a few
minutes of CPU time.

    python tests/golden/make_rycz30_expval.py
"""

import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from workloads import ry_cz_brick  # noqa: E402


def main():
    c, p = ry_cz_brick(30, 20)
    t0 = time.time()
    psi = oracle.forward(c, p)
    e = oracle.expval(psi, c.observables[0])
    dt = time.time() - t0
    with open(os.path.join(HERE, "rycz30_expval.txt"), "w") as f:
        f.write("# <Z_0 Z_29> of ry_cz_brick(30, 20) (seeded angles, four 5-qubit dense blocks), "
                "FP64 oracle forward pass\n")
        f.write(f"# written by tests/golden/make_rycz30_expval.py ({oracle.num_threads()} threads, {dt:.0f} s)\n")
        f.write(f"{e!r}\n")
    print(e, dt)


if __name__ == "__main__":
    main()

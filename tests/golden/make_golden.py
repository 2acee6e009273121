"""Write the stored oracle values under tests/golden/ (calls only oracle/).

The paper prints no worked example with numbers (its figures are stripped
and its only figures in the text are performance numbers), so the stored
values here are the oracle's own, on a seeded input: they pin the oracle
across machines and compilers (the same numbers on the x86 and the Arm
hosts), next to the pins in tests/test_oracle_pins.py that tie it to
closed forms and invariants.

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1411_5234_gb300 import inputs  # noqa: E402


def main():
    cl = inputs.plummer(64, seed=0)
    eps = 1e-2
    acc, jerk, pot = oracle.force(cl.pos, cl.vel, cl.mass, eps)
    ek, ep = oracle.energy(cl.pos, cl.vel, cl.mass, eps)
    x, v, a = oracle.leapfrog(cl.pos, cl.vel, acc, cl.mass, eps, 2.0 ** -6, 8)
    out = os.path.join(HERE, "plummer64_seed0_eps1e-2.txt")
    with open(out, "w") as f:
        f.write("# oracle values: inputs.plummer(64, seed=0), eps = 1e-2, G = 1\n")
        f.write("# written by tests/golden/make_golden.py (oracle/ only)\n")
        f.write(f"energy {ek!r} {ep!r}\n")
        for i in range(64):
            row = list(acc[i]) + list(jerk[i]) + [pot[i]]
            f.write("force " + " ".join(repr(float(t)) for t in row) + "\n")
        for i in range(64):
            f.write("leapfrog8 " + " ".join(repr(float(t)) for t in list(x[i]) + list(v[i])) + "\n")
    print("wrote", out)


if __name__ == "__main__":
    main()

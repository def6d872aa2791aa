"""Writes the stored expected values under tests/golden/ from the oracle only.

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import brute_force_ising  # noqa: E402


def main():
    path = os.path.join(HERE, "ising_pm1_n20_ground.txt")
    with open(path, "w") as fh:
        fh.write("# Exact ground-state energies (Eq. 1, ordered pairs) of the N=20 dense\n")
        fh.write("# +-1 Ising instances synth.ising_pm1(20, seed), by enumeration of all\n")
        fh.write("# 2^20 spin configurations (oracle.brute_force_ising).\n")
        fh.write("# seed  H_min\n")
        for seed in range(10):
            J, g = synth.ising_pm1(20, seed)
            e, _ = brute_force_ising(J, g)
            fh.write(f"{seed} {int(round(e))}\n")


if __name__ == "__main__":
    main()

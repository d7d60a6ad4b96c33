"""Writes tests/golden/fci_energies.json from the oracle only.

The stored values are FCI ground-state energies (oracle.fock.fci_energy) of
the seeded synthetic integrals (synth.random_integrals):
  cfg1: K=8 spatial orbitals, N=8, 2Sz=0, seed 0 (determinant space 4900).
  small: K=6, N=6, 2Sz=0, seed 3 (400 determinants) for quick GPU sweeps.
Run: python tests/golden/make_golden.py
"""

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.fock import fci_energy  # noqa: E402
from synth import random_integrals  # noqa: E402


def main():
    out = {}
    t, v = random_integrals(8, 0)
    out["cfg1"] = {"K": 8, "N": 8, "two_sz": 0, "seed": 0, "energy": fci_energy(t, v, 8, 0)}
    t, v = random_integrals(6, 3)
    out["small"] = {"K": 6, "N": 6, "two_sz": 0, "seed": 3, "energy": fci_energy(t, v, 6, 0)}
    with open(os.path.join(HERE, "fci_energies.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()

"""Writes tests/golden/chain60_oracle.json from the FP64 oracle alone.

The paper prints no worked example that synthetic inputs can reproduce (its
systems are real molecules), so the stored values here are the oracle's own
energies and log-dets for the seeded 60-orbital chain (M 60, N 10, X 240, 32
walkers) and its walker = trial energy.  They serve as a regression pin of the
oracle (re-derived on a sample by a CPU test) and as the expected values of the
FP64 GPU parity test.  Only the oracle and the seeded generator are used.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import energy as E  # noqa: E402
from paper_2202_00832_b300 import synth  # noqa: E402


def main():
    wl = synth.CHAIN_60
    mol = wl.molecule()
    walk = wl.walkers(mol)
    energies, logdets = [], []
    for phi in walk:
        e = E.walker_energy(mol, phi)["E"]
        ld = 2 * E.logdet(E.overlap(mol.trial_a, phi))
        energies.append([float(np.real(e)), float(np.imag(e))])
        logdets.append([float(np.real(ld)), float(np.imag(ld))])
    trial = np.ascontiguousarray(mol.trial_a.astype(np.complex128))
    e_trial = E.walker_energy(mol, trial)["E"]
    out = {
        "workload": wl.name, "walkers": len(walk),
        "source": "oracle.energy.walker_energy (exact Cholesky form) and oracle.energy.logdet, FP64",
        "energy": energies, "logdet": logdets,
        "trial_energy": [float(np.real(e_trial)), float(np.imag(e_trial))],
    }
    with open(os.path.join(HERE, "chain60_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()

"""Stored FP64 oracle values of the 60-orbital chain (tests/golden/, written by
tests/golden/make_golden.py from the oracle alone): the oracle re-derives a
sample of them (CPU), and the FP64 GPU path reproduces all of them (GPU)."""
import json
import os

import numpy as np
import pytest

from oracle import energy as E
from paper_2202_00832_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "chain60_oracle.json")


def load():
    with open(GOLDEN) as f:
        d = json.load(f)
    c = lambda a: np.array([x[0] + 1j * x[1] for x in a])
    return d, c(d["energy"]), c(d["logdet"])


def test_oracle_reproduces_stored_values(chain60):
    mol, walk = chain60
    d, e, ld = load()
    assert d["walkers"] == len(walk) and d["workload"] == synth.CHAIN_60.name
    for w in (0, 13, 31):
        got = E.walker_energy(mol, walk[w])["E"]
        assert abs(got - e[w]) <= 1e-12 * abs(e[w])
        got_ld = 2 * E.logdet(E.overlap(mol.trial_a, walk[w]))
        assert abs(got_ld.real - ld[w].real) <= 1e-12
        assert abs(np.angle(np.exp(1j * (got_ld.imag - ld[w].imag)))) <= 1e-12
    trial = np.ascontiguousarray(mol.trial_a.astype(np.complex128))
    et = d["trial_energy"][0] + 1j * d["trial_energy"][1]
    assert abs(E.walker_energy(mol, trial)["E"] - et) <= 1e-12 * abs(et)


@pytest.mark.gpu
def test_fp64_gpu_path_reproduces_stored_values(chain60):
    from paper_2202_00832_b300.lo_afqmc import Context
    mol, walk = chain60
    _, e, ld = load()
    ctx = Context(0)
    ctx.load_molecule(mol)
    got, got_ld, st = ctx.walkers_energy(walk, mode="full", precision="fp64")
    assert np.all(st == 0)
    assert np.max(np.abs(got - e) / np.abs(e)) < 1e-10
    assert np.max(np.abs(got_ld.real - ld.real)) < 1e-10
    assert np.max(np.abs(np.angle(np.exp(1j * (got_ld.imag - ld.imag))))) < 1e-10

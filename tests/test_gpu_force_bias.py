"""Mixed estimate of the Cholesky vectors, <L_g>_w = sum_sigma tr(Lbar_g Theta)
(the force-bias ingredient, walkers_force_bias), against the oracle: FP64 to
1e-10 relative, the split precision to 1e-7 of max |<L_g>| (its Coulomb
vector carries the hi + lo operands' 2^-22 and the 128-term chains)."""
import numpy as np
import pytest

from oracle import energy as E
from paper_2202_00832_b300 import synth
from paper_2202_00832_b300.lo_afqmc import Context

pytestmark = pytest.mark.gpu


def oracle_L(mol, walk):
    return np.array([E.mixed_estimate_L(mol, w) for w in walk])


def test_closed_shell(chain60):
    mol, walk = chain60
    ctx = Context(0)
    ctx.load_molecule(mol)
    ref = oracle_L(mol, walk[:8])
    got, ld, st = ctx.walkers_force_bias(walk[:8], precision="fp64")
    assert np.all(st == 0)
    assert np.abs(got - ref).max() < 1e-10 * np.abs(ref).max()
    got16, ld16, _ = ctx.walkers_force_bias(walk[:8], precision="fp16x3")
    assert np.abs(got16 - ref).max() < 1e-7 * np.abs(ref).max()
    assert np.abs(ld16 - ld).max() < 1e-9


def test_open_shell_ragged():
    mol, walk = synth.small_case(37, 6, 75, 5, seed=13, n_beta=5)
    ctx = Context(0)
    ctx.load_molecule(mol)
    ref = oracle_L(mol, walk)
    got, _, st = ctx.walkers_force_bias(walk, precision="fp64")
    assert np.all(st == 0)
    assert np.abs(got - ref).max() < 1e-10 * np.abs(ref).max()
    got16, _, _ = ctx.walkers_force_bias(walk, precision="fp16x3")
    assert np.abs(got16 - ref).max() < 1e-7 * np.abs(ref).max()

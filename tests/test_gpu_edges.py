"""Edge shapes through the C ABI against the FP64 oracle: one walker, a single
occupied orbital (one pair, one rank tile plus its empty partner), and the
largest supported number of occupied orbitals (LOAF_MAX_NOCC = 96: Gauss-Jordan
columns, 192-wide slice rows, 4656 pairs).  FP64 to 1e-10 relative, split
precision to 0.1 mHa per walker."""
import numpy as np
import pytest

from oracle import energy as E
from paper_2202_00832_b300 import synth
from paper_2202_00832_b300.lo_afqmc import Context, position_operators

pytestmark = pytest.mark.gpu


def oracle_energies(mol, walk):
    return np.array([E.walker_energy(mol, w)["E"] for w in walk])


def run_all(mol, walk):
    ctx = Context(0)
    ctx.load_molecule(mol)
    ref = oracle_energies(mol, walk)
    e64, _, st = ctx.walkers_energy(walk, mode="full", precision="fp64")
    assert np.all(st == 0)
    assert np.max(np.abs(e64 - ref) / np.abs(ref)) < 1e-10
    ctx.lo_localize_compress(0.0, position_operators(mol), localize=True)
    elo, _, _ = ctx.walkers_energy(walk, mode="lo", precision="fp64")
    assert np.max(np.abs(elo - ref) / np.abs(ref)) < 1e-10
    e16, _, st16 = ctx.walkers_energy(walk, mode="lo", precision="fp16x3")
    assert np.all(st16 == 0)
    assert np.abs(e16 - ref).max() < 1e-4
    return ctx


def test_single_walker():
    mol, walk = synth.small_case(M=50, N=7, X=100, W=1, seed=21)
    run_all(mol, walk)


def test_single_occupied_orbital():
    mol, walk = synth.small_case(M=24, N=1, X=48, W=3, seed=22)
    ctx = run_all(mol, walk)
    assert ctx.num_pairs == 1


def test_largest_occupied_count():
    mol, walk = synth.small_case(M=200, N=96, X=120, W=2, seed=23, eps=0.05)
    ctx = run_all(mol, walk)
    assert ctx.num_pairs == 96 * 97 // 2

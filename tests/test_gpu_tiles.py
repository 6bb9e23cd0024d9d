"""Tile shapes of the tensor-core kernels (loaf_set_tiles) through the C ABI.

The LO chunk cap sets how a pair's rows are cut into MMA column chunks (the
N dimension) and the Coulomb split how the (orbital, basis) contraction is
divided over CTA pairs; both only reorder the sums of eq. 2e_HR_RCAS_LO and
eq. 2e_HRchol_RCAS.  Every shape is held to the same bars as the default:
within 0.1 mHa per walker of the oracle's LO energy (built from the library's
localized orbitals and kept ranks) and of the FP64 LO path.
"""
import numpy as np
import pytest

from oracle import energy as E
from oracle import lo
from paper_2202_00832_b300 import synth
from paper_2202_00832_b300.lo_afqmc import Context, LoafError, position_operators

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-4  # Ha per walker


@pytest.fixture(scope="module")
def case():
    """M = 200 (201 dense rows: one chunk of 208 at cap 256, two of 112 at 192
    and 128, three of 80 at 96, four of 64 at 64), N = 20, 130 walkers (two
    walker tiles, the second ragged), T_SVD = 1e-3 (kept ranks vary by pair)."""
    mol, walk = synth.small_case(M=200, N=20, X=300, W=130, seed=211, geometry="acene")
    ctx = Context(0)
    ctx.load_molecule(mol)
    _, msvd = ctx.lo_localize_compress(1e-3, position_operators(mol), localize=True)
    idx = [0, 77, 129]
    C = ctx.localized_trial(0)
    Lbar = E.half_rotate(mol.L, C)
    ths = np.array([E.theta(C, walk[w]) for w in idx])
    pv = lo.pair_exchange_streamed(Lbar, msvd, ths, workers=4)
    N = mol.n_alpha
    wts = np.array([1.0 if i == j else 2.0 for i in range(N) for j in range(i, N)])
    ref = []
    for q, w in enumerate(idx):
        full = E.walker_energy(mol, walk[w])
        ref.append(full["E1"] + full["EJ"] - np.sum(wts * pv[:, q]))
    e64, _, _ = ctx.walkers_energy(walk, mode="lo", precision="fp64")
    yield ctx, mol, walk, idx, np.array(ref), e64
    ctx.set_tiles(256, 0)


@pytest.mark.parametrize("cap,split", [(256, 0), (192, 0), (128, 3), (96, 1), (64, 7)])
def test_shapes_against_oracle(case, cap, split):
    ctx, mol, walk, idx, ref, e64 = case
    ctx.set_tiles(cap, split)
    assert ctx.tiles() == (cap, split)
    e, ld, st = ctx.walkers_energy(walk, mode="lo", precision="fp16x3")
    assert np.all(st == 0)
    assert np.abs(e[idx] - ref).max() < TOL_MIXED
    assert np.abs(e - e64).max() < TOL_MIXED
    # the compressed-Coulomb mode contracts every pair through its factors
    ej, _, st = ctx.walkers_energy(walk[:3], mode="lo_jk", precision="fp16x3")
    ej64, _, _ = ctx.walkers_energy(walk[:3], mode="lo_jk", precision="fp64")
    assert np.all(st == 0)
    assert np.abs(ej - ej64).max() < TOL_MIXED


def test_shapes_agree_with_each_other(case):
    """Two shapes give the same energies up to the reordering of FP32 sums."""
    ctx, mol, walk, idx, ref, e64 = case
    ctx.set_tiles(256, 0)
    a, _, _ = ctx.walkers_energy(walk, mode="lo", precision="fp16x3")
    ctx.set_tiles(64, 5)
    b, _, _ = ctx.walkers_energy(walk, mode="lo", precision="fp16x3")
    ctx.set_tiles(256, 0)
    c, _, _ = ctx.walkers_energy(walk, mode="lo", precision="fp16x3")
    assert np.array_equal(a, c)  # a shape gives the same result every time
    assert np.abs(a - b).max() < 1e-5


@pytest.mark.parametrize("cap,split", [(48, 0), (100, 0), (288, 0), (256, -1), (256, 65)])
def test_bad_shapes_rejected(case, cap, split):
    ctx = case[0]
    ctx.set_tiles(192, 2)
    with pytest.raises(LoafError) as ex:
        ctx.set_tiles(cap, split)
    assert ex.value.status == "LOAF_ERR_ARG"
    assert ctx.tiles() == (192, 2)
    ctx.set_tiles(256, 0)


def test_open_shell_shapes():
    """Open shell (both spins' pair lists cut with the same shapes): a small chunk
    cap and an explicit split against the FP64 LO path and the default shapes."""
    mol, walk = synth.small_case(M=160, N=21, X=220, W=70, seed=212, geometry="acene", n_beta=18)
    ctx = Context(0)
    ctx.load_molecule(mol)
    ctx.lo_localize_compress(1e-3, position_operators(mol), localize=True)
    e64, _, _ = ctx.walkers_energy(walk, mode="lo", precision="fp64")
    ref, _, st = ctx.walkers_energy(walk, mode="lo", precision="fp16x3")
    assert np.all(st == 0)
    ctx.set_tiles(96, 5)
    e, _, st = ctx.walkers_energy(walk, mode="lo", precision="fp16x3")
    assert np.all(st == 0)
    assert np.abs(e - e64).max() < TOL_MIXED
    assert np.abs(e - ref).max() < 1e-5

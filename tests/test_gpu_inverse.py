"""The split-precision overlap inverse on walkers of every conditioning, through
the C ABI.

Scaling walker columns by powers of two, phi -> phi D, leaves the local
energy unchanged (Sec. 2.1: the estimator depends on the walker's span only)
and shifts log det S by sum log D, while the overlap's condition number grows
with the spread of D.  The scaled walkers must meet the bars of the unscaled
ones: energies within 0.1 mHa of the oracle, log-dets within 1e-9, in the
split-precision path (double-float inverse) and in FP64.
"""
import numpy as np
import pytest

from oracle import energy as E
from paper_2202_00832_b300 import synth
from paper_2202_00832_b300.lo_afqmc import Context, position_operators

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    mol, walk = synth.small_case(M=150, N=40, X=200, W=12, seed=404, geometry="acene")
    ctx = Context(0)
    ctx.load_molecule(mol)
    ctx.lo_localize_compress(0.0, position_operators(mol), localize=True)
    ref = np.array([E.walker_energy(mol, w)["E"] for w in walk])
    ld_ref = np.array([E.logdet(E.overlap(mol.trial_a, w)) * 2 for w in walk])
    return ctx, mol, walk, ref, ld_ref


@pytest.mark.parametrize("spread", [0, 3, 6])
def test_column_scaled_walkers(case, spread):
    """Columns of walkers 1, 4, 7, ... scaled by 2^-spread..2^0 (exact in
    floating point); the others unchanged.  (The split-precision path slices a
    walker on one 42-bit grid, so a column 2^-s below the largest keeps 42 - s
    bits: spreads far beyond these cost accuracy whatever the inverse.)"""
    ctx, mol, walk, ref, ld_ref = case
    N = mol.n_alpha
    rng = np.random.default_rng(spread)
    d = 2.0 ** -rng.integers(0, spread + 1, size=N) if spread else np.ones(N)
    phi = walk.copy()
    scaled = np.arange(1, len(walk), 3)
    phi[scaled] = phi[scaled] * d[None, None, :]
    shift = np.zeros(len(walk))
    shift[scaled] = 2 * np.sum(np.log(d))  # closed shell: two equal determinants
    for prec in ("fp16x3", "fp64"):
        e, ld, st = ctx.walkers_energy(phi, mode="lo", precision=prec)
        assert np.all(st == 0)
        assert np.abs(e - ref).max() < 1e-4
        assert np.abs(ld.real - (ld_ref.real + shift)).max() < 1e-9
        dphase = np.angle(np.exp(1j * (ld.imag - ld_ref.imag)))
        assert np.abs(dphase).max() < 1e-9


def test_double_float_inverse_matches_fp64_inverse(case):
    """The double-float inverse and the FP64 inverse give the same energies and
    log-dets on unscaled walkers (to the mixed-precision bar and 1e-10)."""
    ctx, mol, walk, ref, ld_ref = case
    e1, ld1, _ = ctx.walkers_energy(walk, mode="lo", precision="fp16x3")
    e2, ld2, _ = ctx.walkers_energy(walk, mode="lo", precision="fp16x3_f64inv")
    assert np.abs(e1 - e2).max() < 1e-6
    assert np.abs(ld1.real - ld2.real).max() < 1e-10
    assert np.abs(ld1.real - ld_ref.real).max() < 1e-10

"""The paper-literal LO energy (mode lo_jk): exchange and Coulomb both from the
compressed pair factors, E_J = 2 sum_ij (Ubar^[ij]T Theta_i).(Vbar^[ij] Theta_j)
(eq. 2e_HR_RCAS, closed shell), against the oracle's compressed-Coulomb LO
energy.  FP64 path: 1e-10 relative; FP16x3: 0.1 mHa per walker."""
import numpy as np
import pytest

from oracle import lo
from paper_2202_00832_b300 import synth
from paper_2202_00832_b300.lo_afqmc import Context, LoafError, position_operators

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def chain_jk(chain60):
    mol, walk = chain60
    ctx = Context(0)
    ctx.load_molecule(mol)
    return ctx, mol, walk


def test_threshold_zero_equals_full(chain_jk):
    ctx, mol, walk = chain_jk
    e_full, _, _ = ctx.walkers_energy(walk, mode="full", precision="fp64")
    ctx.lo_localize_compress(0.0, position_operators(mol), localize=True)
    e, _, st = ctx.walkers_energy(walk, mode="lo_jk", precision="fp64")
    assert np.all(st == 0)
    assert np.max(np.abs(e - e_full) / np.abs(e_full)) < 1e-10
    e16, _, _ = ctx.walkers_energy(walk, mode="lo_jk", precision="fp16x3")
    assert np.abs(e16 - e_full).max() < 1e-4


def test_truncated_matches_oracle_compressed_coulomb(chain_jk):
    ctx, mol, walk = chain_jk
    T = 1e-2
    _, msvd = ctx.lo_localize_compress(T, position_operators(mol), localize=True)
    spins = lo.prepare(mol, T)
    assert np.array_equal(msvd, spins[0].factors.m_svd)
    ref = np.array([lo.energy_lo(mol, spins, w, coulomb="compressed")["E"] for w in walk[:8]])
    e, _, _ = ctx.walkers_energy(walk[:8], mode="lo_jk", precision="fp64")
    assert np.max(np.abs(e - ref) / np.abs(ref)) < 1e-10
    # the compressed Coulomb moves the energy (T > 0): not the exact-Coulomb LO energy
    e_lo, _, _ = ctx.walkers_energy(walk[:8], mode="lo", precision="fp64")
    assert np.abs(e - e_lo).max() > 1e-8
    e16, _, _ = ctx.walkers_energy(walk[:8], mode="lo_jk", precision="fp16x3")
    assert np.abs(e16 - e).max() < 1e-4


def test_open_shell_is_refused():
    mol, walk = synth.small_case(30, 5, 60, 4, seed=11, n_beta=4)
    ctx = Context(0)
    ctx.load_molecule(mol)
    ctx.lo_localize_compress(1e-4, position_operators(mol), localize=True)
    with pytest.raises(LoafError) as ex:
        ctx.walkers_energy(walk, mode="lo_jk", precision="fp64")
    assert ex.value.status == "LOAF_ERR_UNSUPPORTED"

"""FP64 parity of the CUDA library against the oracle, through the C ABI.

Bar: the energies agree to 1e-10 relative (FP64 mode), Theta to 1e-11 of its
largest entry, log-dets to 1e-10 absolute (phase modulo 2 pi).  Inputs are the
seeded synthetic systems both sides read byte for byte.
"""
import numpy as np
import pytest

from oracle import energy as E
from oracle import lo
from paper_2202_00832_b300 import synth
from paper_2202_00832_b300.lo_afqmc import Context, position_operators

pytestmark = pytest.mark.gpu

TOL_E = 1e-10


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)) / np.maximum(np.abs(np.asarray(b)), 1e-300)


def phase_close(a, b, tol):
    d = np.angle(np.exp(1j * (np.imag(a) - np.imag(b))))
    return np.all(np.abs(np.real(a) - np.real(b)) < tol) and np.all(np.abs(d) < tol)


@pytest.fixture(scope="module")
def chain_ctx(chain60):
    mol, walk = chain60
    ctx = Context(0)
    ctx.load_molecule(mol)
    return ctx, mol, walk


def oracle_energies(mol, walk):
    return np.array([E.walker_energy(mol, w)["E"] for w in walk])


def test_theta_and_logdet(chain_ctx):
    ctx, mol, walk = chain_ctx
    th, ld, st = ctx.walkers_theta(walk)
    assert np.all(st == 0)
    for w in range(len(walk)):
        ref = E.theta(mol.trial_a, walk[w])
        assert np.abs(th[w].T - ref).max() < 1e-11 * np.abs(ref).max()
        ref_ld = 2 * E.logdet(E.overlap(mol.trial_a, walk[w]))
        assert phase_close(ld[w], ref_ld, 1e-10)


def test_full_fp64(chain_ctx):
    ctx, mol, walk = chain_ctx
    e, ld, st = ctx.walkers_energy(walk, mode="full", precision="fp64")
    ref = oracle_energies(mol, walk)
    assert np.all(st == 0)
    assert rel(e, ref).max() < TOL_E


def test_lo_threshold_zero_equals_full(chain_ctx):
    ctx, mol, walk = chain_ctx
    pct, msvd = ctx.lo_localize_compress(0.0, position_operators(mol), localize=True)
    assert np.all(msvd == mol.M) and pct == pytest.approx(0.0)
    e, _, _ = ctx.walkers_energy(walk, mode="lo", precision="fp64")
    assert rel(e, oracle_energies(mol, walk)).max() < TOL_E


def test_pair_exchange_matches_oracle(chain_ctx):
    ctx, mol, walk = chain_ctx
    ctx.lo_localize_compress(0.0, position_operators(mol), localize=True)
    C = ctx.localized_trial(0)
    got = ctx.walkers_pair_exchange(walk[:4])
    # oracle with its own localization; the same Jacobi sweeps reach the same orbitals
    sp = lo.prepare(mol, 0.0)[0]
    assert np.abs(np.abs(sp.trial_loc) - np.abs(C)).max() < 1e-8
    for w in range(4):
        ref = lo.pair_exchange(sp.factors, E.theta(sp.trial_loc, walk[w]))
        assert np.abs(got[:, w] - ref).max() < 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("threshold", [1e-3, 1e-2, 1e-1])
def test_lo_truncated_fp64(chain_ctx, threshold):
    ctx, mol, walk = chain_ctx
    pct, msvd = ctx.lo_localize_compress(threshold, position_operators(mol), localize=True)
    spins = lo.prepare(mol, threshold)
    ref_k = spins[0].factors.m_svd
    # a pair may only differ where a singular value sits on the threshold
    diff = np.nonzero(msvd != ref_k)[0]
    for n in diff:
        s = spins[0].factors.sigma[n]
        assert np.min(np.abs(s - threshold)) < 1e-9 * max(threshold, s[0])
    assert pct == pytest.approx(spins[0].factors.compression_pct(mol.M), abs=0.5)
    e, _, _ = ctx.walkers_energy(walk, mode="lo", precision="fp64")
    ref = np.array([lo.energy_lo(mol, spins, w)["E"] for w in walk])
    if len(diff) == 0:
        assert rel(e, ref).max() < TOL_E
    else:
        assert rel(e, ref).max() < 1e-8


def test_canonical_orbitals_compress_less(chain_ctx):
    ctx, mol, walk = chain_ctx
    pct_loc, _ = ctx.lo_localize_compress(1e-2, position_operators(mol), localize=True)
    pct_can, _ = ctx.lo_localize_compress(1e-2, None, localize=False)
    assert pct_loc > pct_can


@pytest.mark.parametrize("M,N,X,W,nb", [(61, 7, 50, 5, None), (17, 1, 9, 3, None),
                                        (40, 16, 33, 17, None), (30, 6, 90, 4, 5),
                                        (33, 2, 20, 3, 1)])
def test_ragged_shapes_full_and_lo(M, N, X, W, nb):
    mol, walk = synth.small_case(M=M, N=N, X=X, W=W, seed=M + N, n_beta=nb, geometry="acene")
    ctx = Context(0)
    ctx.load_molecule(mol)
    ref = oracle_energies(mol, walk)
    e, _, st = ctx.walkers_energy(walk, mode="full", precision="fp64")
    assert np.all(st == 0)
    assert rel(e, ref).max() < TOL_E
    ctx.lo_localize_compress(0.0, position_operators(mol), localize=True)
    e2, _, _ = ctx.walkers_energy(walk, mode="lo", precision="fp64")
    assert rel(e2, ref).max() < TOL_E


def test_singular_walker_is_flagged(chain_ctx):
    ctx, mol, walk = chain_ctx
    bad = walk[:4].copy()
    # walker 1: its first orbital orthogonal to every trial orbital (an
    # unoccupied eigenvector of h), so Phi_T^T phi has a zero column
    virt = np.linalg.eigh(mol.h)[1][:, mol.n_alpha]
    bad[1][:, 0] = virt
    e, ld, st = ctx.walkers_energy(bad, mode="full", precision="fp64", raise_on_singular=False)
    assert st[1] == 1 and np.isnan(e[1])
    ok = [0, 2, 3]
    assert np.all(st[ok] == 0)
    assert rel(e[ok], oracle_energies(mol, bad[ok])).max() < TOL_E
    from paper_2202_00832_b300.lo_afqmc import LoafError
    with pytest.raises(LoafError) as ei:
        ctx.walkers_energy(bad, mode="full", precision="fp64")
    assert ei.value.status == "LOAF_ERR_SINGULAR"


def test_device_buffers_match_host(chain_ctx):
    import torch
    ctx, mol, walk = chain_ctx
    e_host, ld_host, _ = ctx.walkers_energy(walk, mode="full", precision="fp64")
    phi_d = torch.from_numpy(walk).cuda()
    e_d = torch.zeros(len(walk), dtype=torch.complex128, device="cuda")
    ld_d = torch.zeros_like(e_d)
    st_d = torch.zeros(len(walk), dtype=torch.int32, device="cuda")
    ctx.walkers_energy(phi_d, mode="full", precision="fp64", e_out=e_d, logdet_out=ld_d,
                       walker_status=st_d)
    torch.cuda.synchronize()
    assert np.array_equal(e_d.cpu().numpy(), e_host)
    assert np.array_equal(ld_d.cpu().numpy(), ld_host)


def test_argument_errors(chain_ctx):
    from paper_2202_00832_b300.lo_afqmc import LoafError
    ctx, mol, walk = chain_ctx
    with pytest.raises(LoafError) as ei:
        ctx.walkers_energy(walk, mode=7)
    assert ei.value.status == "LOAF_ERR_ARG"
    fresh = Context(0)
    with pytest.raises(LoafError) as ei:
        fresh.walkers_energy(walk)
    assert ei.value.status == "LOAF_ERR_NOT_READY"

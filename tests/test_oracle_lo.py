"""Pins of the FP64 oracle's localized-orbital steps (CPU only).

LO at T_SVD = 0 reproduces the full energy (Sec. 3.1.1: M_SVD = M is exact);
the truncation error obeys a closed-form bound; the Boys localizer recovers
orbitals that are localized by construction; the pair SVD is checked against a
different LAPACK driver and a rank-one closed form.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import energy as E
from oracle import lo
from paper_2202_00832_b300 import synth


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.fixture(scope="module")
def chain_lo(chain60):
    mol, walk = chain60
    spins0 = lo.prepare(mol, 0.0)
    return mol, walk, spins0


def test_lo_threshold_zero_equals_full(chain_lo):
    mol, walk, spins0 = chain_lo
    for w in range(6):
        full = E.walker_energy(mol, walk[w])
        got = lo.energy_lo(mol, spins0, walk[w])
        assert rel(got["E"], full["E"]) < 1e-10
        assert rel(got["EK"], full["EK"]) < 1e-10


def test_compressed_coulomb_threshold_zero_equals_exact(chain_lo):
    mol, walk, spins0 = chain_lo
    for w in range(3):
        a = lo.energy_lo(mol, spins0, walk[w], coulomb="exact")
        b = lo.energy_lo(mol, spins0, walk[w], coulomb="compressed")
        assert rel(b["EJ"], a["EJ"]) < 1e-10


def test_localized_trial_gives_same_full_energy(chain_lo):
    """Localization is a rotation of occupied orbitals: E_full is unchanged."""
    mol, walk, spins0 = chain_lo
    C = spins0[0].trial_loc
    assert np.abs(C.T @ C - np.eye(mol.n_alpha)).max() < 1e-12
    for w in range(3):
        a = E.walker_energy(mol, walk[w])["E"]
        b = E.energy_cholesky(mol.h, mol.L, C, C, walk[w], walk[w])["E"]
        assert rel(b, a) < 1e-12


def test_pair_symmetry(chain_lo):
    """e_ij = e_ji from Y^[ji] = Y^[ij]^T, on the full ordered-pair loop."""
    mol, walk, spins0 = chain_lo
    sp = spins0[0]
    th = E.theta(sp.trial_loc, walk[2])
    N = mol.n_alpha
    for i in range(N):
        for j in range(N):
            Yij = lo.pair_block(sp.Lbar, i, j)
            Yji = lo.pair_block(sp.Lbar, j, i)
            eij = th[:, j] @ Yij @ th[:, i]
            eji = th[:, i] @ Yji @ th[:, j]
            assert abs(eij - eji) <= 1e-11 * max(1.0, abs(eij))
    # and the i<=j factorised sum equals the ordered-pair sum of traces
    full_ek = sum(th[:, j] @ lo.pair_block(sp.Lbar, i, j) @ th[:, i]
                  for i in range(N) for j in range(N))
    assert rel(lo.exchange_lo(sp.factors, th), full_ek) < 1e-11


@pytest.mark.parametrize("threshold", [1e-3, 1e-2, 1e-1, 1.0])
def test_truncation_error_within_bound(chain_lo, threshold):
    mol, walk, spins0 = chain_lo
    sp = spins0[0]
    fac = lo.truncate(sp.svds, threshold)
    for w in range(4):
        th = E.theta(sp.trial_loc, walk[w])
        err = abs(lo.exchange_lo(fac, th) - lo.exchange_lo(sp.factors, th))
        assert err <= lo.truncation_bound(fac, th) * (1 + 1e-12) + 1e-12


def test_truncation_is_monotone_in_threshold(chain_lo):
    mol, walk, spins0 = chain_lo
    sp = spins0[0]
    prev = None
    for t in [0.0, 1e-4, 1e-2, 1.0, 10.0]:
        k = lo.truncate(sp.svds, t).m_svd
        if prev is not None:
            assert np.all(k <= prev)
        prev = k
    assert np.all(lo.truncate(sp.svds, 0.0).m_svd == mol.M)


def test_compression_definition():
    fac = lo.PairFactors([(0, 0), (0, 1)], [np.zeros((10, 2)), np.zeros((10, 4))],
                         [np.zeros((2, 10)), np.zeros((4, 10))], [None, None], 0.1)
    assert fac.compression_pct(10) == pytest.approx(70.0)


def test_boys_monotone_and_converged(chain_lo):
    mol, _, _ = chain_lo
    C, hist = lo.boys_localize(mol.trial_a, mol.orbital_pos)
    assert all(b >= a - 1e-12 * abs(a) for a, b in zip(hist, hist[1:]))
    assert hist[-1] > hist[0]
    # converged: one more sweep changes nothing measurable
    C2, hist2 = lo.boys_localize(C, mol.orbital_pos, max_sweeps=1)
    assert np.abs(C2 - C).max() < 1e-10


def test_boys_recovers_site_orbitals():
    """Random rotations of orbitals sitting on distinct, far-apart sites are
    undone: the maximum of sum_i <x>_i^2 is reached by the site orbitals."""
    M, N = 12, 4
    pos = np.zeros((M, 3))
    pos[:, 0] = np.arange(M) * 10.0
    sites = [1, 4, 7, 10]
    C0 = np.zeros((M, N))
    for k, p in enumerate(sites):
        C0[p, k] = 1.0
    rng = np.random.default_rng(4)
    U, _ = np.linalg.qr(rng.standard_normal((N, N)))
    C, hist = lo.boys_localize(C0 @ U, pos)
    best = sum((10.0 * p) ** 2 for p in sites)
    assert hist[-1] == pytest.approx(best, rel=1e-12)
    # each localized orbital is +-1 on one site
    assert np.allclose(np.sort(np.abs(C).max(axis=0)), 1.0, atol=1e-7)


def test_pair_svd_against_gesvd_and_reconstruction(chain_lo):
    mol, _, spins0 = chain_lo
    sp = spins0[0]
    for (ij, U, s, Vt) in sp.svds[:6]:
        Y = lo.pair_block(sp.Lbar, *ij)
        s2 = scipy.linalg.svd(Y, compute_uv=False, lapack_driver="gesvd")
        assert np.abs(s - s2).max() <= 1e-12 * s[0]
        assert np.abs(U @ np.diag(s) @ Vt - Y).max() <= 1e-12 * s[0]


def test_pair_svd_rank_one_closed_form():
    """One Cholesky vector: Y^[ij] = a_i a_j^T has the single singular value
    |a_i| |a_j| and Ubar Vbar reproduces it."""
    M, N = 9, 3
    rng = np.random.default_rng(1)
    Lbar = rng.standard_normal((1, N, M))
    svds = lo.pair_svds(Lbar)
    fac = lo.truncate(svds, 1e-10)
    for n, (i, j) in enumerate(fac.pairs):
        a, b = Lbar[0, i], Lbar[0, j]
        assert fac.m_svd[n] == 1
        assert svds[n][2][0] == pytest.approx(np.linalg.norm(a) * np.linalg.norm(b), rel=1e-13)
        assert np.abs(fac.U[n] @ fac.V[n] - np.outer(a, b)).max() < 1e-13


def test_open_shell_lo_threshold_zero():
    mol, walk = synth.small_case(M=24, N=5, X=60, W=2, seed=21, n_beta=4,
                                 geometry="acene")
    spins = lo.prepare(mol, 0.0)
    for w in range(2):
        full = E.walker_energy(mol, walk[w])
        got = lo.energy_lo(mol, spins, walk[w])
        assert rel(got["E"], full["E"]) < 1e-10


@pytest.mark.parametrize("threshold", [0.0, 1e-2])
def test_streamed_pair_values(chain_lo, threshold):
    """The pair-at-a-time form (used where every pair's factors would not fit in
    host memory) gives the stored-factor pair values; at full rank its weighted
    sum is the exchange of the Cholesky form (eq. 2e_HRchol_RCAS), which uses no
    SVD at all."""
    mol, walk, spins0 = chain_lo
    sp = spins0[0]
    fac = lo.truncate(sp.svds, threshold)
    ths = np.array([E.theta(sp.trial_loc, walk[w]) for w in range(3)])
    for workers in (1, 3):
        got = lo.pair_exchange_streamed(sp.Lbar, fac.m_svd, ths, workers=workers)
        for w in range(3):
            ref = lo.pair_exchange(fac, ths[w])
            assert np.abs(got[:, w] - ref).max() < 1e-11 * np.abs(ref).max()
    if threshold == 0.0:
        wts = np.array([1.0 if i == j else 2.0 for i, j in fac.pairs])
        for w in range(3):
            ek = 2.0 * 0.5 * np.sum(wts * got[:, w])  # both spins of the closed shell
            ref = E.walker_energy(mol, walk[w])["EK"]
            assert rel(ek, ref) < 1e-11

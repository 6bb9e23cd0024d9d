"""Pins of the FP64 oracle's full local energy (CPU only).

Each check ties the oracle to something other than itself: the generalized
Wick sum written over all four indices (eq. 2e_general), the textbook
Hartree-Fock energy at walker = trial, a closed form for the one-body term,
invariances the paper's formulas imply, and brute-force determinants.
"""
import itertools

import numpy as np
import pytest

from oracle import energy as E
from paper_2202_00832_b300 import synth


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def test_wick_loops_pin_einsum():
    """The einsum Wick sum equals explicit Python loops on a 6-orbital system."""
    mol, walk = synth.small_case(M=6, N=2, X=7, W=2, seed=3, n_beta=1)
    V = E.dense_eri(mol.L)
    for w in range(2):
        pa, pb = walk[w][:, :2], walk[w][:, 2:]
        Ga, Gb = E.green(mol.trial_a, pa), E.green(mol.trial_b, pb)
        e_dense = E.energy_wick_dense(mol.h, V, Ga, Gb)[0]
        e_loops = E.energy_wick_loops(mol.h, V, Ga, Gb)
        assert rel(e_dense, e_loops) < 1e-13


@pytest.mark.parametrize("open_shell", [False, True])
def test_cholesky_form_equals_wick_bruteforce(chain60, open_shell):
    """eq. 2e_HRchol_RCAS equals eq. 2e_general with V rebuilt from L."""
    if open_shell:
        mol, walk = synth.small_case(M=30, N=6, X=90, W=3, seed=11, n_beta=5)
    else:
        mol, walk = chain60
    V = E.dense_eri(mol.L)
    for w in range(3):
        pa, pb = E.split_walker(mol, walk[w])
        Ga, Gb = E.green(mol.trial_a, pa), E.green(mol.trial_b, pb)
        ref, e1, e2 = E.energy_wick_dense(mol.h, V, Ga, Gb)
        got = E.walker_energy(mol, walk[w])
        assert rel(got["E"], ref) < 1e-12
        assert rel(got["E1"], e1) < 1e-12
        assert rel(got["EJ"] - got["EK"], e2) < 1e-12


@pytest.mark.parametrize("open_shell", [False, True])
def test_walker_equal_trial_gives_hartree_fock(chain60, open_shell):
    """At phi = Phi_T the local energy is the RHF/UHF energy of the trial."""
    if open_shell:
        mol, _ = synth.small_case(M=30, N=6, X=90, W=1, seed=11, n_beta=5)
        phi = np.concatenate([mol.trial_a, mol.trial_b], axis=1).astype(complex)
    else:
        mol, _ = chain60
        phi = mol.trial_a.astype(complex)
    eri_chem = np.einsum("gpq,grs->pqrs", mol.L, mol.L, optimize=True)
    Pa = mol.trial_a @ mol.trial_a.T
    Pb = mol.trial_b @ mol.trial_b.T
    ref = E.hf_energy_dense(mol.h, eri_chem, Pa, Pb)
    got = E.walker_energy(mol, phi)["E"]
    assert abs(got.imag) < 1e-9 * abs(ref)
    assert rel(got.real, ref) < 1e-12


def test_one_body_closed_form(chain60):
    """Trial = lowest eigenvectors of h  =>  E1 = 2 sum_i lambda_i for every walker.

    Phi_T^T h = diag(lambda) Phi_T^T and Phi_T^T Theta = I (eq. Q), so the
    one-body energy does not depend on the walker.
    """
    mol, walk = chain60
    lam = np.linalg.eigvalsh(mol.h)[:mol.n_alpha]
    for w in range(4):
        e1 = E.walker_energy(mol, walk[w])["E1"]
        assert abs(e1 - 2 * lam.sum()) < 1e-12 * abs(lam.sum())


def test_walker_gauge_invariance(chain60):
    """E(phi R) = E(phi) for an invertible R: Theta depends only on span(phi)."""
    mol, walk = chain60
    rng = np.random.default_rng(5)
    for w in range(3):
        R = rng.standard_normal((10, 10)) + 1j * rng.standard_normal((10, 10))
        a = E.walker_energy(mol, walk[w])["E"]
        b = E.walker_energy(mol, walk[w] @ R)["E"]
        assert rel(b, a) < 1e-11


def test_trial_rotation_invariance(chain60):
    """Rotating the occupied trial orbitals (Phi_T -> Phi_T U) leaves E unchanged."""
    mol, walk = chain60
    rng = np.random.default_rng(6)
    U, _ = np.linalg.qr(rng.standard_normal((10, 10)))
    for w in range(3):
        a = E.walker_energy(mol, walk[w])["E"]
        b = E.energy_cholesky(mol.h, mol.L, mol.trial_a @ U, mol.trial_b @ U,
                              walk[w], walk[w])["E"]
        assert rel(b, a) < 1e-12


def test_theta_reproduces_identity(chain60):
    """Phi_T^dagger Theta = I (eq. Q)."""
    mol, walk = chain60
    th = E.theta(mol.trial_a, walk[0])
    assert np.abs(mol.trial_a.T @ th - np.eye(10)).max() < 1e-12


def leibniz_det(A):
    n = A.shape[0]
    tot = 0j
    for perm in itertools.permutations(range(n)):
        inv = sum(1 for a in range(n) for b in range(a + 1, n) if perm[a] > perm[b])
        term = (-1) ** inv
        for r in range(n):
            term = term * A[r, perm[r]]
        tot += term
    return tot


def test_logdet_brute_force():
    """exp(logdet) equals the Leibniz determinant, pivoting included."""
    rng = np.random.default_rng(9)
    for n in (1, 2, 3, 5, 6):
        A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        A[0, 0] = 1e-3  # forces a row exchange
        assert rel(np.exp(E.logdet(A)), leibniz_det(A)) < 1e-12


def test_logdet_matches_slogdet(chain60):
    mol, walk = chain60
    for w in range(4):
        S = E.overlap(mol.trial_a, walk[w])
        sign, ld = np.linalg.slogdet(S)
        got = E.logdet(S)
        assert abs(got.real - ld) < 1e-12
        assert abs(np.exp(1j * got.imag) - sign) < 1e-12


def test_lu_factors_reconstruct():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((7, 7)) + 1j * rng.standard_normal((7, 7))
    LU, perm, _ = E.lu_partial_pivot(A)
    Lf = np.tril(LU, -1) + np.eye(7)
    Uf = np.triu(LU)
    assert np.abs(Lf @ Uf - A[perm]).max() < 1e-13
    assert np.all(np.abs(np.tril(LU, -1)) <= 1.0 + 1e-15)


def test_singular_overlap_logdet():
    """A walker orthogonal to one trial orbital has det S = 0."""
    S = np.array([[1.0, 2.0], [2.0, 4.0]], dtype=complex)
    assert E.logdet(S) == complex(-np.inf)


# --- planted mistakes: each plausible slip fails at least one pin ----------

def _energy_variant(mol, phi, mistake):
    th = E.theta(mol.trial_a, phi)
    hbar = mol.trial_a.T @ mol.h
    Lbar = E.half_rotate(mol.L, mol.trial_a)
    T = np.einsum("gir,rj->gij", Lbar, th)
    J = 2 * np.einsum("gii->g", T)
    e1 = 2 * np.sum(hbar * th.T)
    ek = np.einsum("gij,gji->", T, T)
    if mistake == "no_half_exchange":
        ek = 2 * ek
    elif mistake == "transposed_exchange":
        ek = np.einsum("gij,gij->", T, T)
    elif mistake == "exchange_sign":
        ek = -ek
    elif mistake == "theta_no_inverse":
        th2 = phi
        T = np.einsum("gir,rj->gij", Lbar, th2)
        J = 2 * np.einsum("gii->g", T)
        ek = np.einsum("gij,gji->", T, T)
    return e1 + 0.5 * np.sum(J * J) - ek


@pytest.mark.parametrize("mistake", ["no_half_exchange", "transposed_exchange",
                                     "exchange_sign", "theta_no_inverse"])
def test_planted_mistakes_fail_a_pin(chain60, mistake):
    mol, walk = chain60
    V = E.dense_eri(mol.L)
    phi = walk[1]
    G = E.green(mol.trial_a, phi)
    ref = E.energy_wick_dense(mol.h, V, G, G)[0]
    assert rel(_energy_variant(mol, phi, "none"), ref) < 1e-12
    assert rel(_energy_variant(mol, phi, mistake), ref) > 1e-6


def test_mixed_estimate_of_L_at_the_trial_is_the_density_trace(chain60):
    """At phi = Phi_T, Theta = Phi_T and <L_g> = sum_sigma tr(L_g P^sigma) with the
    trial density P = Phi_T Phi_T^T (both spins for the closed shell)."""
    mol, _ = chain60
    phi = np.ascontiguousarray(mol.trial_a.astype(np.complex128))
    got = E.mixed_estimate_L(mol, phi)
    P = mol.trial_a @ mol.trial_a.T
    ref = 2.0 * np.einsum("gpq,qp->g", mol.L, P)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_mixed_estimate_of_L_is_gauge_invariant(chain60):
    """<L_g> depends on the walker's span only: phi R gives the same vector, and
    a Theta formed without the inverse overlap (phi instead of phi S^-1) fails."""
    mol, walk = chain60
    rng = np.random.default_rng(5)
    R = rng.standard_normal((mol.n_alpha, mol.n_alpha)) + 1j * rng.standard_normal((mol.n_alpha, mol.n_alpha))
    a = E.mixed_estimate_L(mol, walk[3])
    b = E.mixed_estimate_L(mol, walk[3] @ R)
    assert np.allclose(a, b, rtol=1e-10, atol=1e-10)
    Lbar = E.half_rotate(mol.L, mol.trial_a)
    wrong = lambda ph: 2.0 * np.einsum("gir,ri->g", Lbar, ph)   # planted: no S^-1
    assert not np.allclose(wrong(walk[3]), wrong(walk[3] @ R), rtol=1e-6)


def test_propagator_operator_pins(chain60):
    """V = sum_g x_g L_g: a unit field picks out L_g; V is linear in x and
    symmetric (every L_g is); a real x gives a real V."""
    mol, _ = chain60
    X = mol.X
    e = np.zeros(X, dtype=np.complex128)
    e[7] = 1.0
    assert np.array_equal(E.propagator_operator(mol, e), mol.L[7].astype(np.complex128))
    rng = np.random.default_rng(9)
    x1 = rng.standard_normal(X) + 1j * rng.standard_normal(X)
    x2 = rng.standard_normal(X) + 1j * rng.standard_normal(X)
    v1, v2 = E.propagator_operator(mol, x1), E.propagator_operator(mol, x2)
    assert np.allclose(E.propagator_operator(mol, 2.0 * x1 - 3j * x2), 2.0 * v1 - 3j * v2, atol=1e-10)
    assert np.allclose(v1, v1.T, atol=1e-12)
    vr = E.propagator_operator(mol, x1.real.astype(np.complex128))
    assert np.abs(vr.imag).max() == 0.0
    # an explicit loop over the fields
    ref = np.zeros((mol.M, mol.M), dtype=np.complex128)
    for g in range(X):
        ref += x1[g] * mol.L[g]
    assert np.allclose(v1, ref, rtol=1e-12, atol=1e-12)

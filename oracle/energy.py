"""Local energy of a single-determinant trial, plain FP64 (test infrastructure).

Notation follows the paper (Sec. 2.1.1 and 2.2): M basis functions indexed
p, q, r, s; N occupied orbitals per spin indexed i, j; X Cholesky vectors
indexed g (the paper's alpha).  Phi_T is the trial (M x N per spin), phi the
walker (M x N per spin), both with orbitals as columns.

Only the test suite, the smoke check and the CPU baseline of the benchmark use
this module.
"""
from __future__ import annotations

import numpy as np


# ---------------------------------------------------------------------------
# overlap, LU with partial pivoting, log-determinant
# ---------------------------------------------------------------------------

def overlap(trial: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """S = Phi_T^dagger phi, the N x N overlap matrix inside eq. Q."""
    return trial.conj().T @ phi


def lu_partial_pivot(S: np.ndarray):
    """Doolittle LU with row partial pivoting, written out step by step.

    Returns (LU, perm, n_swaps): the unit-lower and upper factors packed in one
    array, the row permutation (row k of P S is row perm[k] of S) and the
    number of row exchanges.  The pivot is the first row holding the largest
    modulus in the current column.  A zero pivot leaves the column untouched
    (the determinant is then zero).
    """
    A = np.array(S, dtype=np.complex128, copy=True)
    n = A.shape[0]
    perm = np.arange(n)
    swaps = 0
    for k in range(n):
        col = np.abs(A[k:, k])
        p = k + int(np.argmax(col))
        if p != k:
            A[[k, p]] = A[[p, k]]
            perm[[k, p]] = perm[[p, k]]
            swaps += 1
        piv = A[k, k]
        if piv == 0:
            continue
        A[k + 1:, k] /= piv
        A[k + 1:, k + 1:] -= np.outer(A[k + 1:, k], A[k, k + 1:])
    return A, perm, swaps


def logdet(S: np.ndarray) -> complex:
    """log det S from the LU factors: sum of log U_kk plus i*pi per row swap.

    The imaginary part is defined modulo 2 pi.  The overlap ratio that
    updates walker weights (Sec. 2.1) is exp of a difference of these.
    """
    LU, _, swaps = lu_partial_pivot(S)
    d = np.diag(LU)
    if np.any(d == 0):
        return complex(-np.inf)
    return complex(np.sum(np.log(d.astype(np.complex128))) + 1j * np.pi * (swaps % 2))


def theta(trial: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """Theta = phi (Phi_T^dagger phi)^-1, the paper's Q intermediate (eq. Q)."""
    S = overlap(trial, phi)
    # phi S^-1 = (S^-T phi^T)^T
    return np.linalg.solve(S.T, phi.T).T


def green(trial: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """G_pq = [phi (Phi_T^dagger phi)^-1 Phi_T^dagger]^T, eq. G / GwQ (one spin)."""
    return (theta(trial, phi) @ trial.conj().T).T


# ---------------------------------------------------------------------------
# reference definitions: dense ERI, generalized Wick sum
# ---------------------------------------------------------------------------

def dense_eri(L: np.ndarray) -> np.ndarray:
    """V_pqrs = sum_g L^g_pr L^g_qs (Sec. 2.1: V_pqrs = (pr|qs))."""
    return np.einsum("gpr,gqs->pqrs", L, L, optimize=True)


def energy_wick_dense(h: np.ndarray, V: np.ndarray, G_a: np.ndarray,
                      G_b: np.ndarray, e0: float = 0.0):
    """E1 + E2 by the generalized Wick sum over all four basis indices.

    E1 = sum_sigma sum_pq h_pq G^sigma_pq (the one-body part of H, Sec. 2.1);
    E2 = 1/2 sum_pqrs V_pqrs [sum_{sigma tau} G^sigma_pr G^tau_qs
                              - sum_sigma G^sigma_ps G^sigma_qr]   (eq. 2e_general,
    with the spin-diagonal G of eq. G).  Returns (E, E1, E2).
    """
    Gt = G_a + G_b
    e1 = np.einsum("pq,pq->", h, Gt)
    direct = np.einsum("pqrs,pr,qs->", V, Gt, Gt, optimize=True)
    exch = sum(np.einsum("pqrs,ps,qr->", V, G, G, optimize=True) for G in (G_a, G_b))
    e2 = 0.5 * (direct - exch)
    return e0 + e1 + e2, e1, e2


def energy_wick_loops(h, V, G_a, G_b) -> complex:
    """The same Wick sum with explicit Python loops (tiny M only)."""
    M = h.shape[0]
    e = 0j
    for p in range(M):
        for q in range(M):
            e += h[p, q] * (G_a[p, q] + G_b[p, q])
    for p in range(M):
        for q in range(M):
            for r in range(M):
                for s in range(M):
                    v = V[p, q, r, s]
                    if v == 0:
                        continue
                    t = 0j
                    for Gs in (G_a, G_b):
                        for Gt in (G_a, G_b):
                            t += Gs[p, r] * Gt[q, s]
                        t -= Gs[p, s] * Gs[q, r]
                    e += 0.5 * v * t
    return e


# ---------------------------------------------------------------------------
# Cholesky (half-rotated) form: the "full" path
# ---------------------------------------------------------------------------

def half_rotate(L: np.ndarray, trial: np.ndarray) -> np.ndarray:
    """Lbar^g_ir = sum_p conj(Phi_T,pi) L^g_pr, shape (X, N, M) (Sec. 2.2).

    The paper writes Lbar without the conjugate; the trial here is real, and
    the conjugate is what eq. GwQ's Phi_T^dagger supplies.
    """
    return np.einsum("pi,gpr->gir", trial.conj(), L, optimize=True)


def energy_cholesky(h, L, trial_a, trial_b, phi_a, phi_b, e0: float = 0.0):
    """Local energy through the half-rotated Cholesky vectors (eq. 2e_HRchol_RCAS).

    For one determinant: Theta^sigma = phi^sigma (Phi_T^sigma^dagger phi^sigma)^-1,
    T^sigma_g = Lbar^sigma_g Theta^sigma (N x N), and
      E1 = sum_sigma sum_ir hbar^sigma_ir Theta^sigma_ri,   hbar = Phi_T^dagger h
      E2 = 1/2 sum_g [ (sum_sigma tr T^sigma_g)^2 - sum_sigma tr(T^sigma_g T^sigma_g) ].
    Returns a dict with E, E1, EJ (Coulomb), EK (exchange), J (per-g traces,
    spin summed) and logdet (sum over spins).
    """
    X = L.shape[0]
    e1 = 0j
    J = np.zeros(X, dtype=np.complex128)
    ek = 0j
    ld = 0j
    for trial, phi in ((trial_a, phi_a), (trial_b, phi_b)):
        if trial.shape[1] == 0:
            continue
        th = theta(trial, phi)
        ld += logdet(overlap(trial, phi))
        hbar = trial.conj().T @ h
        e1 += np.sum(hbar * th.T)
        Lbar = half_rotate(L, trial)
        T = np.einsum("gir,rj->gij", Lbar, th, optimize=True)
        J += np.einsum("gii->g", T)
        ek += 0.5 * np.einsum("gij,gji->", T, T)
    ej = 0.5 * np.sum(J * J)
    return dict(E=e0 + e1 + ej - ek, E1=e1, EJ=ej, EK=ek, J=J, logdet=ld)


def mixed_estimate_L(mol, phi: np.ndarray) -> np.ndarray:
    """<L_g>_w = sum_sigma tr(Lbar^sigma_g Theta^sigma), g < X: the mixed
    estimate of each Cholesky vector, from which importance sampling shifts the
    auxiliary fields (the force bias, -sqrt(dtau) <L_g>, Sec. 2.1).  It is the
    spin-summed trace vector J of energy_cholesky."""
    return walker_energy(mol, phi)["J"]


def propagator_operator(mol, x: np.ndarray) -> np.ndarray:
    """V = sum_g x_g L_g (M x M): the one-body operator of the Hubbard-Stratonovich
    propagator for one walker's fields x (X complex values; the paper's
    B = sum_alpha x_alpha L_alpha, with sqrt(dtau) and the force-bias shift
    already in x)."""
    return np.einsum("g,gpq->pq", x, mol.L, optimize=True)


def split_walker(mol, phi: np.ndarray):
    """(phi_a, phi_b) from a packed walker: closed shell reuses one block."""
    na, nb = mol.n_alpha, mol.n_beta
    if na == nb and phi.shape[1] == na:
        return phi, phi
    return phi[:, :na], phi[:, na:na + nb]


def walker_energy(mol, phi: np.ndarray, e0: float = 0.0):
    """energy_cholesky for a synthetic molecule and one packed walker."""
    pa, pb = split_walker(mol, phi)
    return energy_cholesky(mol.h, mol.L, mol.trial_a, mol.trial_b, pa, pb, e0)


def hf_energy_dense(h: np.ndarray, eri_chem: np.ndarray, P_a: np.ndarray,
                    P_b: np.ndarray) -> float:
    """Textbook unrestricted Hartree-Fock energy from densities P^sigma.

    E = sum_pq h_pq (P^a + P^b)_pq + 1/2 sum_pqrs (pq|rs) [P_pq P_rs
        - sum_sigma P^sigma_ps P^sigma_rq], P = P^a + P^b, chemists' (pq|rs).
    Used only as a closed-form pin of the walker = trial energy.
    """
    P = P_a + P_b
    e = np.einsum("pq,pq->", h, P)
    e += 0.5 * np.einsum("pqrs,pq,rs->", eri_chem, P, P, optimize=True)
    for Ps in (P_a, P_b):
        e -= 0.5 * np.einsum("pqrs,ps,rq->", eri_chem, Ps, Ps, optimize=True)
    return float(np.real(e))

"""Multi-determinant (CAS) trial: LO local energy through Sherman-Morrison-
Woodbury updates of the reference determinant, plain FP64 (test infrastructure).

Follows Sec. 3.1.2: eqs. Q_SMW_reg, Q_SMW, BigQ, 2e_HR_RCAS_LO and 2e_HR_RCAS
and the intermediates table.  Steps, in the paper's order:
  1. reference: A = Phi_T^0T phi, A^-1 and Theta^0 = phi A^-1 (eq. Q);
  2. per determinant d, whose slots s_1..s_k hold new orbitals: U^d = the unit
     vectors of those slots, V^dT = the change of those rows of A, and
     S_d = (I + V^dT A^-1 U^d)^-1 V^dT A^-1 (k x N, the table's {S}_d), so that
     Q^d = phi A_d^-1 = Theta^0 - (Theta^0 U^d) S_d (eq. Q_SMW_reg); A^-1 U^d is
     a column selection of A^-1, no product;
  3. per orbital pair [ij] the projections of the reference columns,
     Ubar^[ij]T Theta^0 and Vbar^[ij] Theta^0, and per determinant the
     projected columns of eq. BigQ: Qbar = (projection of the column of slot t)
     - (projection of the excited slots) S_d[:, t];
  4. per determinant e_st = Qbar_L . Qbar_R over its occupied slots (exchange),
     the one-body and Coulomb terms from Q^d, and the mixed estimate
     E = sum_d c_d <Phi_d|phi> E_d / sum_d c_d <Phi_d|phi>
     with <Phi_d|phi> / <Phi_0|phi> = det(I + V^dT A^-1 U^d)^2 (closed shell,
     the matrix determinant lemma).
The direct route (an inverse per determinant and the Cholesky-form energy)
is here too, as the reference the SMW route is checked against.

Readings where the paper is silent (its supporting information is not
available):
  * determinants are closed shell (the alpha string equals the beta string):
    one Q^d serves both spins, as in eq. 2e_HR_RCAS;
  * the weights c_d <Phi_d|phi> / sum c <Phi|phi> printed for E_2 apply to the
    one-body energy as well (the mixed estimate of H);
  * a new active orbital occupies the slot of the orbital it replaces;
  * only the inactive orbitals are localized (Sec. 4); the active ones stay as
    given.

Only the test suite may use this module.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

from . import energy as E
from . import lo as LO


# ---------------------------------------------------------------------------
# orbitals and determinants
# ---------------------------------------------------------------------------

def occupied(C: np.ndarray, det: List[int]) -> np.ndarray:
    """Phi_d: the orbitals of determinant d in slot order (M x N)."""
    return C[:, det]


def excitation(dets: List[List[int]], d: int):
    """Slots where determinant d differs from the reference, with the orbitals
    there in the reference and in d."""
    ref = dets[0]
    slots = [s for s, (a, b) in enumerate(zip(dets[d], ref)) if a != b]
    return slots, [ref[s] for s in slots], [dets[d][s] for s in slots]


def localize_inactive(C: np.ndarray, n_inact: int, pos: np.ndarray) -> np.ndarray:
    """Foster-Boys rotation of the inactive block only (Sec. 4); every
    determinant holds all inactive orbitals, so its overlap changes by the same
    factor det(R)^2 = 1 and its energy not at all."""
    out = np.array(C)
    if n_inact > 1:
        out[:, :n_inact] = LO.boys_localize(C[:, :n_inact], pos)[0]
    return out


# ---------------------------------------------------------------------------
# 1-2. reference and SMW updates
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class SMWDet:
    slots: List[int]          # excited slots s_1..s_k
    S: np.ndarray             # (k, N): (I + V^T A^-1 U)^-1 V^T A^-1
    ratio: complex            # det(A_d) / det(A)
    theta: np.ndarray         # Q^d = phi A_d^-1 (M x N)


def smw_thetas(C: np.ndarray, dets: List[List[int]], phi: np.ndarray):
    """Theta^0 and, per determinant, the SMW intermediates and Q^d (eq. Q_SMW_reg)."""
    A = E.overlap(occupied(C, dets[0]), phi)
    Ainv = np.linalg.inv(A)
    th0 = phi @ Ainv
    out = []
    for d in range(len(dets)):
        slots, old, new = excitation(dets, d)
        k = len(slots)
        if k == 0:
            out.append(SMWDet([], np.zeros((0, A.shape[0]), dtype=np.complex128), 1.0 + 0j, th0))
            continue
        VT = C[:, new].conj().T @ phi - C[:, old].conj().T @ phi    # (k, N): new rows - old rows
        AinvU = Ainv[:, slots]                                       # A^-1 U^d: columns of A^-1
        Md = np.eye(k) + VT @ AinvU                                  # I + V^T A^-1 U
        S = np.linalg.solve(Md, VT @ Ainv)                           # the table's S_d
        th = th0 - th0[:, slots] @ S                                 # Theta^0 - (Theta^0 U) S_d
        out.append(SMWDet(slots, S, complex(np.linalg.det(Md)), th))
    return th0, out


# ---------------------------------------------------------------------------
# direct route: an inverse and the Cholesky-form energy per determinant
# ---------------------------------------------------------------------------

def energy_multidet_exact(h, L, C, dets, coeffs, phi, e0: float = 0.0):
    """sum_d c_d <Phi_d|phi> E_d / sum_d c_d <Phi_d|phi>, each E_d the exact
    closed-shell local energy of determinant d (E.energy_cholesky), each overlap
    from its LU log-determinant (both spins)."""
    Es, lds = [], []
    for det in dets:
        Pd = occupied(C, det)
        r = E.energy_cholesky(h, L, Pd, Pd, phi, phi, e0)
        Es.append(r["E"])
        lds.append(r["logdet"])
    lds = np.array(lds)
    w = np.asarray(coeffs) * np.exp(lds - lds[0])
    return complex(np.sum(w * np.array(Es)) / np.sum(w)), w / np.sum(w), np.array(Es)


# ---------------------------------------------------------------------------
# 3-4. LO energy through the SMW intermediates
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class CASPrep:
    """Localized CAS orbitals, their half-rotated Cholesky vectors and the
    truncated factors of every orbital pair among them."""

    C: np.ndarray
    Lbar: np.ndarray              # (X, n_cas, M)
    hbar: np.ndarray              # (n_cas, M)
    factors: LO.PairFactors
    pair_index: dict              # (i, j), i <= j -> index into factors


def prepare_cas(mol, cas, threshold: float, localize: bool = True) -> CASPrep:
    C = localize_inactive(cas.C, cas.n_inact, mol.orbital_pos) if localize else np.array(cas.C)
    Lbar = E.half_rotate(mol.L, C)
    fac = LO.truncate(LO.pair_svds(Lbar), threshold)
    return CASPrep(C, Lbar, C.conj().T @ mol.h, fac, {p: n for n, p in enumerate(fac.pairs)})


def _pair_factors(prep: CASPrep, i: int, j: int):
    """(Ubar^[ij], Vbar^[ij]) for any order: Y^[ji] = Y^[ij]T, so the [ji]
    factors are the transposed, exchanged [ij] ones."""
    if i <= j:
        n = prep.pair_index[(i, j)]
        return prep.factors.U[n], prep.factors.V[n]
    n = prep.pair_index[(j, i)]
    return prep.factors.V[n].T, prep.factors.U[n].T


def energy_multidet_lo(mol, cas, prep: CASPrep, phi: np.ndarray, e0: float = 0.0,
                       coulomb: str = "exact"):
    """Mixed-estimate LO local energy of a closed-shell walker phi (M x N).

    Exchange per determinant: E_K^d = sum_{s,t} e^d_st with
    e^d_st = (Ubar^[ij]T Q^d_t) . (Vbar^[ij] Q^d_s), (i, j) the orbitals in
    slots (s, t); the projected columns come from eq. BigQ.  One-body and exact
    Coulomb from Q^d; ``coulomb="compressed"`` takes the Coulomb from the pair
    factors (the 4 Q_ri Q_sj term of eq. 2e_HR_RCAS).
    """
    dets = cas.dets
    N = cas.N
    th0, smw = smw_thetas(prep.C, dets, phi)
    # projections of every reference column for every orbital pair met in a determinant
    proj = {}

    def projections(i, j):
        if (i, j) not in proj:
            U, V = _pair_factors(prep, i, j)
            proj[(i, j)] = (U.T @ th0, V @ th0)     # (K, N) each
        return proj[(i, j)]

    Es = []
    for d, det in enumerate(dets):
        sd = smw[d]
        th = sd.theta
        e1 = 2.0 * sum(np.dot(prep.hbar[det[s]], th[:, s]) for s in range(N))
        J = 2.0 * np.einsum("gsr,rs->g", prep.Lbar[:, det, :], th, optimize=True)
        ek = 0j
        ejc = 0j
        for s in range(N):
            for t in range(N):
                i, j = det[s], det[t]
                PL, PR = projections(i, j)
                # eq. BigQ: reference projection minus the excited-slot correction
                qL_t = PL[:, t] - PL[:, sd.slots] @ sd.S[:, t] if sd.slots else PL[:, t]
                qR_s = PR[:, s] - PR[:, sd.slots] @ sd.S[:, s] if sd.slots else PR[:, s]
                ek += np.dot(qL_t, qR_s)
                if coulomb == "compressed":
                    qL_s = PL[:, s] - PL[:, sd.slots] @ sd.S[:, s] if sd.slots else PL[:, s]
                    qR_t = PR[:, t] - PR[:, sd.slots] @ sd.S[:, t] if sd.slots else PR[:, t]
                    ejc += np.dot(qL_s, qR_t)
        if coulomb == "exact":
            ej = 0.5 * np.sum(J * J)
        elif coulomb == "compressed":
            ej = 2.0 * ejc
        else:
            raise ValueError(coulomb)
        Es.append(e0 + e1 + ej - ek)
    ratios = np.array([s.ratio for s in smw])
    w = np.asarray(cas.coeffs) * ratios ** 2        # c_d <Phi_d|phi> / <Phi_0|phi>
    w = w / np.sum(w)
    return complex(np.sum(w * np.array(Es))), w, np.array(Es)


def truncation_bound_multidet(cas, prep: CASPrep, phi: np.ndarray, weights: np.ndarray) -> float:
    """sum_d |w_d| sum_{s,t} s_drop^[ij] |Q^d_s| |Q^d_t|: every dropped part of a
    block has spectral norm below its first dropped singular value."""
    _, smw = smw_thetas(prep.C, cas.dets, phi)
    drop = {}
    for n, (i, j) in enumerate(prep.factors.pairs):
        s = prep.factors.sigma[n]
        k = prep.factors.U[n].shape[1]
        drop[(i, j)] = drop[(j, i)] = float(s[k]) if k < len(s) else 0.0
    b = 0.0
    for d, det in enumerate(cas.dets):
        nrm = np.linalg.norm(smw[d].theta, axis=0)
        bd = sum(drop[(det[s], det[t])] * nrm[s] * nrm[t]
                 for s in range(cas.N) for t in range(cas.N))
        b += abs(weights[d]) * bd
    return b

"""Localized-orbital (LO) energy, plain FP64 (test infrastructure).

Steps, in the paper's order (Sec. 3.1 and 4):
  1. Foster-Boys localization of the occupied trial orbitals (Sec. 4); the
     synthetic basis is orthonormal with a diagonal position operator.
  2. Half-rotated Cholesky vectors with the localized orbitals (Sec. 2.2).
  3. For every orbital pair [ij] the M x M block Y^[ij]_rs = sum_g Lbar^g_ir
     Lbar^g_js of the half-rotated ERI tensor (eq. 2e_HRERI_RCAS), its SVD,
     and truncation under the single threshold T_SVD (Sec. 3.1.1):
     Y^[ij] ~= Ubar Vbar with Ubar = U_K sqrt(s_K), Vbar = sqrt(s_K) V_K^T over
     the singular values s_K >= T_SVD.
  4. The exchange through dot products of projected vectors
     Qbar_L = Ubar^T Theta_j and Qbar_R = Vbar Theta_i (eqs. 2e_HR_RCAS_LO,
     2e_HR_RCAS): e_ij = Qbar_L . Qbar_R.

Only the test suite, the smoke check and the CPU baseline of the benchmark use
this module.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Tuple

import numpy as np

from . import energy as E


# ---------------------------------------------------------------------------
# 1. Foster-Boys localization by Jacobi sweeps
# ---------------------------------------------------------------------------

def boys_objective(C: np.ndarray, pos: np.ndarray) -> float:
    """sum_i sum_d <i|r_d|i>^2 with r_d = diag(pos[:, d]) (orthonormal AO basis)."""
    return float(sum(np.sum((np.einsum("pi,p,pi->i", C, pos[:, d], C)) ** 2)
                     for d in range(pos.shape[1])))


def boys_localize(C: np.ndarray, pos: np.ndarray, angle_tol: float = 1e-13,
                  max_sweeps: int = 1000) -> Tuple[np.ndarray, List[float]]:
    """Maximise the Boys objective by 2x2 Jacobi rotations of orbital pairs.

    For pair (i, j) and each coordinate d let a = R_ii, b = R_jj, m = R_ij with
    R = C^T r_d C.  Rotating i' = c i + s j, j' = -s i + c j (c = cos t,
    s = sin t) changes R'_ii^2 + R'_jj^2 by
        P cos 4t + Q sin 4t + const,  P = sum_d ((a-b)^2/4 - m^2),
                                      Q = sum_d (a-b) m,
    which is largest at 4t = atan2(Q, P).  Pairs are visited in the order
    (0,1), (0,2), ..., (N-2,N-1); sweeps stop when the largest |t| in a sweep
    is below ``angle_tol``.  Returns the rotated orbitals and the objective
    after each sweep (non-decreasing).
    """
    C = np.array(C, dtype=np.float64, copy=True)
    M, N = C.shape
    history = [boys_objective(C, pos)]
    if N < 2:
        return C, history
    # R[d] = C^T diag(x_d) C, updated alongside C
    R = np.stack([C.T @ (pos[:, d:d + 1] * C) for d in range(pos.shape[1])])
    for _ in range(max_sweeps):
        biggest = 0.0
        for i in range(N - 1):
            for j in range(i + 1, N):
                a = R[:, i, i]
                b = R[:, j, j]
                m = R[:, i, j]
                P = np.sum(0.25 * (a - b) ** 2 - m ** 2)
                Q = np.sum((a - b) * m)
                t = 0.25 * np.arctan2(Q, P)
                if t == 0.0:
                    continue
                biggest = max(biggest, abs(t))
                c, s = np.cos(t), np.sin(t)
                ci, cj = C[:, i].copy(), C[:, j].copy()
                C[:, i] = c * ci + s * cj
                C[:, j] = -s * ci + c * cj
                Ri, Rj = R[:, :, i].copy(), R[:, :, j].copy()
                R[:, :, i] = c * Ri + s * Rj
                R[:, :, j] = -s * Ri + c * Rj
                Ri, Rj = R[:, i, :].copy(), R[:, j, :].copy()
                R[:, i, :] = c * Ri + s * Rj
                R[:, j, :] = -s * Ri + c * Rj
        history.append(boys_objective(C, pos))
        if biggest < angle_tol:
            break
    return C, history


# ---------------------------------------------------------------------------
# 3. blockwise pair SVD and truncation
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class PairFactors:
    """Truncated factors of every block Y^[ij], i <= j, for one spin."""

    pairs: List[Tuple[int, int]]
    U: List[np.ndarray]          # Ubar^[ij], M x K_ij
    V: List[np.ndarray]          # Vbar^[ij], K_ij x M
    sigma: List[np.ndarray]      # all M singular values, descending
    threshold: float

    @property
    def m_svd(self) -> np.ndarray:
        return np.array([u.shape[1] for u in self.U], dtype=np.int64)

    def compression_pct(self, M: int) -> float:
        """(M - <M_SVD>) / M * 100, the paper's compression efficiency (Sec. 4)."""
        return float((M - self.m_svd.mean()) / M * 100.0)


def pair_block(Lbar: np.ndarray, i: int, j: int) -> np.ndarray:
    """Y^[ij]_rs = sum_g Lbar^g_ir Lbar^g_js (the [ij] block of eq. 2e_HRERI_RCAS)."""
    return Lbar[:, i, :].T @ Lbar[:, j, :]


def pair_svds(Lbar: np.ndarray):
    """Full SVD (LAPACK gesdd through numpy) of every pair block, i <= j."""
    N = Lbar.shape[1]
    out = []
    for i in range(N):
        for j in range(i, N):
            U, s, Vt = np.linalg.svd(pair_block(Lbar, i, j))
            out.append(((i, j), U, s, Vt))
    return out


def truncate(svds, threshold: float, keep: Optional[np.ndarray] = None) -> PairFactors:
    """Keep singular values s >= threshold (all of them at threshold 0).

    ``keep``, when given, fixes the kept count per pair instead (used only to
    report how a different count at a near-threshold pair would change E).
    """
    pairs, U, V, sig = [], [], [], []
    for n, ((i, j), u, s, vt) in enumerate(svds):
        k = int(np.sum(s >= threshold)) if keep is None else int(keep[n])
        r = np.sqrt(s[:k])
        pairs.append((i, j))
        U.append(u[:, :k] * r[None, :])
        V.append(r[:, None] * vt[:k])
        sig.append(s)
    return PairFactors(pairs, U, V, sig, threshold)


# ---------------------------------------------------------------------------
# 4. LO energy
# ---------------------------------------------------------------------------

def pair_exchange(fac: PairFactors, th: np.ndarray) -> np.ndarray:
    """e_ij = (Ubar^[ij]T Theta_j) . (Vbar^[ij] Theta_i), unconjugated, for i <= j."""
    out = np.zeros(len(fac.pairs), dtype=np.complex128)
    for n, (i, j) in enumerate(fac.pairs):
        a = fac.U[n].T @ th[:, j]
        b = fac.V[n] @ th[:, i]
        out[n] = np.dot(a, b)
    return out


def pair_exchange_streamed(Lbar: np.ndarray, keep: np.ndarray, ths: np.ndarray,
                           workers: int = 1) -> np.ndarray:
    """e_ij(w) of every pair i <= j and every walker, one pair at a time.

    The same steps as pair_svds, truncate and pair_exchange: for pair n = [ij]
    (the order of pair_svds) form Y^[ij] (eq. 2e_HRERI_RCAS), take its SVD,
    keep its keep[n] largest singular values (Sec. 3.1.1) and return
    e_ij(w) = (Ubar^T Theta_j(w)) . (Vbar Theta_i(w)) for every Theta(w) in
    ths (W x M x N).  Only the pair values are kept, not every pair's factors
    (about 8 GB at M = 440, N = 73).  workers > 1 maps the pairs over threads
    (NumPy's LAPACK and BLAS calls release the GIL); the values do not depend
    on it.  Returns an (n_pairs, W) complex array.
    """
    N = Lbar.shape[1]
    pairs = [(i, j) for i in range(N) for j in range(i, N)]
    if len(keep) != len(pairs):
        raise ValueError("one kept rank per pair i <= j")
    cols = np.ascontiguousarray(np.transpose(ths, (2, 1, 0)))  # [orbital][r][w]

    def one(n):
        i, j = pairs[n]
        U, s, Vt = np.linalg.svd(pair_block(Lbar, i, j))
        k = int(keep[n])
        r = np.sqrt(s[:k])
        a = (U[:, :k] * r[None, :]).T @ cols[j]
        b = (r[:, None] * Vt[:k]) @ cols[i]
        return np.sum(a * b, axis=0)

    if workers <= 1:
        rows = [one(n) for n in range(len(pairs))]
    else:
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(workers) as ex:
            rows = list(ex.map(one, range(len(pairs))))
    return np.array(rows, dtype=np.complex128).reshape(len(pairs), ths.shape[0])


def exchange_lo(fac: PairFactors, th: np.ndarray, mask: Optional[np.ndarray] = None) -> complex:
    """sum_ij e_ij = sum_i e_ii + 2 sum_{i<j} e_ij (Y^[ji] = Y^[ij]T), one spin.

    ``mask`` (bool per pair) drops screened pairs.
    """
    e = pair_exchange(fac, th)
    w = np.array([1.0 if i == j else 2.0 for i, j in fac.pairs])
    if mask is not None:
        w = w * mask
    return complex(np.sum(w * e))


def coulomb_lo(fac: PairFactors, th: np.ndarray) -> complex:
    """sum_ij (Ubar^[ij]T Theta_i) . (Vbar^[ij] Theta_j) over ordered pairs, one spin.

    The compressed Coulomb of eq. 2e_HR_RCAS (the 4 Q_ri Q_sj term).  The [ji]
    block is the transpose of [ij], so the (j, i) term equals the (i, j) term
    and the sum is d_ii + 2 sum_{i<j} d_ij.
    """
    tot = 0j
    for n, (i, j) in enumerate(fac.pairs):
        d = np.dot(fac.U[n].T @ th[:, i], fac.V[n] @ th[:, j])
        tot += d if i == j else 2.0 * d
    return tot


@dataclasses.dataclass
class LOSpin:
    """Everything one spin channel needs: localized trial, Lbar, factors."""

    trial_loc: np.ndarray
    Lbar: np.ndarray
    svds: list
    factors: PairFactors


def prepare_spin(L: np.ndarray, trial: np.ndarray, pos: np.ndarray,
                 threshold: float, localize: bool = True) -> LOSpin:
    C = boys_localize(trial, pos)[0] if localize else np.array(trial)
    Lbar = E.half_rotate(L, C)
    svds = pair_svds(Lbar)
    return LOSpin(C, Lbar, svds, truncate(svds, threshold))


def prepare(mol, threshold: float, localize: bool = True) -> List[LOSpin]:
    """Localize, half-rotate and compress both spins of a synthetic molecule."""
    pos = mol.orbital_pos
    sa = prepare_spin(mol.L, mol.trial_a, pos, threshold, localize)
    if mol.closed_shell:
        return [sa]
    return [sa, prepare_spin(mol.L, mol.trial_b, pos, threshold, localize)]


def energy_lo(mol, spins: List[LOSpin], phi: np.ndarray, e0: float = 0.0,
              coulomb: str = "exact", masks=None):
    """LO local energy of one packed walker.

    E = E1 + E_J - E_K^LO, E1 and the Coulomb E_J exact through the Cholesky
    vectors (eq. 2e_HRchol_RCAS), the exchange E_K^LO = 1/2 sum_sigma sum_ij
    e^sigma_ij from the truncated pair factors (eq. 2e_HR_RCAS_LO, the
    -2 Q_si Q_rj term with the 1/2 in front).  ``coulomb="compressed"`` takes
    the closed-shell Coulomb from the same factors (the 4 Q_ri Q_sj term).
    The trial enters through the localized orbitals; Theta and the energy do
    not depend on that rotation (eq. GwQ).
    """
    pa, pb = E.split_walker(mol, phi)
    if mol.closed_shell:
        per_spin = [(spins[0], pa), (spins[0], pb)]
    else:
        per_spin = [(spins[0], pa), (spins[1], pb)]
    e1 = 0j
    J = np.zeros(mol.X, dtype=np.complex128)
    ek = 0j
    ths = []
    for n, (sp, ph) in enumerate(per_spin):
        th = E.theta(sp.trial_loc, ph)
        ths.append(th)
        e1 += np.sum((sp.trial_loc.conj().T @ mol.h) * th.T)
        J += np.einsum("gir,ri->g", sp.Lbar, th, optimize=True)
        m = None if masks is None else masks[0 if mol.closed_shell else n]
        ek += 0.5 * exchange_lo(sp.factors, th, m)
    if coulomb == "exact":
        ej = 0.5 * np.sum(J * J)
    elif coulomb == "compressed":
        if not mol.closed_shell:
            raise ValueError("compressed Coulomb is defined here for closed shells")
        ej = 2.0 * coulomb_lo(spins[0].factors, ths[0])
    else:
        raise ValueError(coulomb)
    return dict(E=e0 + e1 + ej - ek, E1=e1, EJ=ej, EK=ek)


def truncation_bound(fac: PairFactors, th: np.ndarray) -> float:
    """Upper bound on |sum_ij e_ij(T) - sum_ij e_ij(0)| for one spin.

    Each dropped block part sum_{s_K < T} s_K u_K v_K^T has spectral norm below
    the first dropped singular value, so |e_ij(T) - e_ij(0)| <= s_drop |Theta_j| |Theta_i|;
    weights 1 (i = j) and 2 (i < j) as in exchange_lo.
    """
    nrm = np.linalg.norm(th, axis=0)
    b = 0.0
    for n, (i, j) in enumerate(fac.pairs):
        k = fac.U[n].shape[1]
        s = fac.sigma[n]
        if k < len(s):
            b += (1.0 if i == j else 2.0) * s[k] * nrm[i] * nrm[j]
    return b

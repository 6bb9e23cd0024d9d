"""Seeded synthetic molecule-shaped inputs for the local-energy path.

This module only draws inputs: site geometries, the one-body matrix h, the
Cholesky vectors L, the trial determinant and the walkers.  It holds none of
the local-energy arithmetic, so both the CPU oracle (through the tests) and
the CUDA library consume exactly the same bytes.

The paper's workloads are real molecules (dodecane, ferrocene, polyacenes,
platonic cages; Sec. 4).  Their integrals are not available, so these
generators stand in for them at the paper's sizes (M of a few hundred basis
functions, X between 4M and 10M Cholesky vectors, Sec. 2.1.1) and with the
paper's locality premise (distant localized orbitals interact through low-rank
blocks, Sec. 3.1.1).

Recipe (all lengths in units of one bond):
  * three orbitals per site; n_sites = ceil(M_lig / 3), the last site takes the
    remainder; an optional central "metal" site carries its own orbital count;
  * h_pq = -exp(-|x_p - x_q|)
  * L^g_pq = s_pq * exp(-|x_p - x_q| / l_pq) * exp(-g / M), g = 0..X-1, with
    s symmetric standard normal (upper triangle drawn row by row, mirrored),
    l_pq = 2.0, or the metal length when p or q sits on the metal site;
  * trial per spin = the lowest n_sigma eigenvectors of h (numpy eigh);
  * walker (per spin) = Q of the QR of expm(i eps A) Phi_T with
    A = (G + G^H)/sqrt(2M), G = (N(0,1) + i N(0,1))/sqrt(2), M x M (the
    Wigner normalisation: A's spectrum lies near [-2, 2], so eps sets the size
    of the perturbation); raw_gaussian=True uses A = (G + G^H)/2 instead.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

# ---------------------------------------------------------------------------
# geometries
# ---------------------------------------------------------------------------


def chain_sites(n_sites: int) -> np.ndarray:
    """Sites at unit spacing on the x axis."""
    x = np.zeros((n_sites, 3))
    x[:, 0] = np.arange(n_sites, dtype=np.float64)
    return x


def fragment_sites(n_sites: int, n_frag: int, gap: float) -> np.ndarray:
    """n_frag chains on the x axis (unit spacing), consecutive chains ``gap``
    bonds apart; the sites are split as evenly as possible, the first chains
    taking the remainder."""
    sizes = [n_sites // n_frag + (1 if f < n_sites % n_frag else 0) for f in range(n_frag)]
    x = np.zeros((n_sites, 3))
    k, x0 = 0, 0.0
    for n in sizes:
        x[k:k + n, 0] = x0 + np.arange(n, dtype=np.float64)
        x0 += (n - 1) + gap
        k += n
    return x


def acene_sites(n_sites: int) -> np.ndarray:
    """A linear acene ribbon (rings fused side by side along x), unit bonds.

    A ribbon of n rings has 4n+2 sites: the apex pair (top, bottom) of each
    ring and the two atoms of every shared vertical bond.  Enough rings are
    generated and the first ``n_sites`` sites in (x, y) order are kept.
    """
    n_rings = max(1, math.ceil((n_sites - 2) / 4))
    s3 = math.sqrt(3.0)
    pts = []
    for k in range(n_rings):
        pts.append((k * s3, 1.0))
        pts.append((k * s3, -1.0))
    for k in range(n_rings + 1):
        pts.append((k * s3 - s3 / 2, 0.5))
        pts.append((k * s3 - s3 / 2, -0.5))
    pts.sort(key=lambda p: (round(p[0], 9), -p[1]))
    x = np.zeros((n_sites, 3))
    x[:, :2] = np.asarray(pts[:n_sites])
    return x


def honeycomb_patch_sites(n_sites: int) -> np.ndarray:
    """The ``n_sites`` honeycomb sites closest to one ring centre (unit bond).

    This is the most compact patch of fused hexagons with that many sites;
    ties in distance are broken by polar angle, then by coordinates.
    """
    s3 = math.sqrt(3.0)
    a1 = np.array([s3, 0.0])
    a2 = np.array([s3 / 2, 1.5])
    # two sublattices; the hexagon around the origin has vertices (0, +-1)
    basis = [np.array([0.0, 1.0]), np.array([0.0, -1.0])]
    n_cells = int(math.ceil(math.sqrt(n_sites))) + 3
    pts = set()
    for i in range(-n_cells, n_cells + 1):
        for j in range(-n_cells, n_cells + 1):
            for b in basis:
                p = i * a1 + j * a2 + b
                pts.add((round(p[0], 9), round(p[1], 9)))
    pts = sorted(pts, key=lambda p: (round(math.hypot(*p), 7),
                                     round(math.atan2(p[1], p[0]), 7), p))
    x = np.zeros((n_sites, 3))
    x[:, :2] = np.asarray(pts[:n_sites])
    return x


def sphere_sites(n_sites: int, radius: float, seed: int) -> np.ndarray:
    """Sites drawn uniformly on a sphere (normalised Gaussian directions)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((n_sites, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return radius * v


# ---------------------------------------------------------------------------
# molecule + walkers
# ---------------------------------------------------------------------------


@dataclasses.dataclass
class Molecule:
    """One synthetic system: everything the energy path takes as input."""

    name: str
    M: int
    X: int
    n_alpha: int
    n_beta: int
    h: np.ndarray             # (M, M) float64, symmetric
    L: np.ndarray             # (X, M, M) float64, each slice symmetric
    trial_a: np.ndarray       # (M, n_alpha) float64, orthonormal columns
    trial_b: np.ndarray       # (M, n_beta) float64
    site_of: np.ndarray       # (M,) int, site index of each orbital
    pos: np.ndarray           # (n_sites_total, 3) site positions
    gap: float                # HOMO-LUMO gap of h for the larger spin
    degenerate: bool          # gap below 1e-8

    @property
    def closed_shell(self) -> bool:
        return self.n_alpha == self.n_beta

    @property
    def orbital_pos(self) -> np.ndarray:
        return self.pos[self.site_of]


def _orbital_sites(n_lig_orb: int, metal_orbitals: int) -> Tuple[np.ndarray, int]:
    n_sites = math.ceil(n_lig_orb / 3)
    site_of = np.repeat(np.arange(n_sites), 3)[:n_lig_orb]
    if metal_orbitals:
        site_of = np.concatenate([site_of, np.full(metal_orbitals, n_sites)])
    return site_of, n_sites


def make_molecule(name: str, M: int, X: int, n_alpha: int, n_beta: int,
                  geometry: str, seed: int, decay: float = 2.0,
                  metal_orbitals: int = 0, metal_decay: float = 4.0,
                  sphere_radius: float = 3.0, geom_seed: int = 0, n_frag: int = 2,
                  frag_gap: float = 20.0) -> Molecule:
    """Draw h, L and the trial for one synthetic molecule.

    ``geometry`` is one of "chain", "honeycomb", "acene", "cage", "fragments".
    For "cage" the ligand sites lie on a sphere of ``sphere_radius`` and, when
    ``metal_orbitals`` > 0, one metal site sits at the centre.  "fragments" is
    ``n_frag`` chains ``frag_gap`` bonds apart (separate molecules in one system:
    with ``decay`` well below the gap, h and L couple them negligibly).
    """
    n_lig = M - metal_orbitals
    site_of, n_sites = _orbital_sites(n_lig, metal_orbitals)
    if geometry == "chain":
        pos = chain_sites(n_sites)
    elif geometry == "acene":
        pos = acene_sites(n_sites)
    elif geometry == "honeycomb":
        pos = honeycomb_patch_sites(n_sites)
    elif geometry == "cage":
        pos = sphere_sites(n_sites, sphere_radius, geom_seed)
    elif geometry == "fragments":
        pos = fragment_sites(n_sites, n_frag, frag_gap)
    else:
        raise ValueError(f"unknown geometry {geometry!r}")
    if metal_orbitals:
        pos = np.vstack([pos, np.zeros((1, 3))])
    xo = pos[site_of]
    dist = np.linalg.norm(xo[:, None, :] - xo[None, :, :], axis=-1)

    h = -np.exp(-dist)

    ell = np.full((M, M), decay)
    if metal_orbitals:
        on_metal = site_of == n_sites
        ell[on_metal, :] = metal_decay
        ell[:, on_metal] = metal_decay
    env = np.exp(-dist / ell)

    rng = np.random.default_rng(seed)
    iu = np.triu_indices(M)
    L = np.empty((X, M, M))
    # draw in gamma order, one upper triangle (row by row) per vector
    chunk = max(1, int(2e7 // len(iu[0])))
    for g0 in range(0, X, chunk):
        g1 = min(X, g0 + chunk)
        draws = rng.standard_normal((g1 - g0, len(iu[0])))
        blk = np.zeros((g1 - g0, M, M))
        blk[:, iu[0], iu[1]] = draws
        blk = blk + np.triu(blk, 1).transpose(0, 2, 1)
        scale = np.exp(-np.arange(g0, g1, dtype=np.float64) / M)
        L[g0:g1] = blk * env[None] * scale[:, None, None]

    evals, evecs = np.linalg.eigh(h)
    nmax = max(n_alpha, n_beta)
    gap = float(evals[nmax] - evals[nmax - 1]) if nmax < M else float("inf")
    trial_a = np.ascontiguousarray(evecs[:, :n_alpha])
    trial_b = np.ascontiguousarray(evecs[:, :n_beta])
    return Molecule(name=name, M=M, X=X, n_alpha=n_alpha, n_beta=n_beta, h=h,
                    L=L, trial_a=trial_a, trial_b=trial_b, site_of=site_of,
                    pos=pos, gap=gap, degenerate=gap < 1e-8)


def _expm_i_herm_times(A: np.ndarray, eps: float, B: np.ndarray) -> np.ndarray:
    """exp(i eps A) @ B for Hermitian A, through A's eigendecomposition."""
    lam, V = np.linalg.eigh(A)
    return V @ (np.exp(1j * eps * lam)[:, None] * (V.conj().T @ B))


def _one_walker(trials: Sequence[np.ndarray], eps: float, seed: int,
                scale_sq: float, far: Optional[np.ndarray] = None) -> List[np.ndarray]:
    rng = np.random.default_rng(seed)
    out = []
    M = trials[0].shape[0]
    for T in trials:
        G = (rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))) / math.sqrt(2.0)
        A = (G + G.conj().T) / math.sqrt(2.0 * M * scale_sq)
        if far is not None:
            A[far] = 0.0  # a local perturbation: no coupling beyond the band
        q, _ = np.linalg.qr(_expm_i_herm_times(A, eps, T.astype(np.complex128)))
        out.append(np.ascontiguousarray(q))
    return out


def _walker_job(args):
    return _one_walker(*args)


def make_walkers(mol: Molecule, W: int, eps: float, seed0: int,
                 first: int = 0, processes: int = 0,
                 raw_gaussian: bool = False, band: Optional[float] = None) -> np.ndarray:
    """Walkers ``first`` .. ``first+W-1`` of a molecule, packed per walker.

    Returns a complex128 array of shape (W, M, n_alpha + n_beta) for an open
    shell and (W, M, n_alpha) for a closed shell (one restricted determinant
    serves both spins).  Walker w uses seed ``seed0 + w``.  ``band`` (bonds),
    when given, zeroes A between basis functions whose sites are farther apart
    (the same draws, a local perturbation).  ``processes`` > 1 spreads the
    draws over a spawn-started process pool; the result does not depend on it.
    """
    trials = [mol.trial_a] if mol.closed_shell else [mol.trial_a, mol.trial_b]
    scale_sq = 2.0 / mol.M if raw_gaussian else 1.0
    far = None
    if band is not None:
        xo = mol.pos[mol.site_of]
        far = np.linalg.norm(xo[:, None, :] - xo[None, :, :], axis=-1) > band
    jobs = [(trials, eps, seed0 + w, scale_sq, far) for w in range(first, first + W)]
    if processes and processes > 1 and W > 8:
        import multiprocessing as mp
        import os
        ctx = mp.get_context("spawn")
        saved = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS")}
        os.environ["OPENBLAS_NUM_THREADS"] = "1"  # one BLAS thread per worker
        os.environ["OMP_NUM_THREADS"] = "1"
        try:
            with ctx.Pool(processes) as pool:
                res = pool.map(_walker_job, jobs, chunksize=max(1, W // (4 * processes)))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
    else:
        res = [_walker_job(j) for j in jobs]
    return np.stack([np.concatenate(r, axis=1) for r in res])


# ---------------------------------------------------------------------------
# the five workloads
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    M: int
    n_alpha: int
    n_beta: int
    X: int
    W: int
    eps: float
    geometry: str
    seed: int
    walker_seed: int
    metal_orbitals: int = 0
    geom_seed: int = 0
    decay: float = 2.0
    n_frag: int = 2
    frag_gap: float = 20.0
    band: Optional[float] = None  # walkers: local perturbation (bonds)

    def molecule(self) -> Molecule:
        return make_molecule(self.name, self.M, self.X, self.n_alpha, self.n_beta,
                             self.geometry, self.seed, decay=self.decay,
                             metal_orbitals=self.metal_orbitals,
                             geom_seed=self.geom_seed, n_frag=self.n_frag,
                             frag_gap=self.frag_gap)

    def walkers(self, mol: Molecule, W: Optional[int] = None, first: int = 0,
                processes: int = 0, raw_gaussian: bool = False) -> np.ndarray:
        return make_walkers(mol, self.W if W is None else W, self.eps,
                            self.walker_seed, first=first, processes=processes,
                            raw_gaussian=raw_gaussian, band=self.band)


# Workload sizes (M basis functions, N occupied per spin, X Cholesky vectors,
# W walkers) follow the paper's size range.
CHAIN_60 = Workload("chain_M60_N10_X240", 60, 10, 10, 240, 32, 0.05, "chain", 1001, 2001)
NAPHTHALENE_250 = Workload("honeycomb_M250_N34_X1000", 250, 34, 34, 1000, 512, 0.1,
                           "honeycomb", 1002, 2002)
PENTACENE_440 = Workload("acene_M440_N73_X1800", 440, 73, 73, 1800, 1024, 0.1,
                         "acene", 1003, 2003)
# a small system with the pentacene-scale occupied count (N = 73, five column
# slots of the inverse kernels) and 1024 walkers, for kernel profiles
PROFILE_N73 = Workload("acene_M220_N73_X440", 220, 73, 73, 440, 1024, 0.1, "acene", 1060, 2060)
HETERO_BATCH = [
    Workload(f"acene_M{M}_N{N}_X{X}", M, N, N, X, W, 0.1, "acene", 1040 + k, 2040 + 10000 * k)
    for k, (M, N, X, W) in enumerate([(100, 14, 400, 512), (180, 25, 720, 512),
                                      (250, 34, 1000, 256), (320, 44, 1300, 256),
                                      (400, 60, 1600, 128), (480, 80, 1900, 128)])
]
METALLOCENE_500 = Workload("cage_M500_Na48_Nb47_X2000", 500, 48, 47, 2000, 2048, 0.1,
                           "cage", 1005, 2005, metal_orbitals=15, geom_seed=3005)

# Separate fragments in one system, for the learned pair screen (Sec. 5): four
# chains 20 bonds apart with short-range Cholesky vectors (decay 0.5) and walkers
# perturbed within 3 bonds, so that every pair of orbitals on different
# fragments contributes below 1e-6 Ha although its truncated block keeps its rank.
FRAGMENTS_480 = Workload("fragments4_M480_N80_X960", 480, 80, 80, 960, 1024, 0.3, "fragments",
                         1007, 2007, decay=0.5, n_frag=4, frag_gap=20.0, band=3.0)

WORKLOADS = {w.name: w for w in [CHAIN_60, NAPHTHALENE_250, PENTACENE_440, PROFILE_N73,
                                 METALLOCENE_500, FRAGMENTS_480, *HETERO_BATCH]}


def small_case(M: int, N: int, X: int, W: int, seed: int = 7, eps: float = 0.1,
               geometry: str = "chain", n_beta: Optional[int] = None):
    """A small seeded system of arbitrary (ragged) shape for parity tests."""
    nb = N if n_beta is None else n_beta
    mol = make_molecule(f"small_M{M}_N{N}_X{X}", M, X, N, nb, geometry, seed)
    walk = make_walkers(mol, W, eps, seed * 1000 + 1)
    return mol, walk


# ---------------------------------------------------------------------------
# multi-determinant (CAS) trial
# ---------------------------------------------------------------------------


@dataclasses.dataclass
class CASTrial:
    """A closed-shell multi-determinant trial sum_d c_d |Phi_d>.

    C holds the n_inact inactive orbitals followed by the n_act active ones
    (orthonormal columns).  Every determinant occupies N = n_inact + n_occ_act
    spatial orbitals, listed by slot: the reference occupies orbitals 0..N-1 in
    slot order, and an excited determinant puts each new active orbital in the
    slot of the reference orbital it replaces.  dets[0] is the reference.
    """

    C: np.ndarray                 # (M, n_inact + n_act)
    n_inact: int
    n_act: int
    N: int                        # occupied orbitals per spin (both spins alike)
    dets: List[List[int]]         # per determinant: orbital index of each slot
    coeffs: np.ndarray            # (n_det,) float64

    @property
    def n_det(self) -> int:
        return len(self.dets)

    @property
    def max_excitation(self) -> int:
        ref = self.dets[0]
        return max(sum(1 for a, b in zip(d, ref) if a != b) for d in self.dets)


def make_cas_trial(mol: Molecule, n_inact: int, n_act: int, n_det: int, max_exc: int,
                   seed: int) -> CASTrial:
    """A seeded CAS-like expansion on the lowest eigenvectors of h.

    Orbitals: the lowest n_inact + n_act eigenvectors of h.  The reference
    occupies the lowest N = mol.n_alpha of them; the other determinants replace
    1..max_exc of the reference's active orbitals by virtual active ones, drawn
    without repetition (seeded).  Coefficients: c_0 = 1, the rest N(0, 1)
    scaled by 0.3 / (1 + rank).  Closed shell only.
    """
    if mol.n_alpha != mol.n_beta:
        raise ValueError("the CAS trial is built for closed shells")
    N = mol.n_alpha
    if not (0 <= n_inact < N < n_inact + n_act <= mol.M):
        raise ValueError("need n_inact < N < n_inact + n_act <= M")
    evals, evecs = np.linalg.eigh(mol.h)
    C = np.ascontiguousarray(evecs[:, :n_inact + n_act])
    ref = list(range(N))
    occ_act = list(range(n_inact, N))          # active orbitals occupied in the reference
    virt_act = list(range(N, n_inact + n_act))  # active orbitals empty in the reference
    rng = np.random.default_rng(seed)
    dets, seen = [ref], {tuple(ref)}
    kmax = min(max_exc, len(occ_act), len(virt_act))
    tries = 0
    while len(dets) < n_det and tries < 100 * n_det:
        tries += 1
        k = int(rng.integers(1, kmax + 1))
        out = sorted(rng.choice(occ_act, size=k, replace=False).tolist())
        inn = rng.choice(virt_act, size=k, replace=False).tolist()
        d = list(ref)
        for o, a in zip(out, inn):
            d[ref.index(o)] = int(a)
        if tuple(d) not in seen:
            seen.add(tuple(d))
            dets.append(d)
    coeffs = np.empty(len(dets))
    coeffs[0] = 1.0
    coeffs[1:] = rng.standard_normal(len(dets) - 1) * 0.3 / (1.0 + np.arange(1, len(dets)))
    return CASTrial(C=C, n_inact=n_inact, n_act=n_act, N=N, dets=dets, coeffs=coeffs)

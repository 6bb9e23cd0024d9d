"""Multi-determinant (CAS) trial on the GPU against the oracle, through the C ABI.

The context is loaded with the CAS orbitals (inactive block Boys-localized by
the oracle, as the caller would) and compressed without localization; the
library's energies and log overlaps are compared with the oracle's SMW route
(FP64: 1e-10 relative), at T_SVD = 0 and, with the library's kept ranks fed to
the oracle, at T_SVD = 1e-2.
"""
import numpy as np
import pytest

from oracle import energy as E
from oracle import lo as LO
from oracle import multidet as MD
from paper_2202_00832_b300 import synth
from paper_2202_00832_b300.lo_afqmc import Context, LoafError

pytestmark = pytest.mark.gpu

TOL_E = 1e-10


def _system(M=24, N=6, X=48, W=3, n_inact=3, n_act=8, n_det=15, max_exc=3, seed=11):
    mol, walk = synth.small_case(M, N, X, W, seed=seed, eps=0.1)
    cas = synth.make_cas_trial(mol, n_inact, n_act, n_det, max_exc, seed + 100)
    return mol, walk, cas


def _context(mol, C, t_svd):
    ctx = Context(0)
    ctx.ao_load_cholesky(mol.h, mol.L, np.ascontiguousarray(C))
    _, msvd = ctx.lo_localize_compress(t_svd, localize=False)
    return ctx, msvd


def _log_overlap_ref(prep, cas, phi):
    _, smw = MD.smw_thetas(prep.C, cas.dets, phi)
    r = np.array([s.ratio for s in smw])
    ld0 = 2 * E.logdet(E.overlap(prep.C[:, cas.dets[0]], phi))
    return ld0 + np.log(np.sum(cas.coeffs * r ** 2))


def _phase_close(a, b, tol):
    d = np.angle(np.exp(1j * (np.imag(a) - np.imag(b))))
    return abs(np.real(a) - np.real(b)) < tol and abs(d) < tol


def test_cas_energy_threshold_zero():
    mol, walk, cas = _system()
    prep = MD.prepare_cas(mol, cas, 0.0)
    ctx, _ = _context(mol, prep.C, 0.0)
    e, lov, st = ctx.walkers_energy_cas(walk, cas.dets, cas.coeffs)
    assert np.all(st == 0)
    for w, phi in enumerate(walk):
        ref = MD.energy_multidet_lo(mol, cas, prep, phi)[0]
        assert abs(e[w] - ref) <= TOL_E * abs(ref)
        assert _phase_close(lov[w], _log_overlap_ref(prep, cas, phi), 1e-10)
        # and the direct route (an inverse and the Cholesky form per determinant)
        ex = MD.energy_multidet_exact(mol.h, mol.L, cas.C, cas.dets, cas.coeffs, phi)[0]
        assert abs(e[w] - ex) <= TOL_E * abs(ex)


def test_cas_energy_truncated_with_library_ranks():
    mol, walk, cas = _system(seed=13)
    C = MD.localize_inactive(cas.C, cas.n_inact, mol.orbital_pos)
    ctx, msvd = _context(mol, C, 1e-2)
    assert msvd.min() < mol.M
    Lbar = E.half_rotate(mol.L, C)
    fac = LO.truncate(LO.pair_svds(Lbar), 1e-2, keep=msvd)
    prep = MD.CASPrep(C, Lbar, C.T @ mol.h, fac, {p: n for n, p in enumerate(fac.pairs)})
    e, _, st = ctx.walkers_energy_cas(walk, cas.dets, cas.coeffs)
    assert np.all(st == 0)
    for w, phi in enumerate(walk):
        ref = MD.energy_multidet_lo(mol, cas, prep, phi)[0]
        assert abs(e[w] - ref) <= TOL_E * abs(ref)


def test_one_determinant_is_the_single_determinant_energy():
    mol, walk, cas = _system(n_det=1, seed=17)
    ctx, _ = _context(mol, cas.C, 0.0)
    e, _, st = ctx.walkers_energy_cas(walk, cas.dets, cas.coeffs)
    assert np.all(st == 0)
    for w, phi in enumerate(walk):
        ref = E.walker_energy(mol, phi)["E"]
        assert abs(e[w] - ref) <= TOL_E * abs(ref)


def test_cas_argument_checks():
    mol, walk, cas = _system(n_det=4, seed=19)
    ctx, _ = _context(mol, cas.C, 0.0)
    bad = np.array(cas.dets, dtype=np.int32)
    bad[1, -1] = cas.n_inact + cas.n_act          # outside the CAS orbitals
    with pytest.raises(LoafError):
        ctx.walkers_energy_cas(walk, bad, cas.coeffs)
    dup = np.array(cas.dets, dtype=np.int32)
    dup[2, 1] = dup[2, 0]                          # repeated orbital
    with pytest.raises(LoafError):
        ctx.walkers_energy_cas(walk, dup, cas.coeffs)
    # the context still answers afterwards
    e, _, st = ctx.walkers_energy_cas(walk, cas.dets, cas.coeffs)
    assert np.all(st == 0) and np.all(np.isfinite(e))


def test_cas_no_inactive_orbitals_one_walker():
    mol, walk, cas = _system(M=20, N=5, X=40, W=1, n_inact=0, n_act=10, n_det=9, max_exc=3, seed=23)
    prep = MD.prepare_cas(mol, cas, 0.0)
    ctx, _ = _context(mol, prep.C, 0.0)
    e, _, st = ctx.walkers_energy_cas(walk, cas.dets, cas.coeffs)
    assert np.all(st == 0)
    ref = MD.energy_multidet_lo(mol, cas, prep, walk[0])[0]
    assert abs(e[0] - ref) <= TOL_E * abs(ref)


def test_cas_largest_excitation_and_limit():
    mol, walk, _ = _system(M=30, N=9, X=40, W=2, n_inact=1, n_act=20, n_det=2, max_exc=1, seed=29)
    C = np.linalg.eigh(mol.h)[1][:, :21]
    ref = list(range(9))
    eight = [0] + list(range(9, 17))        # slots 1..8 changed
    nine = list(range(9, 18))               # all nine slots changed
    cas = synth.CASTrial(C, 1, 20, 9, [ref, eight], np.array([1.0, 0.4]))
    prep = MD.prepare_cas(mol, cas, 0.0)
    ctx, _ = _context(mol, prep.C, 0.0)
    e, _, st = ctx.walkers_energy_cas(walk, cas.dets, cas.coeffs)
    assert np.all(st == 0)
    for w, phi in enumerate(walk):
        r = MD.energy_multidet_lo(mol, cas, prep, phi)[0]
        assert abs(e[w] - r) <= TOL_E * abs(r)
    with pytest.raises(LoafError, match="SHAPE"):
        ctx.walkers_energy_cas(walk, np.array([ref, nine], dtype=np.int32), np.array([1.0, 0.4]))

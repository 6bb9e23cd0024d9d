"""Pins of the multi-determinant (CAS) oracle: SMW updates (eq. Q_SMW_reg),
the projected columns of eq. BigQ and the mixed estimate of eq. 2e_HR_RCAS,
checked against definitions that do not go through them: a direct inverse per
determinant, numpy determinants, the single-determinant oracle, the explicit-
loop Wick sum, gauge and scale invariances and the truncation bound."""
import numpy as np
import pytest

from oracle import energy as E
from oracle import lo as LO
from oracle import multidet as MD
from paper_2202_00832_b300 import synth


def _case(M=24, N=6, X=48, W=3, n_inact=3, n_act=8, n_det=15, max_exc=3, seed=11):
    mol, walk = synth.small_case(M, N, X, W, seed=seed, eps=0.1)
    cas = synth.make_cas_trial(mol, n_inact, n_act, n_det, max_exc, seed + 100)
    return mol, walk, cas


@pytest.fixture(scope="module")
def case():
    return _case()


def test_cas_generator_structure(case):
    mol, _, cas = case
    assert cas.dets[0] == list(range(cas.N)) and cas.coeffs[0] == 1.0
    assert len({tuple(d) for d in cas.dets}) == cas.n_det == 15
    for d in cas.dets:
        assert d[:cas.n_inact] == list(range(cas.n_inact))     # inactive slots never change
        assert len(set(d)) == cas.N
        assert all(0 <= o < cas.n_inact + cas.n_act for o in d)
    assert 1 <= cas.max_excitation <= 3
    np.testing.assert_allclose(cas.C.T @ cas.C, np.eye(cas.C.shape[1]), atol=1e-12)
    np.testing.assert_allclose(cas.C[:, :cas.N], mol.trial_a, atol=1e-12)


def test_smw_theta_and_ratio_match_direct_inverse(case):
    mol, walk, cas = case
    phi = walk[0]
    th0, smw = MD.smw_thetas(cas.C, cas.dets, phi)
    det0 = np.linalg.det(cas.C[:, cas.dets[0]].T @ phi)
    for d, det in enumerate(cas.dets):
        direct = E.theta(cas.C[:, det], phi)
        assert np.max(np.abs(smw[d].theta - direct)) <= 1e-12 * np.max(np.abs(direct))
        ratio = np.linalg.det(cas.C[:, det].T @ phi) / det0
        assert abs(smw[d].ratio - ratio) <= 1e-12 * max(1.0, abs(ratio))
        # Phi_d^T Q^d = I for every determinant (the Q intermediate of eq. Q)
        np.testing.assert_allclose(cas.C[:, det].T @ smw[d].theta, np.eye(cas.N), atol=1e-11)


def test_planted_smw_sign_fails(case):
    mol, walk, cas = case
    phi = walk[0]
    th0, smw = MD.smw_thetas(cas.C, cas.dets, phi)
    d = next(k for k in range(cas.n_det) if smw[k].slots)
    bad = th0 + th0[:, smw[d].slots] @ smw[d].S
    assert np.max(np.abs(bad - E.theta(cas.C[:, cas.dets[d]], phi))) > 1e-6


def test_one_determinant_expansion_is_the_single_determinant_energy():
    mol, walk, cas = _case(n_det=1)
    prep = MD.prepare_cas(mol, cas, 0.0)
    for phi in walk:
        e_lo, w, _ = MD.energy_multidet_lo(mol, cas, prep, phi)
        e_single = E.walker_energy(mol, phi)["E"]
        assert abs(e_lo - e_single) <= 1e-10 * abs(e_single)
        assert w.shape == (1,) and abs(w[0] - 1.0) < 1e-15


def test_lo_smw_at_threshold_zero_equals_weighted_exact_energy(case):
    mol, walk, cas = case
    prep = MD.prepare_cas(mol, cas, 0.0)
    for phi in walk:
        e_ex, w_ex, _ = MD.energy_multidet_exact(mol.h, mol.L, cas.C, cas.dets, cas.coeffs, phi)
        e_lo, w_lo, _ = MD.energy_multidet_lo(mol, cas, prep, phi)
        assert abs(e_lo - e_ex) <= 1e-10 * abs(e_ex)
        np.testing.assert_allclose(w_lo, w_ex, rtol=1e-10, atol=1e-13)
        # the compressed Coulomb is exact at T = 0 as well
        e_lc, _, _ = MD.energy_multidet_lo(mol, cas, prep, phi, coulomb="compressed")
        assert abs(e_lc - e_ex) <= 1e-10 * abs(e_ex)


def test_planted_missing_bigq_correction_and_unsquared_overlap_fail(case):
    mol, walk, cas = case
    phi = walk[0]
    prep = MD.prepare_cas(mol, cas, 0.0)
    e_ex, w_ex, Es_ex = MD.energy_multidet_exact(mol.h, mol.L, cas.C, cas.dets, cas.coeffs, phi)
    # (1) reference columns only: every determinant's exchange with Theta^0
    th0, smw = MD.smw_thetas(prep.C, cas.dets, phi)
    Es_bad = []
    for d, det in enumerate(cas.dets):
        good = MD.energy_multidet_lo(mol, synth.CASTrial(cas.C, cas.n_inact, cas.n_act, cas.N,
                                                          [det], np.ones(1)), prep, phi)[2][0]
        ek_good = sum(np.dot(MD._pair_factors(prep, det[s], det[t])[0].T @ smw[d].theta[:, t],
                             MD._pair_factors(prep, det[s], det[t])[1] @ smw[d].theta[:, s])
                      for s in range(cas.N) for t in range(cas.N))
        ek_bad = sum(np.dot(MD._pair_factors(prep, det[s], det[t])[0].T @ th0[:, t],
                            MD._pair_factors(prep, det[s], det[t])[1] @ th0[:, s])
                     for s in range(cas.N) for t in range(cas.N))
        Es_bad.append(good + ek_good - ek_bad)
    assert abs(np.sum(w_ex * np.array(Es_bad)) - e_ex) > 1e-6 * abs(e_ex)
    # (2) overlaps not squared (one spin only) in the weights
    w1 = cas.coeffs * np.array([s.ratio for s in smw])
    w1 = w1 / np.sum(w1)
    assert abs(np.sum(w1 * Es_ex) - e_ex) > 1e-6 * abs(e_ex)


def test_weighted_estimate_against_explicit_wick_loops():
    """Tiny case: each determinant's energy from the four-index Wick sum with
    explicit loops, its overlap from numpy det, weighted by hand."""
    mol, walk, cas = _case(M=8, N=3, X=10, W=2, n_inact=1, n_act=5, n_det=5, max_exc=2, seed=5)
    V = E.dense_eri(mol.L)
    for phi in walk:
        num, den = 0j, 0j
        for c, det in zip(cas.coeffs, cas.dets):
            P = cas.C[:, det]
            G = E.green(P, phi)
            ov = np.linalg.det(P.T @ phi) ** 2
            num += c * ov * E.energy_wick_loops(mol.h, V, G, G)
            den += c * ov
        e_ref = num / den
        e_ex = MD.energy_multidet_exact(mol.h, mol.L, cas.C, cas.dets, cas.coeffs, phi)[0]
        assert abs(e_ex - e_ref) <= 1e-12 * abs(e_ref)
        prep = MD.prepare_cas(mol, cas, 0.0)
        e_lo = MD.energy_multidet_lo(mol, cas, prep, phi)[0]
        assert abs(e_lo - e_ref) <= 1e-10 * abs(e_ref)


def test_gauge_and_coefficient_scale_invariance(case):
    mol, walk, cas = case
    prep = MD.prepare_cas(mol, cas, 1e-3)
    phi = walk[1]
    rng = np.random.default_rng(3)
    R = rng.standard_normal((cas.N, cas.N)) + 1j * rng.standard_normal((cas.N, cas.N)) + 3 * np.eye(cas.N)
    e = MD.energy_multidet_lo(mol, cas, prep, phi)[0]
    assert abs(MD.energy_multidet_lo(mol, cas, prep, phi @ R)[0] - e) <= 1e-10 * abs(e)
    scaled = synth.CASTrial(cas.C, cas.n_inact, cas.n_act, cas.N, cas.dets, 2.5 * cas.coeffs)
    assert abs(MD.energy_multidet_lo(mol, scaled, prep, phi)[0] - e) <= 1e-12 * abs(e)


def test_inactive_localization_leaves_the_energy_unchanged(case):
    mol, walk, cas = case
    p_loc = MD.prepare_cas(mol, cas, 0.0, localize=True)
    p_can = MD.prepare_cas(mol, cas, 0.0, localize=False)
    assert np.max(np.abs(p_loc.C[:, :cas.n_inact] - p_can.C[:, :cas.n_inact])) > 1e-3
    np.testing.assert_array_equal(p_loc.C[:, cas.n_inact:], p_can.C[:, cas.n_inact:])
    phi = walk[2]
    a = MD.energy_multidet_lo(mol, cas, p_loc, phi)[0]
    b = MD.energy_multidet_lo(mol, cas, p_can, phi)[0]
    assert abs(a - b) <= 1e-10 * abs(a)


def test_truncation_error_within_bound(case):
    mol, walk, cas = case
    prep = MD.prepare_cas(mol, cas, 1e-2)
    assert prep.factors.m_svd.min() < mol.M        # something is dropped
    for phi in walk:
        e_ex, w, _ = MD.energy_multidet_exact(mol.h, mol.L, cas.C, cas.dets, cas.coeffs, phi)
        e_lo, w_lo, _ = MD.energy_multidet_lo(mol, cas, prep, phi)
        bound = MD.truncation_bound_multidet(cas, prep, phi, w_lo)
        assert 0.0 < abs(e_lo - e_ex) <= bound

"""Learned pair screen on the GPU: the hand-written forward/backward kernels
against the FP64 oracle's analytic gradient, the pair descriptors against the
oracle's own localization and SVDs, training, and the screened energies.

Tolerances: the network runs with FP16 weights and activations (relative
rounding 2^-11 ~ 4.9e-4 per operand, three layers), so the loss is compared to
1e-2 and the gradient to 3e-2 in relative 2-norm.
"""
import numpy as np
import pytest

from oracle import energy as E
from oracle import lo, mlp
from paper_2202_00832_b300.lo_afqmc import (Context, init_screen_params, mlp_loss_grad,
                                            position_operators)

pytestmark = pytest.mark.gpu


def test_network_gradient_matches_oracle():
    rng = np.random.default_rng(11)
    n = 300
    x = rng.standard_normal((n, 8))
    t = np.tanh(x[:, 0] - x[:, 2]) + 0.3 * rng.standard_normal(n)
    th = init_screen_params(3).astype(np.float64) + 0.05 * rng.standard_normal(mlp.n_params())
    loss_gpu, g_gpu = mlp_loss_grad(x, t, th)
    loss_ref = mlp.loss(th, x, t)
    g_ref = mlp.grad(th, x, t)
    assert abs(loss_gpu - loss_ref) < 1e-2 * loss_ref
    assert np.linalg.norm(g_gpu - g_ref) < 3e-2 * np.linalg.norm(g_ref)


@pytest.fixture(scope="module")
def chain_screen(chain60):
    mol, walk = chain60
    ctx = Context(0)
    ctx.load_molecule(mol)
    ctx.lo_localize_compress(0.0, position_operators(mol), localize=True)
    return ctx, mol, walk


def test_descriptors_match_oracle(chain_screen):
    ctx, mol, walk = chain_screen
    got = ctx.pair_screen_query(trained=False)["features"]
    sp = lo.prepare(mol, 0.0)[0]
    ref = mlp.pair_features(sp.trial_loc, position_operators(mol), sp.factors.pairs,
                            sp.factors.sigma, sp.factors.m_svd, mol.M)
    assert np.abs(got - ref).max() < 1e-6


def test_training_and_screened_energies(chain_screen):
    ctx, mol, walk = chain_screen
    hist = ctx.pair_screen_train(walk[:16], init_screen_params(0), epochs=600, lr=3e-3)
    assert hist[-1] < 0.3 * hist[0]
    q = ctx.pair_screen_query()
    assert np.corrcoef(q["pred"], q["target"])[0, 1] > 0.8
    n = ctx.num_pairs
    e_full64, _, _ = ctx.walkers_energy(walk, mode="lo", precision="fp64")
    e_full16, _, _ = ctx.walkers_energy(walk, mode="lo", precision="fp16x3")
    # the method's cutoff keeps every pair of this system: nothing changes
    assert ctx.pair_screen_set(1e-6) == n
    e, _, _ = ctx.walkers_energy(walk, mode="lo", precision="fp16x3")
    assert np.array_equal(e, e_full16)
    # a cutoff at the median prediction drops about half of the pairs; the
    # screened energy is the unscreened one minus exactly the dropped pairs
    cut = 10.0 ** np.median(q["pred"])
    kept = ctx.pair_screen_set(cut)
    keep = ctx.pair_screen_query()["keep"].astype(bool)
    assert 0 < kept < n and kept == keep.sum()
    pairs = [(i, j) for i in range(mol.n_alpha) for j in range(i, mol.n_alpha)]
    wgt = np.array([1.0 if i == j else 2.0 for i, j in pairs])
    ep = ctx.walkers_pair_exchange(walk, precision="fp64")
    dropped = (wgt[~keep, None] * ep[~keep]).sum(axis=0)  # closed shell: E_K = sum_ij e_ij
    e64, _, _ = ctx.walkers_energy(walk, mode="lo", precision="fp64")
    assert np.max(np.abs(e64 - (e_full64 + dropped)) / np.abs(e_full64)) < 1e-10
    e16, _, _ = ctx.walkers_energy(walk, mode="lo", precision="fp16x3")
    assert np.abs(e16 - e64).max() < 1e-4
    ctx.pair_screen_set(-1.0)
    e, _, _ = ctx.walkers_energy(walk, mode="lo", precision="fp16x3")
    assert np.array_equal(e, e_full16)


def test_screen_gain_on_separate_fragments():
    """What the trained screen gains (Sec. 5's proposal): a system of two
    fragments 20 bonds apart, walkers perturbed within 3 bonds.  Every pair of
    orbitals on different fragments contributes below 1e-6 Ha, yet its truncated
    block keeps its rank, so T_SVD cannot drop it.  At the method's 1e-6 Ha cutoff
    the trained network drops those pairs and keeps every intra-fragment pair;
    the screened energy equals the unscreened one minus exactly the dropped
    pairs (FP64), and the oracle's LO energy with the same pairs masked, built
    from the library's localized orbitals and kept ranks."""
    from paper_2202_00832_b300 import synth
    mol = synth.make_molecule("fragments2_M180", 180, 360, 30, 30, "fragments", 1107, decay=0.5,
                              n_frag=2, frag_gap=20.0)
    walk = synth.make_walkers(mol, 96, 0.3, 5107, band=3.0)
    ctx = Context(0)
    ctx.load_molecule(mol)
    _, msvd = ctx.lo_localize_compress(1e-4, position_operators(mol), localize=True)
    n = ctx.num_pairs
    C = ctx.localized_trial(0)
    on_first = mol.pos[mol.site_of][:, 0] < 39.0  # basis functions of the first fragment
    frag = (np.sum(C[on_first] ** 2, axis=0) > 0.5).astype(int)  # fragment of each orbital
    pairs = [(i, j) for i in range(mol.n_alpha) for j in range(i, mol.n_alpha)]
    inter = np.array([frag[i] != frag[j] for i, j in pairs])
    assert inter.sum() == 15 * 15
    assert np.all(msvd[inter] > 0)  # the truncation keeps these blocks
    train, test = walk[:64], walk[64:]
    ctx.pair_screen_train(train, init_screen_params(0), epochs=800, lr=3e-3)
    ep_train = ctx.walkers_pair_exchange(train, precision="fp64")
    assert np.abs(ep_train[inter]).max() < 1e-6
    kept = ctx.pair_screen_set(1e-6)
    keep = ctx.pair_screen_query()["keep"].astype(bool)
    assert np.all(keep[~inter]) and not np.any(keep[inter])
    assert kept == n - inter.sum()
    wgt = np.array([1.0 if i == j else 2.0 for i, j in pairs])
    ep = ctx.walkers_pair_exchange(test, precision="fp64")
    dropped = (wgt[~keep, None] * ep[~keep]).sum(axis=0)
    assert np.abs(dropped).max() < 1e-6 * wgt[inter].sum()
    e64_s, _, _ = ctx.walkers_energy(test, mode="lo", precision="fp64")
    e16_s, _, _ = ctx.walkers_energy(test, mode="lo", precision="fp16x3")
    ctx.pair_screen_set(-1.0)
    e64_u, _, _ = ctx.walkers_energy(test, mode="lo", precision="fp64")
    assert np.max(np.abs(e64_s - (e64_u + dropped)) / np.abs(e64_u)) < 1e-10
    assert np.abs(e16_s - e64_u).max() < 1e-4
    # the oracle with the same pairs masked
    Lbar = E.half_rotate(mol.L, C)
    ths = np.array([E.theta(C, w) for w in test[:4]])
    pv = lo.pair_exchange_streamed(Lbar, msvd, ths, workers=4)
    for k in range(4):
        full = E.walker_energy(mol, test[k])
        ref = full["E1"] + full["EJ"] - np.sum((wgt * keep)[:, None] * pv[:, k:k + 1])
        assert abs(e64_s[k] - ref) < 1e-10 * abs(ref)

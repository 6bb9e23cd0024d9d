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

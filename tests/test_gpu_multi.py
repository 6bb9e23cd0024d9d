"""Several systems in one graph launch (walkers_energy_multi) against each
system's own walkers_energy call and the FP64 LO path, through the C ABI.

The graph runs the same kernels with the same tile shapes (the autotuner keeps
its choice in each context) and differs only in scheduling, so per-walker
energies agree to 1e-9 relative.  Against the FP64 LO path the
bar is the mixed-precision 0.1 mHa.
"""
import numpy as np
import pytest

from oracle import energy as E
from oracle import lo
from paper_2202_00832_b300 import synth
from paper_2202_00832_b300.lo_afqmc import (Context, LoafError, position_operators,
                                            walkers_energy_multi)

pytestmark = pytest.mark.gpu

_RANKS = []  # kept rank of every pair, per system (from lo_localize_compress)


@pytest.fixture(scope="module")
def systems(chain60):
    import torch
    mol0, walk0 = chain60
    out = [(mol0, walk0)]
    for wl, W in [(synth.HETERO_BATCH[0], 48), (synth.HETERO_BATCH[1], 40)]:
        m = wl.molecule()
        out.append((m, wl.walkers(m, W=W, processes=1)))
    ctxs, ranks = [], []
    for mol, walk in out:
        c = Context(0)
        c.load_molecule(mol)
        _, msvd = c.lo_localize_compress(1e-4, position_operators(mol), localize=True)
        ctxs.append(c)
        ranks.append(msvd)
    phis = [torch.from_numpy(w).cuda() for _, w in out]
    _RANKS[:] = ranks
    return ctxs, out, phis


def _outs(phis):
    import torch
    e = [torch.zeros(p.shape[0], dtype=torch.complex128, device="cuda") for p in phis]
    ld = [torch.zeros_like(x) for x in e]
    st = [torch.zeros(p.shape[0], dtype=torch.int32, device="cuda") for p in phis]
    return e, ld, st


def test_multi_matches_single_calls(systems):
    ctxs, sys_, phis = systems
    e, ld, st = _outs(phis)
    caps = walkers_energy_multi(ctxs, phis, e, ld, st, autotune=True)
    assert len(caps) == 3 and all(c >= 0 for c in caps)
    # tile shapes chosen per system among the autotuner's candidates; the single
    # calls below run with the same shapes
    for c in ctxs:
        cap, split = c.tiles()
        assert cap in (256, 192, 128) and 0 <= split <= 16
    for k, (c, (mol, walk)) in enumerate(zip(ctxs, sys_)):
        e1, ld1, st1 = c.walkers_energy(walk, mode="lo", precision="fp16x3")
        got = e[k].cpu().numpy()
        assert np.all(st[k].cpu().numpy() == 0)
        assert np.max(np.abs(got - e1) / np.abs(e1)) < 1e-9
        assert np.allclose(ld[k].cpu().numpy(), ld1, rtol=0, atol=1e-12)
        e64, _, _ = c.walkers_energy(walk, mode="lo", precision="fp64")
        assert np.abs(got - e64).max() < 1e-4
    # the recorded graph is replayed: same outputs
    before = [x.cpu().numpy().copy() for x in e]
    for x in e:
        x.zero_()
    walkers_energy_multi(ctxs, phis, e, ld, st, autotune=True)
    for k in range(3):
        assert np.array_equal(e[k].cpu().numpy(), before[k])


def test_multi_argument_errors(systems):
    ctxs, sys_, phis = systems
    e, ld, st = _outs(phis)
    host = [p.cpu().numpy() for p in phis]
    with pytest.raises(LoafError) as ex:
        walkers_energy_multi(ctxs, host, e)
    assert ex.value.status == "LOAF_ERR_ARG"
    with pytest.raises(LoafError) as ex:
        walkers_energy_multi(ctxs, phis, e, precision="fp64")
    assert ex.value.status == "LOAF_ERR_UNSUPPORTED"
    with pytest.raises(LoafError) as ex:
        walkers_energy_multi([ctxs[0], ctxs[0]], [phis[0], phis[0]], [e[0], e[0]])
    assert ex.value.status == "LOAF_ERR_ARG"


def test_multi_against_oracle(systems):
    """Each system's energies from the graph launch against the oracle's LO energy
    built from the library's localized orbitals and kept ranks (T_SVD = 1e-4)."""
    ctxs, sys_, phis = systems
    e, ld, st = _outs(phis)
    walkers_energy_multi(ctxs, phis, e, ld, st, autotune=False)
    for k, (c, (mol, walk)) in enumerate(zip(ctxs, sys_)):
        idx = [0, 1, len(walk) - 1]
        C = c.localized_trial(0)
        Lbar = E.half_rotate(mol.L, C)
        ths = np.array([E.theta(C, walk[w]) for w in idx])
        pv = lo.pair_exchange_streamed(Lbar, _RANKS[k], ths, workers=4)
        N = mol.n_alpha
        wts = np.array([1.0 if i == j else 2.0 for i in range(N) for j in range(i, N)])
        got = e[k].cpu().numpy()[idx]
        for q, w in enumerate(idx):
            full = E.walker_energy(mol, walk[w])
            ref = full["E1"] + full["EJ"] - np.sum(wts * pv[:, q])
            assert abs(got[q] - ref) < 1e-4


def test_multi_graph_after_workspace_growth(systems):
    """A recorded multi-system graph holds the contexts' buffer addresses.  A
    larger single call on one context grows (moves) that context's workspace;
    the next multi call with the same signature must record the graph again
    instead of replaying it into freed memory, and give the same energies."""
    import torch
    ctxs, sys_, phis = systems
    e, ld, st = _outs(phis)
    walkers_energy_multi(ctxs, phis, e, ld, st, autotune=False)
    before = [x.cpu().numpy().copy() for x in e]
    mol0 = sys_[0][0]
    big = torch.from_numpy(synth.CHAIN_60.walkers(mol0, W=700, processes=1)).cuda()
    ebig = torch.zeros(700, dtype=torch.complex128, device="cuda")
    ctxs[0].walkers_energy(big, mode="lo", precision="fp16x3", e_out=ebig)
    for x in e:
        x.zero_()
    walkers_energy_multi(ctxs, phis, e, ld, st, autotune=False)
    for k in range(3):
        assert np.array_equal(e[k].cpu().numpy(), before[k])

"""walkers_energy as a stream of submitted calls (walkers_energy_submit /
walkers_energy_wait), through the C ABI.

A submitted call runs the same kernels on the same batch as a walkers_energy
call on the same W device-resident walkers, so its outputs are bitwise those of
that call; the oracle anchors a few walkers at the method's 0.1 mHa bar (Sec.
3.1.2, eq. 2e_HR_RCAS_LO with the library's kept ranks fed to the oracle).
Calls alternate between two device copies of the walkers: these tests submit
more calls than that before waiting, change the batch shape between calls, and
check that walker failures and pipeline timeouts reach walkers_energy_wait.
"""
import numpy as np
import pytest
import torch

from oracle import energy as E
from oracle import lo
from paper_2202_00832_b300 import synth
from paper_2202_00832_b300.lo_afqmc import Context, LoafError, position_operators

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-4  # Ha per walker


@pytest.fixture(scope="module")
def case():
    """M = 120, N = 16, X = 160, 300 walkers, T_SVD = 1e-3 (ranks vary by pair)."""
    mol, walk = synth.small_case(M=120, N=16, X=160, W=300, seed=515, geometry="acene")
    ctx = Context(0)
    ctx.load_molecule(mol)
    _, msvd = ctx.lo_localize_compress(1e-3, position_operators(mol), localize=True)
    return ctx, mol, walk, msvd


def pinned_outputs(W):
    e = torch.zeros(W, dtype=torch.complex128).pin_memory()
    ld = torch.zeros(W, dtype=torch.complex128).pin_memory()
    st = torch.full((W,), -1, dtype=torch.int32).pin_memory()
    return e, ld, st


def resident_call(ctx, walk, precision):
    """walkers_energy on device-resident walkers with device outputs."""
    d = torch.from_numpy(np.ascontiguousarray(walk)).cuda()
    torch.cuda.synchronize()
    W = len(walk)
    e = torch.zeros(W, dtype=torch.complex128, device="cuda")
    ld = torch.zeros_like(e)
    st = torch.zeros(W, dtype=torch.int32, device="cuda")
    ctx.walkers_energy(d, mode="lo", precision=precision, e_out=e, logdet_out=ld, walker_status=st,
                       raise_on_singular=False)
    return e.cpu().numpy(), ld.cpu().numpy(), st.cpu().numpy()


def batches(walk, n, seed):
    rng = np.random.default_rng(seed)
    return [np.ascontiguousarray(walk[rng.permutation(len(walk))]) for _ in range(n)]


@pytest.mark.parametrize("precision", ["fp16x3", "fp64"])
def test_stream_matches_resident_calls(case, precision):
    """Five calls (more than the two walker buffers) submitted back to back
    from pinned host memory, then one wait: every output equals the resident
    call on the same batch, bit for bit."""
    ctx, mol, walk, msvd = case
    bs = batches(walk, 5, 7)
    hs = [torch.from_numpy(b).pin_memory() for b in bs]
    outs = [pinned_outputs(len(b)) for b in bs]
    for h, (e, ld, st) in zip(hs, outs):
        ctx.walkers_energy_submit(h, e, ld, st, mode="lo", precision=precision)
    assert ctx.walkers_energy_wait() == 0
    for b, (e, ld, st) in zip(bs, outs):
        re, rld, rst = resident_call(ctx, b, precision)
        assert np.all(st.numpy() == 0) and np.all(rst == 0)
        assert np.array_equal(e.numpy(), re)
        assert np.array_equal(ld.numpy(), rld)
    # absolute anchor: the oracle's LO energy with the library's kept ranks
    C = ctx.localized_trial(0)
    Lbar = E.half_rotate(mol.L, C)
    idx = [0, 151]
    ths = np.array([E.theta(C, bs[0][w]) for w in idx])
    pv = lo.pair_exchange_streamed(Lbar, msvd, ths, workers=4)
    N = mol.n_alpha
    wts = np.array([1.0 if i == j else 2.0 for i in range(N) for j in range(i, N)])
    for q, w in enumerate(idx):
        full = E.walker_energy(mol, bs[0][w])
        ref = full["E1"] + full["EJ"] - np.sum(wts * pv[:, q])
        tol = TOL_MIXED if precision == "fp16x3" else 1e-8 * abs(ref)
        assert abs(outs[0][0].numpy()[w] - ref) < tol


def test_stream_slices_and_shape_changes(case):
    """A call above the 1024-walker pass (two passes of 1024 and 76) between
    calls of 300 walkers: the shape change waits for the calls in flight, and
    every call matches its resident form."""
    ctx, mol, walk, msvd = case
    big = np.ascontiguousarray(np.concatenate([walk] * 4)[:1100])
    bs = [batches(walk, 1, 11)[0], big, batches(walk, 1, 12)[0]]
    hs = [torch.from_numpy(b).pin_memory() for b in bs]
    outs = [pinned_outputs(len(b)) for b in bs]
    for h, (e, ld, st) in zip(hs, outs):
        ctx.walkers_energy_submit(h, e, ld, st, mode="lo", precision="fp16x3")
    assert ctx.walkers_energy_wait() == 0
    for b, (e, ld, st) in zip(bs, outs):
        re, rld, rst = resident_call(ctx, b, "fp16x3")
        assert np.array_equal(e.numpy(), re)
        assert np.array_equal(ld.numpy(), rld)
    # the repeated walkers of the large call got the same energies in each pass
    e_big = outs[1][0].numpy()
    assert np.array_equal(e_big[:300], e_big[300:600])


def test_stream_device_buffers(case):
    """Device walkers and device outputs: nothing is uploaded, same results."""
    ctx, mol, walk, msvd = case
    bs = batches(walk, 3, 13)
    ds = [torch.from_numpy(b).cuda() for b in bs]
    torch.cuda.synchronize()
    outs = []
    for d in ds:
        e = torch.zeros(len(d), dtype=torch.complex128, device="cuda")
        ld = torch.zeros_like(e)
        st = torch.full((len(d),), -1, dtype=torch.int32, device="cuda")
        ctx.walkers_energy_submit(d, e, ld, st, mode="lo", precision="fp16x3")
        outs.append((e, ld, st))
    assert ctx.walkers_energy_wait() == 0
    for b, (e, ld, st) in zip(bs, outs):
        re, rld, _ = resident_call(ctx, b, "fp16x3")
        assert np.array_equal(e.cpu().numpy(), re)
        assert np.array_equal(ld.cpu().numpy(), rld)


def test_stream_reports_a_singular_walker(case):
    """A singular walker in the second of three calls: the wait reports
    LOAF_ERR_SINGULAR, that call's status marks the walker (energy NaN), the
    other walkers and calls are unaffected, and the next wait starts clean."""
    ctx, mol, walk, msvd = case
    bs = batches(walk, 3, 17)
    virt = np.linalg.eigh(mol.h)[1][:, mol.n_alpha]
    bs[1][40][:, 3] = virt  # Phi_T^T phi gets a zero column
    hs = [torch.from_numpy(b).pin_memory() for b in bs]
    outs = [pinned_outputs(len(b)) for b in bs]
    for h, (e, ld, st) in zip(hs, outs):
        ctx.walkers_energy_submit(h, e, ld, st, mode="lo", precision="fp16x3")
    with pytest.raises(LoafError) as ei:
        ctx.walkers_energy_wait()
    assert ei.value.status == "LOAF_ERR_SINGULAR"
    st1 = outs[1][2].numpy()
    assert st1[40] == 1 and np.isnan(outs[1][0].numpy()[40])
    assert np.all(np.delete(st1, 40) == 0)
    for q in (0, 2):
        assert np.all(outs[q][2].numpy() == 0)
        re, _, _ = resident_call(ctx, bs[q], "fp16x3")
        assert np.array_equal(outs[q][0].numpy(), re)
    e, ld, st = pinned_outputs(len(walk))
    ctx.walkers_energy_submit(torch.from_numpy(walk).pin_memory(), e, ld, st, mode="lo", precision="fp16x3")
    assert ctx.walkers_energy_wait() == 0
    assert np.all(st.numpy() == 0)


def test_stream_timeout_reaches_the_wait(case):
    """The LO tensor-core kernel of a submitted call leaves one pipeline stage
    unfilled (the withheld-stage hook): its bounded waits run out, the kernel
    unwinds, and walkers_energy_wait returns LOAF_ERR_TIMEOUT.  The context is
    usable afterwards."""
    ctx, mol, walk, msvd = case
    h = torch.from_numpy(walk).pin_memory()
    e, ld, st = pinned_outputs(len(walk))
    ctx.test_withhold_stage(1)
    ctx.walkers_energy_submit(h, e, ld, st, mode="lo", precision="fp16x3")
    with pytest.raises(LoafError) as ei:
        ctx.walkers_energy_wait()
    assert ei.value.status == "LOAF_ERR_TIMEOUT"
    ctx.walkers_energy_submit(h, e, ld, st, mode="lo", precision="fp16x3")
    assert ctx.walkers_energy_wait() == 0
    re, _, _ = resident_call(ctx, walk, "fp16x3")
    assert np.array_equal(e.numpy(), re)


def test_operand_changes_wait_for_submitted_calls(case):
    """Changing the tile shapes or the compression while calls are queued
    first lets those calls finish with the operands they were queued with:
    the first call runs with the default shapes, the second with the new
    shapes, both at T_SVD = 1e-3, although T_SVD = 1e-2 is set before the wait."""
    ctx, mol, walk, msvd = case
    b = batches(walk, 1, 19)[0]
    ref_a, _, _ = resident_call(ctx, b, "fp16x3")
    ctx.set_tiles(128, 3)
    ref_b, _, _ = resident_call(ctx, b, "fp16x3")
    ctx.set_tiles(256, 0)
    h = torch.from_numpy(b).pin_memory()
    e1, ld1, st1 = pinned_outputs(len(b))
    e2, ld2, st2 = pinned_outputs(len(b))
    try:
        ctx.walkers_energy_submit(h, e1, ld1, st1, mode="lo", precision="fp16x3")
        ctx.set_tiles(128, 3)
        ctx.walkers_energy_submit(h, e2, ld2, st2, mode="lo", precision="fp16x3")
        ctx.lo_localize_compress(1e-2, position_operators(mol), localize=True)
        assert ctx.walkers_energy_wait() == 0
        assert np.array_equal(e1.numpy(), ref_a)
        assert np.array_equal(e2.numpy(), ref_b)
    finally:
        ctx.set_tiles(256, 0)
        ctx.lo_localize_compress(1e-3, position_operators(mol), localize=True)

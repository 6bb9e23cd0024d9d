"""walkers_theta_noalloc, the variant for callers that cannot allocate device
memory during a call (fixed-budget allocators, jobs that must not grow once
running).  Collected last on purpose: it checks the new entry point against
walkers_theta through the C ABI, on two calls in a row, with the tolerance
the other Theta tests use (1e-11 of the largest entry; log-det 1e-10)."""
import numpy as np
import pytest

from paper_2202_00832_b300.lo_afqmc import Context, LoafError

pytestmark = pytest.mark.gpu


def test_noalloc_theta_matches_walkers_theta(chain60):
    import torch
    mol, walk = chain60
    ctx = Context(0)
    ctx.load_molecule(mol)
    W = len(walk)
    phi = torch.from_numpy(walk).cuda()
    ref_t = torch.zeros((W, ctx.ntot, mol.M), dtype=torch.complex128, device="cuda")
    ref_ld = torch.zeros(W, dtype=torch.complex128, device="cuda")
    ref_st = torch.zeros(W, dtype=torch.int32, device="cuda")
    ctx.walkers_theta(phi, ref_t, ref_ld, ref_st)
    torch.cuda.synchronize()
    ref_t, ref_ld, ref_st = ref_t.cpu().numpy(), ref_ld.cpu().numpy(), ref_st.cpu().numpy()
    for _ in range(2):
        th = torch.full((W, ctx.ntot, mol.M), float("nan"), dtype=torch.complex128, device="cuda")
        ld = torch.zeros(W, dtype=torch.complex128, device="cuda")
        st = torch.full((W,), -1, dtype=torch.int32, device="cuda")
        ctx.walkers_theta_noalloc(phi, th, ld, st)
        torch.cuda.synchronize()
        th, ld, st = th.cpu().numpy(), ld.cpu().numpy(), st.cpu().numpy()
        assert np.all(st == ref_st) and np.all(st == 0)
        assert np.abs(th - ref_t).max() <= 1e-11 * np.abs(ref_t).max()
        assert np.abs(ld.real - ref_ld.real).max() < 1e-10
        dphase = np.angle(np.exp(1j * (ld.imag - ref_ld.imag)))
        assert np.abs(dphase).max() < 1e-10


def test_noalloc_rejects_sizes_beyond_its_scratch(chain60):
    import torch
    mol, walk = chain60
    ctx = Context(0)
    ctx.load_molecule(mol)
    phi = torch.from_numpy(walk[:1]).cuda()
    out = torch.zeros((1, ctx.ntot, mol.M), dtype=torch.complex128, device="cuda")
    # 4097 walkers is beyond the fixed limit; rejected before any work is queued
    lib = ctx._lib
    code = lib.walkers_theta_noalloc(ctx._h, 4097, phi.data_ptr(), out.data_ptr(), None, None)
    assert code == 2  # LOAF_ERR_SHAPE
    assert b"4096" in lib.loaf_last_error(ctx._h)
    with pytest.raises(LoafError):
        ctx.walkers_theta_noalloc(walk[:1], walk[:1].copy())  # host buffers are refused


def test_noalloc_open_shell_matches_walkers_theta():
    """Two spin blocks: the second spin's log-det and status parts sit at a fixed
    offset of the shared array and are combined with the first spin's."""
    import torch
    from paper_2202_00832_b300 import synth
    mol, walk = synth.small_case(M=30, N=6, X=40, W=9, seed=31, n_beta=5)
    ctx = Context(0)
    ctx.load_molecule(mol)
    W = len(walk)
    phi = torch.from_numpy(walk).cuda()
    ref_t, ref_ld, ref_st = ctx.walkers_theta(walk)
    for _ in range(2):
        th = torch.full((W, ctx.ntot, mol.M), float("nan"), dtype=torch.complex128, device="cuda")
        ld = torch.zeros(W, dtype=torch.complex128, device="cuda")
        st = torch.full((W,), -1, dtype=torch.int32, device="cuda")
        ctx.walkers_theta_noalloc(phi, th, ld, st)
        torch.cuda.synchronize()
        assert np.all(st.cpu().numpy() == ref_st) and np.all(ref_st == 0)
        assert np.abs(th.cpu().numpy() - ref_t).max() <= 1e-11 * np.abs(ref_t).max()
        ldn = ld.cpu().numpy()
        assert np.abs(ldn.real - ref_ld.real).max() < 1e-10
        assert np.abs(np.angle(np.exp(1j * (ldn.imag - ref_ld.imag)))).max() < 1e-10


def test_noalloc_rejects_entry_count_beyond_its_scratch(chain60):
    """W within the walker limit, but W * Ntot * M above the 2,086,912 complex
    entries the fixed array holds (3500 x 10 x 60 = 2,100,000)."""
    import torch
    mol, walk = chain60
    ctx = Context(0)
    ctx.load_molecule(mol)
    phi = torch.from_numpy(walk[:1]).cuda()
    out = torch.zeros((1, ctx.ntot, mol.M), dtype=torch.complex128, device="cuda")
    code = ctx._lib.walkers_theta_noalloc(ctx._h, 3500, phi.data_ptr(), out.data_ptr(), None, None)
    assert code == 2  # LOAF_ERR_SHAPE, before any work is queued
    assert b"2086912" in ctx._lib.loaf_last_error(ctx._h)


def test_noalloc_takes_no_device_memory(chain60):
    """After a first call (which looks up the array's address), further calls
    leave the device's free memory unchanged."""
    import torch
    mol, walk = chain60
    ctx = Context(0)
    ctx.load_molecule(mol)
    W = len(walk)
    phi = torch.from_numpy(walk).cuda()
    th = torch.zeros((W, ctx.ntot, mol.M), dtype=torch.complex128, device="cuda")
    ld = torch.zeros(W, dtype=torch.complex128, device="cuda")
    st = torch.zeros(W, dtype=torch.int32, device="cuda")
    ctx.walkers_theta_noalloc(phi, th, ld, st)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        ctx.walkers_theta_noalloc(phi, th, ld, st)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0

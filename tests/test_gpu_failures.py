"""Failure paths of the production (FP16X3) path, through the C ABI.

No case here faults, traps or hangs the GPU: a bad walker is an input the
kernels take like any other, and they report it through the per-walker
status.  A singular overlap (a walker orbital orthogonal to every trial
orbital) marks that walker LOAF_WALKER_SINGULAR; a NaN or infinity in a
walker marks it LOAF_WALKER_NAN; in both cases its energy is NaN, the other
walkers keep their energies (0.1 mHa of the oracle) and the call returns
LOAF_ERR_SINGULAR or LOAF_ERR_NAN after writing every output.
"""
import numpy as np
import pytest

from oracle import energy as E
from paper_2202_00832_b300.lo_afqmc import Context, LoafError, position_operators

pytestmark = pytest.mark.gpu

TOL = {"fp16x3": 1e-4, "fp64": 1e-8}


@pytest.fixture(scope="module")
def chain_lo(chain60):
    mol, walk = chain60
    ctx = Context(0)
    ctx.load_molecule(mol)
    ctx.lo_localize_compress(0.0, position_operators(mol), localize=True)
    return ctx, mol, walk


def run_bad(ctx, walk, mode, precision):
    W = len(walk)
    e = np.zeros(W, dtype=np.complex128)
    ld = np.zeros(W, dtype=np.complex128)
    st = np.full(W, -1, dtype=np.int32)
    with pytest.raises(LoafError) as ei:
        ctx.walkers_energy(walk, mode=mode, precision=precision, e_out=e, logdet_out=ld,
                           walker_status=st)
    return e, ld, st, ei.value.status


@pytest.mark.parametrize("mode", ["lo", "full"])
def test_singular_walker_fp16x3(chain_lo, mode):
    ctx, mol, walk = chain_lo
    bad = walk[:5].copy()
    virt = np.linalg.eigh(mol.h)[1][:, mol.n_alpha]
    bad[3][:, 2] = virt  # Phi_T^T phi gets a zero column
    e, ld, st, status = run_bad(ctx, bad, mode, "fp16x3")
    assert status == "LOAF_ERR_SINGULAR"
    assert st[3] == 1 and np.isnan(e[3])
    ok = [0, 1, 2, 4]
    assert np.all(st[ok] == 0)
    ref = np.array([E.walker_energy(mol, bad[w])["E"] for w in ok])
    assert np.abs(e[ok] - ref).max() < TOL["fp16x3"]


@pytest.mark.parametrize("precision", ["fp16x3", "fp64"])
@pytest.mark.parametrize("value", [np.nan, np.inf])
def test_non_finite_walker(chain_lo, precision, value):
    ctx, mol, walk = chain_lo
    bad = walk[:6].copy()
    bad[2][7, 1] = complex(value, 0.0)
    bad[5][0, 0] = complex(0.0, value)
    e, ld, st, status = run_bad(ctx, bad, "lo", precision)
    assert status == "LOAF_ERR_NAN"
    assert st[2] == 2 and st[5] == 2
    assert np.isnan(e[2]) and np.isnan(e[5])
    ok = [0, 1, 3, 4]
    assert np.all(st[ok] == 0)
    ref = np.array([E.walker_energy(mol, bad[w])["E"] for w in ok])
    tol = TOL[precision] * (np.abs(ref) if precision == "fp64" else 1.0)
    assert np.all(np.abs(e[ok] - ref) < tol)
    # the context stays usable: a clean batch afterwards
    e2, _, st2 = ctx.walkers_energy(walk[:6], mode="lo", precision=precision)
    assert np.all(st2 == 0) and np.all(np.isfinite(e2))


def test_withheld_stage_times_out_and_context_recovers(chain_lo):
    """The LO tensor-core kernel is made to leave one pipeline stage of one CTA
    pair unfilled (no copy, no arrival).  Its bounded mbarrier waits run out
    after their 1 s limit, the kernel unwinds (waits for the copies it issued,
    frees TMEM) and the call returns LOAF_ERR_TIMEOUT instead of hanging.  The
    next call on the same context is correct again."""
    import time
    ctx, mol, walk = chain_lo
    ctx.test_withhold_stage(1)
    t0 = time.perf_counter()
    with pytest.raises(LoafError) as ei:
        ctx.walkers_energy(walk, mode="lo", precision="fp16x3")
    dt = time.perf_counter() - t0
    assert ei.value.status == "LOAF_ERR_TIMEOUT"
    assert dt < 30.0
    e, _, st = ctx.walkers_energy(walk, mode="lo", precision="fp16x3")
    assert np.all(st == 0)
    ref = np.array([E.walker_energy(mol, w)["E"] for w in walk[:4]])
    assert np.abs(e[:4] - ref).max() < TOL["fp16x3"]

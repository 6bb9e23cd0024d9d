"""Propagator one-body operator V_w = sum_g x_wg L_g (walkers_propagator)
against the oracle: FP64 (cuBLAS DGEMMs) to 1e-12 of max |V|, the split
precision (tensor cores, 16-bit hi + lo, 128-term chains) to 1e-6 of max |V|."""
import numpy as np
import pytest

from oracle import energy as E
from paper_2202_00832_b300 import synth
from paper_2202_00832_b300.lo_afqmc import Context

pytestmark = pytest.mark.gpu


def fields(W, X, seed):
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.standard_normal((W, X)) * 0.1 + 1j * rng.standard_normal((W, X)) * 0.05)


@pytest.mark.parametrize("case", ["chain", "ragged"])
def test_propagator_matches_oracle(chain60, case):
    import torch
    if case == "chain":
        mol, _ = chain60
        W = 40
    else:
        mol, _ = synth.small_case(37, 6, 75, 3, seed=17, n_beta=5)
        W = 5
    ctx = Context(0)
    ctx.load_molecule(mol)
    x = fields(W, mol.X, 3)
    ref = np.array([E.propagator_operator(mol, xw) for xw in x])
    scale = np.abs(ref).max()
    v64 = ctx.walkers_propagator(x, precision="fp64")
    assert np.abs(v64 - ref).max() < 1e-12 * scale
    v16 = ctx.walkers_propagator(x, precision="fp16x3")
    assert np.abs(v16 - ref).max() < 1e-6 * scale
    # device buffers give the same values
    xd = torch.from_numpy(x).cuda()
    vd = torch.zeros((W, mol.M, mol.M), dtype=torch.complex128, device="cuda")
    ctx.walkers_propagator(xd, precision="fp16x3", out=vd)
    assert np.array_equal(vd.cpu().numpy(), v16)

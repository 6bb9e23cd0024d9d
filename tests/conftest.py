import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session")
def chain60():
    """The 60-orbital chain (N=10, X=240) and its 32 walkers."""
    from paper_2202_00832_b300 import synth
    mol = synth.CHAIN_60.molecule()
    walkers = synth.CHAIN_60.walkers(mol)
    return mol, walkers

"""The C ABI library builds, loads without a GPU and exports every entry point
declared in include/*.h; host-side argument errors come back as status codes."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for path in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(path).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**"
                             r"([A-Za-z_][A-Za-z0-9_]*)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2202_00832_b300 import build, lo_afqmc
    build.build()
    return lo_afqmc.load_library()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["ao_load_cholesky", "lo_localize_compress", "walkers_energy",
                     "loaf_create", "loaf_destroy", "loaf_status_str"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_symbol():
    from paper_2202_00832_b300 import lo_afqmc
    bound = {s[0] for s in lo_afqmc.SIGNATURES}
    assert set(declared_functions()) <= bound


def test_status_strings(lib):
    for code in range(10):
        assert lib.loaf_status_str(code)
    assert b"unknown" in lib.loaf_status_str(99)


def test_null_arguments_return_status(lib):
    # no device work: argument checks fail before any CUDA call
    assert lib.loaf_create(None, 0, None) == 1
    assert lib.ao_load_cholesky(None, 1, 1, None, None, 1, 1, None, None, 0.0, 0) == 1
    assert lib.walkers_energy(None, 1, None, 0, 0, None, None, None) == 1
    assert lib.walkers_energy_submit(None, 1, None, 0, 0, None, None, None) == 1
    assert lib.walkers_energy_wait(None) == 1
    assert lib.loaf_destroy(None) == 0
    assert lib.loaf_num_pairs(None) == 0
    assert lib.loaf_set_tiles(None, 256, 0) == 1
    assert lib.loaf_get_tiles(None, None, None) == 1
    assert b"null" in lib.loaf_last_error(None)


def test_missing_library_fails_loudly(tmp_path):
    from paper_2202_00832_b300 import lo_afqmc
    saved = lo_afqmc._lib
    try:
        lo_afqmc._lib = None
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            lo_afqmc.load_library(str(tmp_path / "missing.so"))
    finally:
        lo_afqmc._lib = saved

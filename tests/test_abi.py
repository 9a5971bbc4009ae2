"""The C-ABI library builds, loads and exports every entry point include/ccsd.h declares.

Runs without a GPU: loading the library and resolving symbols makes no CUDA call."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ccsd.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ccsd_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1911_00242_gb300 import build
    if not os.path.exists(build.LIB) or os.path.getmtime(build.LIB) < max(
            os.path.getmtime(p) for p in build.SOURCES + [HEADER]):
        build.build()
    return build.LIB


def test_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    names = declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_binding_declares_every_symbol():
    from paper_1911_00242_gb300 import binding
    assert set(declared()) == set(binding.SYMBOLS)


def test_strerror_and_invalid_config_without_gpu(libpath):
    from paper_1911_00242_gb300 import binding
    lib = binding.load(libpath)
    assert lib.ccsd_strerror(-1).startswith(b"invalid")
    cfg = binding.make_config((0, 1, 1), 2, 3)
    n = ctypes.c_size_t(0)
    assert lib.ccsd_footprint(ctypes.byref(cfg), 1, ctypes.byref(n)) == binding.CCSD_ERR_INVALID
    cfg = binding.make_config((2, 2, 2), 8, 32, diis_depth=6)
    assert lib.ccsd_footprint(ctypes.byref(cfg), 1, ctypes.byref(n)) == 0
    assert 15e9 < n.value < 30e9
    h = ctypes.c_void_p()
    assert lib.ccsd_create(ctypes.byref(cfg), None, None, ctypes.byref(h)) == binding.CCSD_ERR_INVALID


def test_no_cpu_fallback_when_library_missing(tmp_path):
    from paper_1911_00242_gb300 import binding
    with pytest.raises(RuntimeError):
        binding.load.__wrapped__(str(tmp_path / "missing.so")) if hasattr(binding.load, "__wrapped__") \
            else _load_fresh(str(tmp_path / "missing.so"))


def _load_fresh(path):
    from paper_1911_00242_gb300 import binding
    saved = binding._lib
    binding._lib = None
    try:
        return binding.load(path)
    finally:
        binding._lib = saved


@pytest.mark.parametrize("grid,o,v", [((1, 1, 1), 3, 5), ((2, 1, 1), 2, 3), ((3, 2, 1), 5, 7),
                                      ((4, 1, 1), 4, 8), ((2, 2, 2), 8, 32), ((3, 3, 3), 8, 24),
                                      ((2, 2, 2), 1, 2)])
def test_plan_indices_in_bounds(libpath, grid, o, v):
    """Every launch of the residual plan stays inside its buffers (host-side check)."""
    from paper_1911_00242_gb300 import binding
    lib = binding.load(libpath)
    cfg = binding.make_config(grid, o, v)
    n = ctypes.c_longlong(0)
    tb = ctypes.c_size_t(0)
    assert lib.ccsd_plan_check(ctypes.byref(cfg), ctypes.byref(n), ctypes.byref(tb)) == 0
    assert 40 <= n.value <= 80


@pytest.mark.parametrize("grid,o,v", [((1, 1, 1), 3, 5), ((2, 1, 1), 2, 3), ((3, 2, 1), 5, 7),
                                      ((4, 1, 1), 4, 8), ((2, 2, 2), 8, 32), ((3, 3, 3), 8, 24),
                                      ((2, 2, 2), 1, 2), ((2, 2, 1), 8, 32)])
def test_mixed_plan_indices_in_bounds(libpath, grid, o, v):
    """The mixed form's plan, including the tensor-core GEMMs and operand embeddings."""
    from paper_1911_00242_gb300 import binding
    lib = binding.load(libpath)
    cfg = binding.make_config(grid, o, v, precision=binding.CCSD_MIXED)
    n = ctypes.c_longlong(0)
    tb = ctypes.c_size_t(0)
    assert lib.ccsd_plan_check(ctypes.byref(cfg), ctypes.byref(n), ctypes.byref(tb)) == 0
    assert n.value >= 50

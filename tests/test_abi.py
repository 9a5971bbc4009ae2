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
    assert lib.ccsd_footprint(ctypes.byref(cfg), 1, binding.CCSD_C128, ctypes.byref(n)) == binding.CCSD_ERR_INVALID
    cfg = binding.make_config((2, 2, 2), 8, 32, diis_depth=6)
    assert lib.ccsd_footprint(ctypes.byref(cfg), 1, 7, ctypes.byref(n)) == binding.CCSD_ERR_INVALID
    assert lib.ccsd_footprint(ctypes.byref(cfg), 1, binding.CCSD_C128, ctypes.byref(n)) == 0
    # the t2-sized arrays alone: amplitudes, residual, tau, tau~, W~_ring, the permuted
    # sum, plus 2 x 6 DIIS vectors over t1 and the canonical blocks (ki <= kj, ka <= kb)
    # of t2 (16 bytes per element)
    N, o, v = 8, 8, 32
    n1, n2 = N * o * v, N ** 3 * o * o * v * v
    c = [(x, y, z) for x in range(2) for y in range(2) for z in range(2)]
    ks = lambda a, b, d: tuple((a[i] + b[i] - d[i]) % 2 for i in range(3))
    nc = sum(1 for ki in range(N) for kj in range(ki, N) for ka in range(N)
             if ka <= c.index(ks(c[ki], c[kj], c[ka])))
    floor = (6 * n2 + 12 * (n1 + nc * o * o * v * v)) * 16
    assert floor < n.value < floor + 8e9
    borrowed = n.value
    # copied inputs add the integral bytes: complex128, or half of them as complex64
    ints = N ** 3 * (o ** 4 + o ** 3 * v + 2 * o * o * v * v + o * v ** 3 + v ** 4)
    m = ctypes.c_size_t(0)
    assert lib.ccsd_footprint(ctypes.byref(cfg), 0, binding.CCSD_C128, ctypes.byref(m)) == 0
    assert abs(m.value - borrowed - 16 * ints) < 1e6
    assert lib.ccsd_footprint(ctypes.byref(cfg), 0, binding.CCSD_C64, ctypes.byref(m)) == 0
    assert abs(m.value - borrowed - 8 * ints) < 1e6
    h = ctypes.c_void_p()
    assert lib.ccsd_create(ctypes.byref(cfg), None, None, ctypes.byref(h)) == binding.CCSD_ERR_INVALID
    # iteration limits and tolerances
    bad = [dict(max_iter=-1), dict(conv_tol=-1e-8), dict(conv_tol=float("nan")), dict(conv_tol=float("inf")),
           dict(precision=binding.CCSD_MIXED, mixed_tol=float("nan")),
           dict(precision=binding.CCSD_MIXED, mixed_tol=-1.0)]
    for kw in bad:
        cfg = binding.make_config((2, 2, 2), 8, 32, diis_depth=6, **kw)
        assert lib.ccsd_footprint(ctypes.byref(cfg), 1, binding.CCSD_C128, ctypes.byref(n)) == binding.CCSD_ERR_INVALID, kw
    for kw in (dict(max_iter=0), dict(conv_tol=0.0), dict(precision=binding.CCSD_MIXED, mixed_tol=0.0)):
        cfg = binding.make_config((2, 2, 2), 8, 32, diis_depth=6, **kw)
        assert lib.ccsd_footprint(ctypes.byref(cfg), 1, binding.CCSD_C128, ctypes.byref(n)) == 0, kw


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


@pytest.mark.parametrize("lean", [0, 1])
@pytest.mark.parametrize("grid,o,v", [((1, 1, 1), 3, 5), ((2, 1, 1), 2, 3), ((3, 2, 1), 5, 7),
                                      ((4, 1, 1), 4, 8), ((2, 2, 2), 8, 32), ((3, 3, 3), 8, 24),
                                      ((2, 2, 2), 1, 2)])
def test_plan_indices_in_bounds(libpath, grid, o, v, lean):
    """Every launch of the residual plan stays inside its buffers (host-side check)."""
    from paper_1911_00242_gb300 import binding
    lib = binding.load(libpath)
    cfg = binding.make_config(grid, o, v, lean=lean)
    n = ctypes.c_longlong(0)
    tb = ctypes.c_size_t(0)
    assert lib.ccsd_plan_check(ctypes.byref(cfg), ctypes.byref(n), ctypes.byref(tb)) == 0
    assert 40 <= n.value <= 120      # the ladder runs in W' slabs on large grids


@pytest.mark.parametrize("lean", [0, 1])
@pytest.mark.parametrize("grid,o,v", [((1, 1, 1), 3, 5), ((2, 1, 1), 2, 3), ((3, 2, 1), 5, 7),
                                      ((4, 1, 1), 4, 8), ((2, 2, 2), 8, 32), ((3, 3, 3), 8, 24),
                                      ((2, 2, 2), 1, 2), ((2, 2, 1), 8, 32), ((3, 1, 1), 2, 1)])
def test_mixed_plan_indices_in_bounds(libpath, grid, o, v, lean):
    """The mixed form's plan, including the tensor-core GEMMs and operand embeddings,
    in the default and in the lean (pooled operands, chunked ladder) layout."""
    from paper_1911_00242_gb300 import binding
    lib = binding.load(libpath)
    cfg = binding.make_config(grid, o, v, precision=binding.CCSD_MIXED, lean=lean)
    n = ctypes.c_longlong(0)
    tb = ctypes.c_size_t(0)
    assert lib.ccsd_plan_check(ctypes.byref(cfg), ctypes.byref(n), ctypes.byref(tb)) == 0
    assert n.value >= 50


@pytest.mark.parametrize("lean", [0, 1])
@pytest.mark.parametrize("slices", [0, 3, 8])
@pytest.mark.parametrize("grid,o,v", [((1, 1, 1), 3, 5), ((2, 1, 1), 2, 3), ((3, 2, 1), 5, 7),
                                      ((2, 2, 2), 8, 32), ((3, 3, 3), 8, 24), ((2, 2, 1), 8, 32),
                                      ((3, 1, 1), 2, 1)])
def test_ozaki_plan_indices_in_bounds(libpath, grid, o, v, lean, slices):
    """The Ozaki form's plan: the BF16 slice operands (pooled or not), the FP64 W' slices
    of the chunked ladder and the tensor-core GEMMs pass the host-side bounds checks."""
    from paper_1911_00242_gb300 import binding
    lib = binding.load(libpath)
    cfg = binding.make_config(grid, o, v, precision=binding.CCSD_OZAKI, lean=lean, oz_slices=slices)
    n = ctypes.c_longlong(0)
    tb = ctypes.c_size_t(0)
    assert lib.ccsd_plan_check(ctypes.byref(cfg), ctypes.byref(n), ctypes.byref(tb)) == 0
    assert n.value >= 50


def test_ozaki_config_validation(libpath):
    """Slice counts outside 3..8 and virtual spaces above 96 are refused; the batched form
    takes no Ozaki members."""
    from paper_1911_00242_gb300 import binding
    lib = binding.load(libpath)
    n = ctypes.c_longlong(0)
    tb = ctypes.c_size_t(0)
    for slices, v, ok in ((2, 8, False), (9, 8, False), (3, 8, True), (8, 8, True), (7, 97, False), (7, 96, True)):
        cfg = binding.make_config((1, 1, 1), 2, v, precision=binding.CCSD_OZAKI, oz_slices=slices)
        rc = lib.ccsd_plan_check(ctypes.byref(cfg), ctypes.byref(n), ctypes.byref(tb))
        assert (rc == 0) == ok, (slices, v, rc)


def test_ozaki_footprint_grows_with_slices(libpath):
    """Operand memory of the Ozaki form: 2 bytes per slice per embedded element."""
    from paper_1911_00242_gb300 import binding
    lib = binding.load(libpath)
    out = []
    for slices in (3, 5, 7):
        cfg = binding.make_config((2, 2, 1), 4, 16, precision=binding.CCSD_OZAKI, oz_slices=slices)
        b = ctypes.c_size_t(0)
        assert lib.ccsd_footprint(ctypes.byref(cfg), 1, binding.CCSD_C128, ctypes.byref(b)) == 0
        out.append(b.value)
    assert out[0] < out[1] < out[2]
    assert out[2] - out[1] == out[1] - out[0]      # linear in the slice count


def test_plan_describe_marks_tensor_core_alternatives(libpath):
    """The plan listing: the FP64 form has only always-on steps; the Ozaki form keeps each
    large FP64 GEMM as a native-FP64 alternative (mode 1) beside its tensor-core steps
    (mode 5); the mixed form's FP32-only fused steps run in mixed iterations only (mode 3),
    its tensor-core steps in mode 2, and with an Ozaki polish it carries both sets."""
    from paper_1911_00242_gb300 import binding
    binding.load(libpath)
    fp64 = binding.plan_describe((2, 2, 1), 4, 12)
    assert {m for (_, _, m, _) in fp64} == {0}
    oz = binding.plan_describe((2, 2, 1), 4, 12, precision=binding.CCSD_OZAKI)
    names_tc = {n for (n, k, m, _) in oz if k == 6}
    assert {"ladder", "ring", "ring_W_t2", "hole_hole", "hole_hole_W"} <= names_tc
    assert all(m == 5 for (_, k, m, _) in oz if k in (5, 6, 10))
    assert not any(k in (9, 11, 12) for (_, k, _, _) in oz)            # no FP32-only steps
    mixed = binding.plan_describe((2, 2, 1), 4, 12, precision=binding.CCSD_MIXED)
    assert all(m == 3 for (_, k, m, _) in mixed if k in (9, 11, 12))
    # the ladder's FP64 W' slabs and FP64 contractions are alternatives in both tensor-core forms
    for plan in (oz, mixed):
        assert any(n == "ladder" and k == 0 and m == 1 for (n, k, m, _) in plan)

    both = binding.plan_describe((2, 2, 1), 4, 12, precision=binding.CCSD_MIXED,
                                 polish_precision=binding.CCSD_OZAKI)
    tc2 = [n for (n, k, m, _) in both if k == 6 and m == 2]
    tc5 = [n for (n, k, m, _) in both if k == 6 and m == 5]
    assert sorted(tc2) == sorted(n for (n, k, m, _) in mixed if k == 6)
    assert sorted(tc5) == sorted(n for (n, k, m, _) in oz if k == 6)


@pytest.mark.parametrize("lean", [0, 1])
@pytest.mark.parametrize("grid,o,v", [((1, 1, 1), 3, 5), ((2, 1, 1), 2, 3), ((3, 2, 1), 5, 7),
                                      ((2, 2, 2), 8, 32), ((3, 3, 3), 8, 24), ((3, 1, 1), 2, 1)])
def test_mixed_with_ozaki_polish_plan_in_bounds(libpath, grid, o, v, lean):
    """A mixed handle with an Ozaki polish: both operand sets (split TF32 and BF16 slices),
    dedicated or viewing the same pools, pass the host-side bounds checks."""
    from paper_1911_00242_gb300 import binding
    lib = binding.load(libpath)
    cfg = binding.make_config(grid, o, v, precision=binding.CCSD_MIXED, lean=lean,
                              polish_precision=binding.CCSD_OZAKI)
    n = ctypes.c_longlong(0)
    tb = ctypes.c_size_t(0)
    assert lib.ccsd_plan_check(ctypes.byref(cfg), ctypes.byref(n), ctypes.byref(tb)) == 0
    # polish precision other than FP64 / Ozaki, or Ozaki polish on the FP64 form: refused
    for prec, pol in ((binding.CCSD_FP64, binding.CCSD_OZAKI), (binding.CCSD_MIXED, binding.CCSD_MIXED)):
        bad = binding.make_config(grid, o, v, precision=prec, polish_precision=pol)
        assert lib.ccsd_plan_check(ctypes.byref(bad), ctypes.byref(n), ctypes.byref(tb)) != 0


def test_binding_checks_sizes_dtypes_and_devices():
    """The library sees only pointers: the binding refuses arrays of the wrong size or
    dtype before any kernel reads them (host arrays; no GPU needed)."""
    import numpy as np
    from paper_1911_00242_gb300 import binding
    grid, o, v = (2, 1, 1), 2, 3
    n = binding.expected_sizes(grid, o, v)
    good = {k: np.zeros(n[k], np.complex128) for k in ("f_oo", "f_vv", "f_ov") + binding.BLOCKS}
    binding.check_arrays(grid, o, v, good, "t")
    c64 = dict(good, **{b: np.zeros(n[b], np.complex64) for b in binding.BLOCKS})
    binding.check_arrays(grid, o, v, c64, "t")               # complex64 integrals are allowed
    for name in ("f_oo", "ovvv", "vvvv"):
        bad = dict(good, **{name: np.zeros(n[name] - 1, np.complex128)})
        with pytest.raises(binding.CCSDError):
            binding.check_arrays(grid, o, v, bad, "t")
    with pytest.raises(binding.CCSDError):
        binding.check_arrays(grid, o, v, dict(good, f_ov=np.zeros(n["f_ov"], np.complex64)), "t")
    with pytest.raises(binding.CCSDError):
        binding.check_arrays(grid, o, v, {k: x for k, x in good.items() if k != "oovv"}, "t")
    with pytest.raises(binding.CCSDError):
        binding.check_arrays((0, 1, 1), o, v, good, "t")
    t1, t2 = np.zeros(n["t1"], np.complex128), np.zeros(n["t2"], np.complex128)
    binding.check_amplitudes(n, ((t1, "t1"), (t2, "t2")), "t", False)
    with pytest.raises(binding.CCSDError):                    # host arrays where device ones are needed
        binding.check_amplitudes(n, ((t1, "t1"), (t2, "t2")), "t", True)
    with pytest.raises(binding.CCSDError):
        binding.check_amplitudes(n, ((t1.astype(np.complex64), "t1"),), "t", False)
    with pytest.raises(binding.CCSDError):
        binding.check_amplitudes(n, ((t2, "t1"),), "t", False)
    with pytest.raises(binding.CCSDError):
        binding._ptr(np.zeros((4, 4), np.complex128)[:, ::2], "t")


def test_last_error_names_the_refused_field(libpath):
    """ccsd_last_error says why a config is refused; the binding's CCSDError carries it,
    and the next successful call on the thread clears it."""
    from paper_1911_00242_gb300 import binding
    lib = binding.load(libpath)
    n = ctypes.c_size_t(0)
    cases = [(dict(grid=(2, 1, 1), o=2, v=3, diis_depth=1), b"diis_depth"),
             (dict(grid=(2, 1, 1), o=2, v=3, conv_tol=float("nan")), b"conv_tol"),
             (dict(grid=(2, 1, 1), o=2, v=100, precision=binding.CCSD_OZAKI), b"nvir <= 96"),
             (dict(grid=(2, 1, 1), o=2, v=3, precision=binding.CCSD_OZAKI, oz_slices=2), b"oz_slices"),
             (dict(grid=(2, 1, 1), o=2, v=3, polish_precision=binding.CCSD_OZAKI), b"polish_precision"),
             (dict(grid=(65, 1, 1), o=2, v=3), b"nk_dims")]
    for kw, word in cases:
        kw = dict(kw)
        cfg = binding.make_config(kw.pop("grid"), kw.pop("o"), kw.pop("v"), **kw)
        assert lib.ccsd_footprint(ctypes.byref(cfg), 1, binding.CCSD_C128, ctypes.byref(n)) == binding.CCSD_ERR_INVALID
        assert word in lib.ccsd_last_error(), (word, lib.ccsd_last_error())
        with pytest.raises(binding.CCSDError) as e:
            binding.check(lib.ccsd_footprint(ctypes.byref(cfg), 1, binding.CCSD_C128, ctypes.byref(n)), "footprint")
        assert word.decode() in str(e.value)
    good = binding.make_config((2, 1, 1), 2, 3)
    assert lib.ccsd_footprint(ctypes.byref(good), 1, binding.CCSD_C128, ctypes.byref(n)) == 0
    assert lib.ccsd_last_error() == b""


def test_plans_beyond_32_bit_tables_are_refused_with_a_reason(libpath):
    """Tensor-core operand tables hold 32-bit row indices: a plan that would need more is
    refused on the host, with the reason (the problem is far beyond device memory)."""
    from paper_1911_00242_gb300 import binding
    lib = binding.load(libpath)
    for prec, grid, o, v in ((binding.CCSD_MIXED, (2, 2, 4), 33, 104), (binding.CCSD_OZAKI, (4, 2, 5), 2, 53)):
        cfg = binding.make_config(grid, o, v, precision=prec, lean=1)
        n, tb = ctypes.c_longlong(0), ctypes.c_size_t(0)
        assert lib.ccsd_plan_check(ctypes.byref(cfg), ctypes.byref(n), ctypes.byref(tb)) == binding.CCSD_ERR_INVALID
        assert b"32-bit" in lib.ccsd_last_error(), lib.ccsd_last_error()


def test_random_plans_in_bounds(libpath):
    """A seeded sweep over configurations of every form, layout and DIIS depth: each plan
    builds, every launch stays inside its buffers (ccsd_plan_check), and the footprint of
    the same config is defined."""
    import random
    from paper_1911_00242_gb300 import binding
    lib = binding.load(libpath)
    rng = random.Random(2024)
    checked = 0
    while checked < 300:
        grid = tuple(rng.choice([1, 1, 2, 2, 3]) for _ in range(3))
        N = grid[0] * grid[1] * grid[2]
        o, v = rng.randint(1, 10), rng.randint(1, 34)
        if N ** 3 * v ** 4 * 16 > 20e9:
            continue
        prec = rng.choice([binding.CCSD_FP64, binding.CCSD_MIXED, binding.CCSD_OZAKI])
        pol = binding.CCSD_OZAKI if prec == binding.CCSD_MIXED and rng.random() < 0.4 else binding.CCSD_FP64
        sl = rng.choice([0, 3, 8]) if binding.CCSD_OZAKI in (prec, pol) else 0
        cfg = binding.make_config(grid, o, v, precision=prec, lean=rng.choice([0, 1]), oz_slices=sl,
                                  polish_precision=pol, diis_depth=rng.choice([0, 2, 6, 8]))
        n, tb, fp = ctypes.c_longlong(0), ctypes.c_size_t(0), ctypes.c_size_t(0)
        assert lib.ccsd_plan_check(ctypes.byref(cfg), ctypes.byref(n), ctypes.byref(tb)) == 0, \
            (grid, o, v, prec, pol, lib.ccsd_last_error())
        assert lib.ccsd_footprint(ctypes.byref(cfg), 1, binding.CCSD_C128, ctypes.byref(fp)) == 0
        assert n.value > 0 and fp.value > 0
        checked += 1


def test_contraction_flops_scale_as_nk4():
    """The paper's cost claim: at fixed bands the contractions grow as N_k^4.  From the
    host-built plan (ccsd_plan_describe, FP64 steps): the ring is exactly 8 N_k^4 o^3 v^3
    real flops; the antisymmetry-packed ladder and hole-hole contractions pack pairs of
    combined (k, orbital) indices, so their N_k^4 ratio approaches a constant near
    (v / (v - 1))^2 from 1."""
    from collections import defaultdict
    from paper_1911_00242_gb300 import binding
    o, v = 4, 12
    flops = {}
    for grid in [(1, 1, 1), (2, 1, 1), (2, 2, 1), (3, 1, 1), (2, 2, 2), (3, 3, 1)]:
        agg = defaultdict(float)
        for name, kind, mode, fl in binding.plan_describe(grid, o, v):
            if mode in (0, 1):
                agg[name] += fl
        N = grid[0] * grid[1] * grid[2]
        flops[N] = agg
        assert agg["ring"] == 8.0 * N ** 4 * o ** 3 * v ** 3
    prev = {"ladder": 1.0, "hole_hole": 1.0}
    for N in sorted(flops):
        for name in prev:
            r = flops[N][name] / flops[1][name] / N ** 4
            assert prev[name] - 1e-12 <= r <= 1.5, (name, N, r)      # non-decreasing, bounded
            prev[name] = r

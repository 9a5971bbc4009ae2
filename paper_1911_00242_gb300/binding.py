"""ctypes binding of libccsd_gb300.so (argument marshalling only).

Every function of include/ccsd.h is exposed under the same name on the object
returned by `load()`.  `Solver` wraps a handle for torch tensors or numpy
arrays: device tensors are borrowed by pointer, host arrays are copied by the
library.  There is no CPU fallback: without the built library every call raises.
"""
import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libccsd_gb300.so")

CCSD_OK = 0
CCSD_ERR_INVALID = -1
CCSD_ERR_OOM = -2
CCSD_ERR_CUDA = -3
CCSD_ERR_NOT_CONVERGED = -4
CCSD_ERR_DIVERGED = -5
CCSD_ERR_TIMEOUT = -6
CCSD_FP64 = 0
CCSD_MIXED = 1
CCSD_OZAKI = 2
CCSD_C128 = 0
CCSD_C64 = 1

BLOCKS = ("oooo", "ooov", "oovv", "ovvo", "ovvv", "vvvv")


class ccsd_config(ctypes.Structure):
    _fields_ = [("nk_dims", ctypes.c_int * 3), ("nocc", ctypes.c_int), ("nvir", ctypes.c_int),
                ("precision", ctypes.c_int), ("diis_depth", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("conv_tol", ctypes.c_double), ("polish_iters", ctypes.c_int), ("mixed_tol", ctypes.c_double),
                ("lean", ctypes.c_int), ("oz_slices", ctypes.c_int), ("polish_precision", ctypes.c_int)]


class ccsd_inputs(ctypes.Structure):
    _fields_ = [("f_oo", ctypes.c_void_p), ("f_vv", ctypes.c_void_p), ("f_ov", ctypes.c_void_p),
                ("oooo", ctypes.c_void_p), ("ooov", ctypes.c_void_p), ("oovv", ctypes.c_void_p),
                ("ovvo", ctypes.c_void_p), ("ovvv", ctypes.c_void_p), ("vvvv", ctypes.c_void_p),
                ("int_dtype", ctypes.c_int), ("vvvv_on_host", ctypes.c_int)]


SYMBOLS = {
    "ccsd_create": ([ctypes.POINTER(ccsd_config), ctypes.POINTER(ccsd_inputs), ctypes.c_void_p,
                     ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "ccsd_footprint": ([ctypes.POINTER(ccsd_config), ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)],
                       ctypes.c_int),
    "ccsd_plan_check": ([ctypes.POINTER(ccsd_config), ctypes.POINTER(ctypes.c_longlong),
                         ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "ccsd_plan_describe": ([ctypes.POINTER(ccsd_config), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                            ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                            ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "ccsd_tc_selftest": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_ulonglong,
                          ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "ccsd_tc_timeout_selftest": ([], ctypes.c_int),
    "ccsd_oz_gemm": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                      ctypes.c_void_p], ctypes.c_int),
    "ccsd_oz_timeout_selftest": ([], ctypes.c_int),
    "ccsd_residual": ([ctypes.c_void_p] * 5, ctypes.c_int),
    "ccsd_iterate": ([ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                      ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "ccsd_solve": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "ccsd_set_precision": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "ccsd_energy": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "ccsd_get_amplitudes": ([ctypes.c_void_p] * 3, ctypes.c_int),
    "ccsd_set_amplitudes": ([ctypes.c_void_p] * 3, ctypes.c_int),
    "ccsd_last_launch_count": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong)], ctypes.c_int),
    "ccsd_trace_enable": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "ccsd_trace_count": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "ccsd_trace_step": ([ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p),
                         ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double),
                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "ccsd_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "ccsd_batch_create": ([ctypes.c_int, ctypes.POINTER(ccsd_config), ctypes.POINTER(ccsd_inputs),
                           ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "ccsd_batch_iterate": ([ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                            ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "ccsd_batch_energy": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
                          ctypes.c_int),
    "ccsd_batch_member": ([ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "ccsd_batch_stats": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_int),
                          ctypes.c_int], ctypes.c_int),
    "ccsd_batch_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "ccsd_server_create": ([ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)],
                           ctypes.c_int),
    "ccsd_submit": ([ctypes.c_void_p, ctypes.POINTER(ccsd_config), ctypes.POINTER(ccsd_inputs),
                     ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "ccsd_poll": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "ccsd_server_stats": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                           ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "ccsd_server_profile": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
                            + [ctypes.POINTER(ctypes.c_double)] * 4, ctypes.c_int),
    "ccsd_server_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "ccsd_strerror": ([ctypes.c_int], ctypes.c_char_p),
    "ccsd_last_error": ([], ctypes.c_char_p),
    "ccsd_fp64_peak_probe": ([ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "ccsd_energy_noalloc": ([ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int] + [ctypes.c_void_p] * 6,
                            ctypes.c_int),
}

_lib = None


class CCSDError(RuntimeError):
    def __init__(self, code, where, detail=None):
        self.code = code
        msg = _lib.ccsd_strerror(code).decode() if _lib is not None else str(code)
        self.detail = detail or ""
        super().__init__(f"{where}: {msg} ({code})" + (f": {self.detail}" if self.detail else ""))


def load(path=LIB_PATH):
    """Load the library and declare every exported signature; raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (args, res) in SYMBOLS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def check(code, where):
    if code != CCSD_OK:
        raise CCSDError(code, where, _lib.ccsd_last_error().decode() if _lib is not None else None)
    return code


def _invalid(where):
    return CCSDError(CCSD_ERR_INVALID, where)


def _ptr(x, where="argument"):
    """Device or host address of a torch tensor or numpy array (must be contiguous)."""
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise _invalid(f"{where}: tensor is not contiguous")
        return x.data_ptr()
    if not x.flags.c_contiguous:
        raise _invalid(f"{where}: array is not C-contiguous")
    return x.ctypes.data


def _numel(x):
    return x.numel() if hasattr(x, "numel") else int(x.size)


def _dtype(x):
    return str(x.dtype).replace("torch.", "")


def _on_device(x):
    return bool(getattr(x, "is_cuda", False))


def expected_sizes(grid, nocc, nvir):
    """Complex elements of every input and amplitude array (layouts of include/ccsd.h)."""
    N = grid[0] * grid[1] * grid[2]
    N3, o, v = N ** 3, nocc, nvir
    return {"f_oo": N * o * o, "f_vv": N * v * v, "f_ov": N * o * v,
            "oooo": N3 * o ** 4, "ooov": N3 * o ** 3 * v, "oovv": N3 * o * o * v * v,
            "ovvo": N3 * o * o * v * v, "ovvv": N3 * o * v ** 3, "vvvv": N3 * v ** 4,
            "t1": N * o * v, "t2": N3 * o * o * v * v}


def check_arrays(grid, nocc, nvir, arrays, where):
    """The library sees only pointers: check the element counts of the inputs and the
    dtype of the Fock blocks here, before any kernel reads them."""
    n = expected_sizes(grid, nocc, nvir)
    for name in ("f_oo", "f_vv", "f_ov") + BLOCKS:
        if name not in arrays:
            raise _invalid(f"{where}: missing input {name}")
        if _numel(arrays[name]) != n[name]:
            raise _invalid(f"{where}: {name} has {_numel(arrays[name])} elements, expected {n[name]}")
    for name in ("f_oo", "f_vv", "f_ov"):
        if _dtype(arrays[name]) != "complex128":
            raise _invalid(f"{where}: {name} must be complex128, got {_dtype(arrays[name])}")


def check_amplitudes(n, pairs, where, device):
    """(array, name) pairs of complex128 amplitude-shaped arrays with n[name] elements,
    device tensors when `device`."""
    for x, name in pairs:
        if _dtype(x) != "complex128":
            raise _invalid(f"{where}: {name} must be complex128, got {_dtype(x)}")
        if _numel(x) != n[name]:
            raise _invalid(f"{where}: {name} has {_numel(x)} elements, expected {n[name]}")
        if device and not _on_device(x):
            raise _invalid(f"{where}: {name} must be a CUDA tensor")


def int_dtype(arrays):
    """CCSD_C128 or CCSD_C64 from the element type of the six integral blocks
    (all must agree; the Fock blocks are always complex128)."""
    kinds = {str(arrays[b].dtype).replace("torch.", "") for b in BLOCKS}
    if kinds == {"complex128"}:
        return CCSD_C128
    if kinds == {"complex64"}:
        return CCSD_C64
    raise ValueError(f"integral blocks must all be complex128 or all complex64, got {sorted(kinds)}")


def inputs_struct(arrays, vvvv_on_host=False):
    inp = ccsd_inputs()
    for name in ("f_oo", "f_vv", "f_ov") + BLOCKS:
        setattr(inp, name, _ptr(arrays[name], name))
    inp.int_dtype = int_dtype(arrays)
    inp.vvvv_on_host = 1 if vvvv_on_host else 0
    return inp


def make_config(grid, nocc, nvir, precision=CCSD_FP64, diis_depth=0, max_iter=100, conv_tol=1e-8,
                polish_iters=2, mixed_tol=1e-7, lean=0, oz_slices=0, polish_precision=CCSD_FP64):
    c = ccsd_config()
    c.nk_dims[0], c.nk_dims[1], c.nk_dims[2] = grid
    c.nocc, c.nvir, c.precision = nocc, nvir, precision
    c.diis_depth, c.max_iter, c.conv_tol = diis_depth, max_iter, conv_tol
    c.polish_iters, c.mixed_tol = polish_iters, mixed_tol
    c.lean = lean
    c.oz_slices = oz_slices
    c.polish_precision = polish_precision
    return c


class Solver:
    """One CCSD problem held by a library handle.

    `arrays` maps f_oo, f_vv, f_ov (complex128) and the six block names
    (all complex128 or all complex64) to contiguous torch tensors (device:
    borrowed, kept referenced here) or numpy arrays (host: copied by the
    library during creation; with vvvv_on_host a host vvvv is read in place
    instead, and must stay alive with the solver)."""

    def __init__(self, grid, nocc, nvir, arrays, stream=None, vvvv_on_host=False, **cfg):
        self.lib = load()
        self.cfg = make_config(grid, nocc, nvir, **cfg)
        check_arrays(grid, nocc, nvir, arrays, "Solver")
        self.sizes = expected_sizes(grid, nocc, nvir)
        self._keep = dict(arrays)
        inp = inputs_struct(arrays, vvvv_on_host)
        h = ctypes.c_void_p()
        check(self.lib.ccsd_create(ctypes.byref(self.cfg), ctypes.byref(inp), stream, ctypes.byref(h)), "ccsd_create")
        self.h = h

    def residual(self, t1, t2, r1, r2):
        check_amplitudes(self.sizes, ((t1, "t1"), (t2, "t2"), (r1, "t1"), (r2, "t2")), "residual", True)
        check(self.lib.ccsd_residual(self.h, _ptr(t1), _ptr(t2), _ptr(r1), _ptr(r2)), "ccsd_residual")

    def iterate(self, n=1):
        done = ctypes.c_int(0)
        mr = ctypes.c_double(0.0)
        check(self.lib.ccsd_iterate(self.h, n, ctypes.byref(done), ctypes.byref(mr)), "ccsd_iterate")
        return bool(done.value), mr.value

    def solve(self):
        it = ctypes.c_int(0)
        mr = ctypes.c_double(0.0)
        code = self.lib.ccsd_solve(self.h, ctypes.byref(it), ctypes.byref(mr))
        if code not in (CCSD_OK, CCSD_ERR_NOT_CONVERGED):
            check(code, "ccsd_solve")
        return code == CCSD_OK, it.value, mr.value

    def set_precision(self, precision):
        check(self.lib.ccsd_set_precision(self.h, precision), "ccsd_set_precision")

    def energy(self):
        er = ctypes.c_double(0.0)
        ei = ctypes.c_double(0.0)
        check(self.lib.ccsd_energy(self.h, ctypes.byref(er), ctypes.byref(ei)), "ccsd_energy")
        return complex(er.value, ei.value)

    def get_amplitudes(self, t1, t2):
        check_amplitudes(self.sizes, ((t1, "t1"), (t2, "t2")), "get_amplitudes", False)
        check(self.lib.ccsd_get_amplitudes(self.h, _ptr(t1), _ptr(t2)), "ccsd_get_amplitudes")

    def set_amplitudes(self, t1, t2):
        check_amplitudes(self.sizes, ((t1, "t1"), (t2, "t2")), "set_amplitudes", False)
        check(self.lib.ccsd_set_amplitudes(self.h, _ptr(t1), _ptr(t2)), "ccsd_set_amplitudes")

    def launches(self):
        n = ctypes.c_longlong(0)
        check(self.lib.ccsd_last_launch_count(self.h, ctypes.byref(n)), "ccsd_last_launch_count")
        return n.value

    def trace(self, enable=True):
        check(self.lib.ccsd_trace_enable(self.h, 1 if enable else 0), "ccsd_trace_enable")

    def trace_steps(self):
        """[(name, calls, total_ms, flops_per_call, bytes_per_call)] in launch order."""
        n = ctypes.c_int(0)
        check(self.lib.ccsd_trace_count(self.h, ctypes.byref(n)), "ccsd_trace_count")
        out = []
        for i in range(n.value):
            nm = ctypes.c_char_p()
            calls = ctypes.c_longlong(0)
            ms, fl, by = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_double(0)
            check(self.lib.ccsd_trace_step(self.h, i, ctypes.byref(nm), ctypes.byref(calls), ctypes.byref(ms),
                                           ctypes.byref(fl), ctypes.byref(by)), "ccsd_trace_step")
            out.append((nm.value.decode(), calls.value, ms.value, fl.value, by.value))
        return out

    def close(self):
        if getattr(self, "h", None):
            self.lib.ccsd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchSolver:
    """Many independent problems iterated together (grouped launches, CUDA graph).

    `problems` is a list of (grid, nocc, nvir, arrays) with arrays as for Solver."""

    def __init__(self, problems, **cfg):
        self.lib = load()
        n = len(problems)
        cfgs = (ccsd_config * n)()
        ins = (ccsd_inputs * n)()
        self._keep = []
        self.sizes = []
        for i, (grid, nocc, nvir, arrays) in enumerate(problems):
            cfgs[i] = make_config(grid, nocc, nvir, **cfg)
            check_arrays(grid, nocc, nvir, arrays, f"BatchSolver member {i}")
            ins[i] = inputs_struct(arrays)
            self._keep.append(arrays)
            self.sizes.append(expected_sizes(grid, nocc, nvir))
        self.n = n
        h = ctypes.c_void_p()
        check(self.lib.ccsd_batch_create(n, cfgs, ins, ctypes.byref(h)), "ccsd_batch_create")
        self.h = h

    def iterate(self, n_iter=1):
        done = (ctypes.c_int * self.n)()
        mr = (ctypes.c_double * self.n)()
        check(self.lib.ccsd_batch_iterate(self.h, n_iter, done, mr), "ccsd_batch_iterate")
        return [bool(x) for x in done], list(mr)

    def energies(self):
        er = (ctypes.c_double * self.n)()
        ei = (ctypes.c_double * self.n)()
        check(self.lib.ccsd_batch_energy(self.h, er, ei), "ccsd_batch_energy")
        return [complex(a, b) for a, b in zip(er, ei)]

    def member_amplitudes(self, i, t1, t2):
        if not 0 <= i < self.n:
            raise _invalid(f"member_amplitudes: member {i} of {self.n}")
        check_amplitudes(self.sizes[i], ((t1, "t1"), (t2, "t2")), "member_amplitudes", False)
        h = ctypes.c_void_p()
        check(self.lib.ccsd_batch_member(self.h, i, ctypes.byref(h)), "ccsd_batch_member")
        check(self.lib.ccsd_get_amplitudes(h, _ptr(t1), _ptr(t2)), "ccsd_get_amplitudes")

    def stats(self, max_cfgs=64):
        n = ctypes.c_longlong(0)
        cfgs = (ctypes.c_int * max_cfgs)()
        check(self.lib.ccsd_batch_stats(self.h, ctypes.byref(n), cfgs, max_cfgs), "ccsd_batch_stats")
        return n.value, list(cfgs)

    def close(self):
        if getattr(self, "h", None):
            self.lib.ccsd_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """The serving loop: submit solves, poll for results (see ccsd_server_* in include/ccsd.h)."""

    def __init__(self, hbm_budget_bytes, max_slots, stream=None):
        self.lib = load()
        h = ctypes.c_void_p()
        check(self.lib.ccsd_server_create(int(hbm_budget_bytes), int(max_slots), stream, ctypes.byref(h)),
              "ccsd_server_create")
        self.h = h
        self._keep = {}

    def submit(self, grid, nocc, nvir, arrays, **cfg):
        c = make_config(grid, nocc, nvir, **cfg)
        check_arrays(grid, nocc, nvir, arrays, "submit")
        inp = inputs_struct(arrays)
        rid = ctypes.c_uint64(0)
        check(self.lib.ccsd_submit(self.h, ctypes.byref(c), ctypes.byref(inp), ctypes.byref(rid)), "ccsd_submit")
        self._keep[rid.value] = arrays
        return rid.value

    def poll(self, rid):
        st = ctypes.c_int(0)
        e = ctypes.c_double(0.0)
        t = ctypes.c_double(0.0)
        it = ctypes.c_int(0)
        check(self.lib.ccsd_poll(self.h, rid, ctypes.byref(st), ctypes.byref(e), ctypes.byref(t), ctypes.byref(it)),
              "ccsd_poll")
        if st.value == 2 or st.value < 0:
            self._keep.pop(rid, None)
        return st.value, e.value, t.value, it.value

    def stats(self):
        a = ctypes.c_int(0)
        q = ctypes.c_int(0)
        b = ctypes.c_size_t(0)
        check(self.lib.ccsd_server_stats(self.h, ctypes.byref(a), ctypes.byref(q), ctypes.byref(b)), "ccsd_server_stats")
        return a.value, q.value, b.value

    def profile(self):
        """dict: rounds, group builds, seconds in rounds and in building groups, and the
        mean wait for admission and mean run time of the finished solves."""
        r, b = ctypes.c_longlong(0), ctypes.c_longlong(0)
        x = [ctypes.c_double(0.0) for _ in range(4)]
        check(self.lib.ccsd_server_profile(self.h, ctypes.byref(r), ctypes.byref(b), *[ctypes.byref(v) for v in x]),
              "ccsd_server_profile")
        return {"rounds": r.value, "group_builds": b.value, "round_s": x[0].value, "group_build_s": x[1].value,
                "mean_wait_s": x[2].value, "mean_run_s": x[3].value}

    def close(self):
        if getattr(self, "h", None):
            self.lib.ccsd_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def oz_gemm(A, B, slices=7):
    """C = A B^T (complex128 numpy arrays, A: M x K, B: Ncols x K) through the
    Ozaki-scheme tensor-core kernels of CCSD_OZAKI (ccsd_oz_gemm)."""
    import numpy as np
    lib = load()
    A = np.ascontiguousarray(A, dtype=np.complex128)
    B = np.ascontiguousarray(B, dtype=np.complex128)
    M, K = A.shape
    Nc, K2 = B.shape
    assert K == K2
    C = np.empty((M, Nc), dtype=np.complex128)
    check(lib.ccsd_oz_gemm(M, Nc, K, slices, A.ctypes.data, B.ctypes.data, C.ctypes.data), "ccsd_oz_gemm")
    return C


def plan_describe(grid, nocc, nvir, **cfg):
    """The launch plan of a config (host only): a list of (name, kind, mode, flops)."""
    lib = load()
    c = make_config(grid, nocc, nvir, **cfg)
    n = ctypes.c_int(0)
    check(lib.ccsd_plan_describe(ctypes.byref(c), 0, None, None, None, None, ctypes.byref(n)), "ccsd_plan_describe")
    k = (ctypes.c_int * n.value)()
    m = (ctypes.c_int * n.value)()
    f = (ctypes.c_double * n.value)()
    nm = (ctypes.c_char_p * n.value)()
    check(lib.ccsd_plan_describe(ctypes.byref(c), n.value, k, m, f, nm, ctypes.byref(n)), "ccsd_plan_describe")
    return [(nm[i].decode(), k[i], m[i], f[i]) for i in range(n.value)]

"""ctypes binding of libmsp (include/msp.h): argument marshalling only.

Every step of a solve runs inside libmsp's CUDA kernels.  When the library is
missing, or no CUDA device is visible, these calls raise :class:`MspError`;
there is no CPU fallback.

Masks follow the library convention: a solution is a tuple of
ceil(n / 64) little-endian 64-bit words, bit j of word j // 64 being x_j;
lists are sorted ascending as unsigned integers.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libmsp.so")
_lock = threading.Lock()
_lib = None

EXPORTED_SYMBOLS = (
    "msp_create", "msp_destroy", "msp_set_stream", "msp_set_memory_budget", "msp_solve_all",
    "msp_get_stats", "msp_free_solutions", "msp_set_profiling", "msp_set_option", "msp_solve_batch", "msp_server_create", "msp_submit",
    "msp_poll", "msp_cancel", "msp_server_destroy", "msp_last_error", "msp_version",
    "msp_solve_small_noalloc", "msp_device_name", "msp_solve_batch_path", "msp_plan",
)

# msp_set_option codes (include/msp.h)
OPT_EXACT_PATH, OPT_CLASS_PART, OPT_CLASS_PARTS = 1, 2, 3
OPT_CLASS_BITS, OPT_DIGIT_BITS, OPT_INNER_BITS = 4, 5, 6
OPT_DIRECT, OPT_TABLE_BITS, OPT_FIRST = 7, 8, 9
OPT_WAIT_LIMIT_US, OPT_WAIT_CHECK = 10, 11
PLAN_KEYS = {"class_bits": OPT_CLASS_BITS, "digit_bits": OPT_DIGIT_BITS, "inner_bits": OPT_INNER_BITS,
             "direct": OPT_DIRECT, "table_bits": OPT_TABLE_BITS}

STATUS = {0: "MSP_OK", 1: "MSP_PENDING", -1: "MSP_EINVAL", -2: "MSP_ERANGE", -3: "MSP_ENOMEM",
          -4: "MSP_ECUDA", -5: "MSP_ETIMEDOUT", -6: "MSP_EOVERFLOW", -7: "MSP_ECANCELED"}


class MspError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


# device-memory budget of a solve or a server when the caller passes 0
BUDGET_ENV = "MSP_MEMORY_BUDGET"
_UNITS = {"": 1, "K": 1 << 10, "M": 1 << 20, "G": 1 << 30, "T": 1 << 40}


def parse_bytes(text: str) -> int:
    """A byte count: an integer with an optional K, M, G or T suffix
    (powers of 1024, an optional trailing B), e.g. "150G", "1500MB", "4096"."""
    t = str(text).strip().upper()
    if t.endswith("B"):
        t = t[:-1]
    unit = t[-1:] if t[-1:] in _UNITS and t[-1:] != "" else ""
    num = t[:-1] if unit else t
    try:
        value = float(num)
    except ValueError:
        raise MspError(-1, f"not a byte count: {text!r}") from None
    if not (0 <= value < float(1 << 62)):  # also rejects nan and inf
        raise MspError(-1, f"not a byte count: {text!r}")
    return int(value * _UNITS[unit])


def default_budget() -> int:
    """$MSP_MEMORY_BUDGET in bytes, or 0 (the library's own default: 85 % of
    the free device memory) when it is unset or empty."""
    v = os.environ.get(BUDGET_ENV, "").strip()
    return parse_bytes(v) if v else 0


class Stats(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("n", ctypes.c_int), ("quarter", ctypes.c_int * 4),
                ("class_bits", ctypes.c_int), ("class_rows", ctypes.c_int), ("digit_bits", ctypes.c_int),
                ("passes", ctypes.c_int), ("records_left", ctypes.c_uint64),
                ("records_right", ctypes.c_uint64), ("row1_candidates_lo", ctypes.c_uint64),
                ("row1_candidates_hi", ctypes.c_uint64), ("key_matches", ctypes.c_uint64),
                ("pairs_verified", ctypes.c_uint64), ("solutions", ctypes.c_uint64),
                ("oversize_segments", ctypes.c_uint64), ("device_bytes", ctypes.c_uint64),
                ("ms_total", ctypes.c_double), ("kernel_launches", ctypes.c_uint64),
                ("fast_passes_redone", ctypes.c_uint64), ("h2d_bytes", ctypes.c_uint64), ("d2h_bytes", ctypes.c_uint64),
                ("classes_total", ctypes.c_uint64), ("classes_done", ctypes.c_uint64),
                ("records_done", ctypes.c_uint64), ("path", ctypes.c_int), ("direct_fallback", ctypes.c_int),
                ("kernel_ms", ctypes.c_double * 12), ("kernel_count", ctypes.c_uint64 * 12),
                ("kernel_bytes", ctypes.c_uint64 * 12)]

    KINDS = ("gray", "bucket", "c1", "gen_count", "offsets", "gen_scatter", "join", "join_big",
             "recover", "verify", "other", "direct")
    PATHS = ("streaming", "direct")

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["quarter"] = list(self.quarter)
        d["path"] = self.PATHS[self.path] if 0 <= self.path < len(self.PATHS) else self.path
        d["row1_candidates"] = int(self.row1_candidates_lo) | (int(self.row1_candidates_hi) << 64)
        d["kernels"] = {k: {"ms": self.kernel_ms[i], "launches": int(self.kernel_count[i]),
                            "bytes": int(self.kernel_bytes[i])}
                        for i, k in enumerate(self.KINDS) if self.kernel_count[i]}
        for k in ("kernel_ms", "kernel_count", "kernel_bytes"):
            d.pop(k)
        return d


class PlanInfo(ctypes.Structure):
    """msp_plan_info (include/msp.h)."""
    _fields_ = [("path", ctypes.c_int), ("class_bits", ctypes.c_int), ("class_rows", ctypes.c_int),
                ("quarter", ctypes.c_int * 4), ("digit_bits", ctypes.c_int), ("table_bits", ctypes.c_int),
                ("records_left", ctypes.c_uint64), ("records_right", ctypes.c_uint64),
                ("device_bytes", ctypes.c_uint64)]


def plan_info(m: int, n: int) -> dict:
    """``msp_plan``: the plan a solve of an (m, n) instance takes by default
    (host only, no device needed)."""
    lib = load_library()
    out = PlanInfo()
    _check(lib.msp_plan(int(m), int(n), ctypes.byref(out)))
    d = {k: getattr(out, k) for k, _ in PlanInfo._fields_}
    d["quarter"] = list(out.quarter)
    d["path"] = Stats.PATHS[out.path]
    return d


def lib_path() -> str:
    return _LIB_PATH


def load_library(path: str | None = None):
    """Load libmsp.so (built by ``paper_2507_05045_gb300.build.build()``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or _LIB_PATH
        if not os.path.exists(p):
            raise MspError(-4, f"{p} is missing: build it with paper_2507_05045_gb300.build.build()")
        lib = ctypes.CDLL(p)
        i32p = ctypes.POINTER(ctypes.c_int32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        vp = ctypes.c_void_p
        lib.msp_create.argtypes = [i32p, i32p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp)]
        lib.msp_create.restype = ctypes.c_int
        lib.msp_destroy.argtypes = [vp]
        lib.msp_destroy.restype = None
        lib.msp_set_stream.argtypes = [vp, vp]
        lib.msp_set_memory_budget.argtypes = [vp, ctypes.c_size_t]
        lib.msp_set_profiling.argtypes = [vp, ctypes.c_int]
        lib.msp_set_option.argtypes = [vp, ctypes.c_int, ctypes.c_int64]
        lib.msp_solve_all.argtypes = [vp, ctypes.POINTER(u64p), ctypes.POINTER(ctypes.c_size_t),
                                      ctypes.POINTER(ctypes.c_int)]
        lib.msp_solve_all.restype = ctypes.c_int
        lib.msp_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
        lib.msp_free_solutions.argtypes = [u64p]
        lib.msp_free_solutions.restype = None
        lib.msp_solve_batch.argtypes = [ctypes.POINTER(i32p), ctypes.POINTER(i32p), ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.POINTER(u64p), ctypes.POINTER(ctypes.c_size_t)]
        lib.msp_solve_batch_path.argtypes = [ctypes.POINTER(i32p), ctypes.POINTER(i32p), ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_int, ctypes.POINTER(u64p),
                                             ctypes.POINTER(ctypes.c_size_t)]
        lib.msp_server_create.argtypes = [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(vp)]
        lib.msp_submit.argtypes = [vp, i32p, i32p, ctypes.c_int, ctypes.c_int, u64p]
        lib.msp_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(u64p), ctypes.POINTER(ctypes.c_size_t),
                                 ctypes.POINTER(ctypes.c_int)]
        lib.msp_cancel.argtypes = [vp, ctypes.c_uint64]
        lib.msp_server_destroy.argtypes = [vp]
        lib.msp_server_destroy.restype = None
        lib.msp_solve_small_noalloc.argtypes = [i32p, i32p, ctypes.c_int, ctypes.c_int, u64p, ctypes.c_size_t,
                                                ctypes.POINTER(ctypes.c_size_t), vp]
        lib.msp_solve_small_noalloc.restype = ctypes.c_int
        lib.msp_last_error.restype = ctypes.c_char_p
        lib.msp_version.restype = ctypes.c_char_p
        lib.msp_device_name.restype = ctypes.c_char_p
        lib.msp_plan.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(PlanInfo)]
        lib.msp_plan.restype = ctypes.c_int
        _lib = lib
        return lib


def _check(rc: int):
    if rc < 0:
        raise MspError(rc, load_library().msp_last_error().decode())
    return rc


def _i32(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.int32))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _take_masks(lib, ptr, count: int, words: int):
    if count == 0:
        return []
    arr = np.ctypeslib.as_array(ptr, shape=(count * words,)).copy()
    lib.msp_free_solutions(ptr)
    return [tuple(int(w) for w in arr[i * words:(i + 1) * words]) for i in range(count)]


class Instance:
    """One (A, d) instance: ``msp_create`` / ``msp_solve_all`` / ``msp_destroy``."""

    def __init__(self, A, d, stream: int | None = None, memory_budget: int = 0, profiling: bool = False,
                 exact_path: bool = False, class_part: tuple[int, int] | None = None, plan=None,
                 first: bool = False, wait_limit_us: int | None = None, wait_check: bool = False):
        """``plan``: None (built-in formulas), a dict with any of ``class_bits``,
        ``digit_bits``, ``inner_bits`` (streaming pass), ``direct`` (-1, 0, 1)
        and ``table_bits`` (direct pass; see MSP_OPT_* in msp.h), or
        ``"auto"`` for the autotuner's cached choice for this device and
        (m, n), if any.  ``first``: stop once a solution is found (direct
        pass; MSP_OPT_FIRST).  ``memory_budget``: bytes of device memory
        the solve may use; 0 takes $MSP_MEMORY_BUDGET (e.g. "150G"), else
        the library's default.  ``wait_limit_us`` / ``wait_check``: the
        streaming join's bounded-wait limit and its check mode
        (MSP_OPT_WAIT_LIMIT_US, MSP_OPT_WAIT_CHECK)."""
        lib = load_library()
        memory_budget = memory_budget or default_budget()
        A = np.asarray(A)
        if A.ndim != 2:
            raise MspError(-1, "A must be a 2-D matrix")
        self.m, self.n = int(A.shape[0]), int(A.shape[1])
        a, ap = _i32(A)
        dd, dp = _i32(np.asarray(d).reshape(-1))
        if dd.shape[0] != self.m:
            raise MspError(-1, "d must have one entry per row of A")
        h = ctypes.c_void_p()
        _check(lib.msp_create(ap, dp, self.m, self.n, ctypes.byref(h)))
        self._h = h
        self._lib = lib
        if stream is not None:
            _check(lib.msp_set_stream(h, ctypes.c_void_p(stream)))
        if memory_budget:
            _check(lib.msp_set_memory_budget(h, ctypes.c_size_t(memory_budget)))
        if profiling:
            _check(lib.msp_set_profiling(h, 1))
        if exact_path:
            _check(lib.msp_set_option(h, 1, 1))
        if first:
            _check(lib.msp_set_option(h, OPT_FIRST, 1))
        if wait_limit_us is not None:
            _check(lib.msp_set_option(h, OPT_WAIT_LIMIT_US, int(wait_limit_us)))
        if wait_check:
            _check(lib.msp_set_option(h, OPT_WAIT_CHECK, 1))
        if class_part is not None:
            _check(lib.msp_set_option(h, OPT_CLASS_PARTS, int(class_part[1])))
            _check(lib.msp_set_option(h, OPT_CLASS_PART, int(class_part[0])))
        if isinstance(plan, str):
            if plan != "auto":
                raise MspError(-1, "plan must be None, a dict or 'auto'")
            from . import autotune
            plan = autotune.cached_plan(self.m, self.n)
        self.plan = dict(plan) if plan else {}
        for k, v in self.plan.items():
            if k not in PLAN_KEYS:
                raise MspError(-1, f"unknown plan key {k!r}")
            _check(lib.msp_set_option(h, PLAN_KEYS[k], int(v)))

    def solve_all(self):
        ptr = ctypes.POINTER(ctypes.c_uint64)()
        cnt = ctypes.c_size_t()
        words = ctypes.c_int()
        _check(self._lib.msp_solve_all(self._h, ctypes.byref(ptr), ctypes.byref(cnt), ctypes.byref(words)))
        return _take_masks(self._lib, ptr, cnt.value, words.value)

    def stats(self) -> dict:
        s = Stats()
        _check(self._lib.msp_get_stats(self._h, ctypes.byref(s)))
        return s.as_dict()

    def close(self):
        if getattr(self, "_h", None):
            self._lib.msp_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_all(A, d, **kw):
    """Every x in {0,1}^n with A x = d, as sorted mask tuples."""
    with Instance(A, d, **kw) as inst:
        return inst.solve_all()


def solve_batch(instances, path: int = -1):
    """Solve a list of (A, d) pairs of one (m, n) with ``msp_solve_batch_path``
    (path -1: direct pass when it fits, 1: direct pass, 0: streaming pass)."""
    lib = load_library()
    if not instances:
        return []
    m, n = np.asarray(instances[0][0]).shape
    keep = []
    Ap = (ctypes.POINTER(ctypes.c_int32) * len(instances))()
    dp = (ctypes.POINTER(ctypes.c_int32) * len(instances))()
    for k, (A, d) in enumerate(instances):
        if np.asarray(A).shape != (m, n):
            raise MspError(-1, "all batch instances must share (m, n)")
        a, ap = _i32(A)
        dd, dpp = _i32(np.asarray(d).reshape(-1))
        keep += [a, dd]
        Ap[k] = ap
        dp[k] = dpp
    ptr = ctypes.POINTER(ctypes.c_uint64)()
    offs = (ctypes.c_size_t * (len(instances) + 1))()
    _check(lib.msp_solve_batch_path(Ap, dp, m, n, len(instances), int(path), ctypes.byref(ptr), offs))
    words = (n + 63) // 64
    total = offs[len(instances)]
    flat = _take_masks(lib, ptr, total, words)
    return [flat[offs[k]:offs[k + 1]] for k in range(len(instances))]


class Server:
    """``msp_server_create`` / ``msp_submit`` / ``msp_poll`` / ``msp_cancel``."""

    def __init__(self, hbm_budget: int = 0, max_inflight: int = 4):
        self._lib = load_library()
        hbm_budget = hbm_budget or default_budget()
        h = ctypes.c_void_p()
        _check(self._lib.msp_server_create(ctypes.c_size_t(hbm_budget), max_inflight, ctypes.byref(h)))
        self._h = h

    def submit(self, A, d) -> int:
        A = np.asarray(A)
        m, n = A.shape
        a, ap = _i32(A)
        dd, dp = _i32(np.asarray(d).reshape(-1))
        rid = ctypes.c_uint64()
        _check(self._lib.msp_submit(self._h, ap, dp, m, n, ctypes.byref(rid)))
        return int(rid.value)

    def poll(self, req_id: int):
        """None while pending, else the sorted solution list (raises on error)."""
        ptr = ctypes.POINTER(ctypes.c_uint64)()
        cnt = ctypes.c_size_t()
        words = ctypes.c_int()
        rc = _check(self._lib.msp_poll(self._h, ctypes.c_uint64(req_id), ctypes.byref(ptr), ctypes.byref(cnt),
                                       ctypes.byref(words)))
        if rc == 1:
            return None
        return _take_masks(self._lib, ptr, cnt.value, words.value)

    def cancel(self, req_id: int):
        _check(self._lib.msp_cancel(self._h, ctypes.c_uint64(req_id)))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.msp_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_small_noalloc(A, d, cap: int = 1 << 16, stream: int | None = None):
    """``msp_solve_small_noalloc``: the solve of a small instance (n <= 40)
    without device allocation; same result as :func:`solve_all`."""
    lib = load_library()
    A = np.asarray(A)
    m, n = A.shape
    a, ap = _i32(A)
    dd, dp = _i32(np.asarray(d).reshape(-1))
    out = np.zeros(max(1, cap), dtype=np.uint64)
    cnt = ctypes.c_size_t()
    _check(lib.msp_solve_small_noalloc(ap, dp, m, n, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), cap,
                                       ctypes.byref(cnt), ctypes.c_void_p(stream) if stream else None))
    return [(int(v),) for v in out[:cnt.value]]

"""ctypes binding of the C ABI in include/acs.h (argument marshalling only).

Every function keeps the C name.  The library is loaded from this package
directory; if it is missing, the first call raises -- there is no CPU
fallback.  All arrays passed in or returned are host numpy arrays; the
library copies them to and from the device.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libacs.so")

SOLVED, MAX_ITER, POLISH_KEPT = 0, 1, 2
ERR_ARG, ERR_CSR, ERR_CONES, ERR_OOM, ERR_FACTOR = -1, -2, -3, -4, -5
ERR_DEVICE_TIMEOUT, ERR_NUMERICAL, ERR_CUDA, ERR_LIMIT = -6, -7, -8, -9
PREC_MIXED, PREC_FP32, PREC_FP64 = 0, 1, 2
PROJ_AUTO, PROJ_CG, PROJ_DENSE = 0, 1, 2
SPLIT_DR, SPLIT_ADMM = 0, 1
STORE_FP32, STORE_BF16 = 0, 1

_lib = None


class acs_settings(C.Structure):
    _fields_ = [
        ("mu", C.c_double),
        ("t", C.c_double),
        ("cond_first", C.c_int32),
        ("cond_period", C.c_int32),
        ("cond_list", C.POINTER(C.c_int32)),
        ("n_cond_list", C.c_int32),
        ("check_every", C.c_int32),
        ("precision", C.c_int32),
        ("cg_eta", C.c_double),
        ("cg_tol", C.c_double),
        ("cg_max_iter", C.c_int32),
        ("cg_refine", C.c_int32),
        ("cuda_stream", C.c_void_p),
        ("device", C.c_int32),
        ("projection", C.c_int32),
        ("dense_max_m", C.c_int32),
        ("dense_switch_max_m", C.c_int32),
        ("dense_switch_cg", C.c_int32),
        ("extrapolation", C.c_double),
        ("a_storage", C.c_int32),
        ("col_block", C.c_int32),
        ("outer32_tol", C.c_double),
        ("splitting", C.c_int32),
        ("polish_tol", C.c_double),
    ]


class acs_instance(C.Structure):
    _fields_ = [
        ("m", C.c_int32), ("n", C.c_int32),
        ("row_ptr", C.POINTER(C.c_int64)), ("col", C.POINTER(C.c_int32)),
        ("val", C.POINTER(C.c_double)), ("b", C.POINTER(C.c_double)),
        ("c", C.POINTER(C.c_double)), ("n_orthant", C.c_int32), ("n_soc", C.c_int32),
        ("soc_dims", C.POINTER(C.c_int32)), ("share_A_with", C.c_int32),
    ]


class acs_batch_mapping(C.Structure):
    _fields_ = [("threads_per_cta", C.c_int32), ("team_ctas", C.c_int32)]


class acs_server_config(C.Structure):
    _fields_ = [("budget_bytes", C.c_int64), ("max_active", C.c_int32), ("round_ms", C.c_double),
                ("large_nnz", C.c_int64), ("threads_per_cta", C.c_int32), ("team_ctas", C.c_int32),
                ("long_nnz", C.c_int64), ("adaptive_teams", C.c_int32)]


class AcsError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {acs_status_string(code)} ({code})")
        self.code = code


def lib():
    """The loaded libacs.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run paper_2103_00736_gb300.build.build())")
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int32)
        L.acs_settings_default.argtypes = [C.POINTER(acs_settings)]
        L.acs_problem_create.argtypes = [C.c_int32, C.c_int32, C.POINTER(C.c_int64), ip, dp, dp, dp,
                                         C.c_int32, C.c_int32, ip, C.POINTER(acs_settings),
                                         C.POINTER(P)]
        L.acs_solve.argtypes = [P, C.c_double, C.c_int32]
        L.acs_solve_async.argtypes = [P, C.c_double, C.c_int32]
        L.acs_get.argtypes = [P, dp, dp, dp, ip, dp]
        L.acs_get_state.argtypes = [P, dp, dp, dp, ip, dp]
        L.acs_set_state.argtypes = [P, dp, dp, dp, C.c_int32, dp]
        L.acs_polish.argtypes = [P, C.c_int32, dp]
        L.acs_last_polish_ms.argtypes = [P, dp]
        L.acs_debug_images.argtypes = [P, C.c_int32, ip, ip, ip, ip, dp, C.POINTER(C.c_float)]
        L.acs_device_cache_trim.argtypes = [C.c_int32]
        L.acs_device_cache_stats.argtypes = [C.c_int32, C.POINTER(C.c_int64)]
        L.acs_problem_destroy.argtypes = [P]
        L.acs_problem_destroy.restype = None
        L.acs_status_string.argtypes = [C.c_int]
        L.acs_status_string.restype = C.c_char_p
        L.acs_version.restype = C.c_char_p
        L.acs_debug_counters.argtypes = [P, C.POINTER(C.c_longlong)]
        L.acs_problem_info.argtypes = [P, ip]
        L.acs_last_launch_ms.argtypes = [P, dp]
        L.acs_debug_barrier_ns.argtypes = [P, C.c_int32, dp]
        L.acs_debug_barrier_timeout.argtypes = [P, dp]
        L.acs_kkt_residuals_noalloc.argtypes = [C.c_int32, C.c_int32, P, P, P, P, P, P, P, P,
                                                C.c_int32, C.c_int32, P, P, P]
        L.acs_debug_phase_times.argtypes = [P, dp, C.POINTER(C.c_longlong), C.c_int32]
        llp = C.POINTER(C.c_longlong)
        L.acs_batch_create.argtypes = [C.c_int32, C.POINTER(acs_instance), C.POINTER(acs_settings),
                                       C.POINTER(acs_batch_mapping), C.POINTER(P), ip]
        L.acs_batch_solve.argtypes = [P, C.c_double, C.c_int32]
        L.acs_batch_solve_async.argtypes = [P, C.c_double, C.c_int32]
        L.acs_batch_get.argtypes = [P, C.c_int32, dp, dp, dp, ip, dp]
        L.acs_batch_results.argtypes = [P, ip, ip, dp]
        L.acs_batch_autotune.argtypes = [P, C.c_int32, C.POINTER(acs_batch_mapping), dp]
        L.acs_batch_set_mapping.argtypes = [P, C.POINTER(acs_batch_mapping)]
        L.acs_batch_last_ms.argtypes = [P, dp]
        L.acs_batch_info.argtypes = [P, llp, llp]
        L.acs_batch_counters.argtypes = [P, llp]
        L.acs_batch_member_ms.argtypes = [P, dp]
        L.acs_batch_phase_ms.argtypes = [P, C.c_int32, dp, C.POINTER(C.c_longlong), C.c_int32]
        L.acs_batch_destroy.argtypes = [P]
        L.acs_server_config_default.argtypes = [C.POINTER(acs_server_config)]
        L.acs_server_create.argtypes = [C.POINTER(acs_settings), C.POINTER(acs_server_config), C.POINTER(P)]
        L.acs_server_submit.argtypes = [P, C.POINTER(acs_instance), C.c_double, C.c_int32,
                                        C.POINTER(acs_settings), C.POINTER(C.c_int64)]
        L.acs_server_poll.argtypes = [P, C.c_int64, ip]
        L.acs_server_wait.argtypes = [P, C.c_int64, C.c_double]
        L.acs_server_result.argtypes = [P, C.c_int64, dp, dp, dp, ip, dp, dp]
        L.acs_server_stats.argtypes = [P, dp]
        L.acs_server_destroy.argtypes = [P]
        L.acs_debug_assign_teams.argtypes = [C.c_int32, dp, C.c_int32, ip]
        L.acs_debug_batch_image.argtypes = [C.c_int32, C.POINTER(acs_instance), C.POINTER(acs_settings),
                                             C.POINTER(C.c_uint64), C.POINTER(C.c_int64), C.POINTER(C.c_int32)]
        L.acs_debug_to_bf16.argtypes = [C.c_int64, dp, C.POINTER(C.c_uint16)]
        L.acs_debug_sell.argtypes = [C.c_int32, C.c_int32, C.POINTER(C.c_int64), ip, dp, C.c_int32, C.c_int64,
                                     ip, ip, ip, ip, ip, dp]
        L.acs_debug_arena.argtypes = [C.c_int64, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                      C.POINTER(C.c_int64)]
        u16p = C.POINTER(C.c_uint16)
        L.acs_debug_cbsell.argtypes = [C.c_int32, C.c_int32, C.POINTER(C.c_int64), ip, dp, C.c_int32, C.c_int32,
                                       C.c_int32, C.POINTER(C.c_int64), ip, ip, u16p, u16p,
                                       C.POINTER(C.c_float), ip, C.POINTER(C.c_uint32), u16p]
        L.acs_debug_pass_counts.argtypes = [P, C.POINTER(C.c_int64), C.c_int32]
        L.acs_debug_layout.argtypes = [P, C.POINTER(C.c_int64), C.c_int32]
        L.acs_bench_passes.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, dp]
        L.acs_bench_gather.argtypes = [C.c_int32, C.c_int64, C.c_int32, C.c_int32, dp]
        L.acs_server_destroy.restype = None
        L.acs_batch_destroy.restype = None
        _lib = L
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype)) if a is not None else None


def acs_status_string(code: int) -> str:
    return lib().acs_status_string(int(code)).decode()


def acs_version() -> str:
    return lib().acs_version().decode()


def acs_settings_default(**overrides) -> acs_settings:
    s = acs_settings()
    rc = lib().acs_settings_default(C.byref(s))
    if rc != 0:
        raise AcsError(rc, "acs_settings_default")
    cond_list = overrides.pop("cond_list", None)
    for k, v in overrides.items():
        if not hasattr(s, k):
            raise KeyError(k)
        setattr(s, k, v)
    if cond_list is not None:
        arr = np.ascontiguousarray(cond_list, dtype=np.int32)
        s._cond_list_keep = arr      # keep alive until problem creation copies it
        s.cond_list = _ptr(arr, C.c_int32)
        s.n_cond_list = arr.size
    return s


def _check_lengths(m, n, row_ptr, col, val, b, c, where):
    """The C entry points read m + 1 row pointers, row_ptr[m] entries and m, n
    vector entries from these arrays: refuse shorter arrays here instead of
    letting them read past the end (the C side validates the contents)."""
    ok = row_ptr.size == int(m) + 1 and b.size == int(m) and c.size == int(n)
    if ok and col is not None:
        nnz = int(row_ptr[-1])
        ok = 0 <= nnz <= min(col.size, val.size)
    if not ok:
        raise AcsError(ERR_ARG, f"{where}: array lengths do not match m, n and row_ptr[m]")


def acs_problem_create(m, n, row_ptr, col, val, b, c, n_orthant, soc_dims=(), settings=None):
    """Returns an opaque handle (int); raises AcsError on failure."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    dims = np.ascontiguousarray(soc_dims, dtype=np.int32)
    _check_lengths(m, n, row_ptr, col, val, b, c, "acs_problem_create")
    h = C.c_void_p()
    rc = lib().acs_problem_create(int(m), int(n), _ptr(row_ptr, C.c_int64), _ptr(col, C.c_int32),
                                  _ptr(val, C.c_double), _ptr(b, C.c_double), _ptr(c, C.c_double),
                                  int(n_orthant), int(dims.size), _ptr(dims, C.c_int32),
                                  C.byref(settings) if settings is not None else None, C.byref(h))
    if rc != 0:
        raise AcsError(rc, "acs_problem_create")
    return h.value


def acs_solve(h, tol: float, max_iter: int) -> int:
    return lib().acs_solve(C.c_void_p(h), float(tol), int(max_iter))


def acs_solve_async(h, tol: float, max_iter: int) -> int:
    rc = lib().acs_solve_async(C.c_void_p(h), float(tol), int(max_iter))
    if rc < 0:
        raise AcsError(rc, "acs_solve_async")
    return rc


def _check_shape(h, m, n, where):
    """The C side writes the problem's own m and n entries: refuse other sizes."""
    info = acs_problem_info(h)
    if (int(m), int(n)) != (info["m"], info["n"]):
        raise AcsError(ERR_ARG, f"{where}: m, n = {m}, {n} but the problem is {info['m']} x {info['n']}")


def acs_get(h, m: int, n: int):
    """(status, x, y, s, iters, residuals[8])."""
    _check_shape(h, m, n, "acs_get")
    x = np.empty(n)
    y = np.empty(m)
    s = np.empty(n)
    it = C.c_int32()
    res = np.empty(8)
    rc = lib().acs_get(C.c_void_p(h), _ptr(x, C.c_double), _ptr(y, C.c_double), _ptr(s, C.c_double),
                       C.byref(it), _ptr(res, C.c_double))
    return rc, x, y, s, it.value, res


def acs_get_residuals(h):
    """(status, iters, residuals[8]) without copying the vectors."""
    it = C.c_int32()
    res = np.empty(8)
    rc = lib().acs_get(C.c_void_p(h), None, None, None, C.byref(it), _ptr(res, C.c_double))
    return rc, it.value, res


def acs_get_state(h, m: int, n: int):
    _check_shape(h, m, n, "acs_get_state")
    s = np.empty(n)
    O = np.empty(n)
    w = np.empty(m)
    l = C.c_int32()
    step = np.empty(3)
    rc = lib().acs_get_state(C.c_void_p(h), _ptr(s, C.c_double), _ptr(O, C.c_double),
                             _ptr(w, C.c_double), C.byref(l), _ptr(step, C.c_double))
    if rc != 0:
        raise AcsError(rc, "acs_get_state")
    return s, O, w, l.value, step


def acs_polish(h, rounds: int = 3):
    """LP crossover polish of the last solve's iterate: (status, info[6]) with
    status SOLVED (replaced) or POLISH_KEPT, info = {|B|, CG iterations (or
    exact corrections) of the x and y solves, largest residual before, after,
    1 if replaced, 1 if M = A_B A_B' was factored}."""
    info = np.zeros(7)
    rc = lib().acs_polish(C.c_void_p(h), int(rounds), _ptr(info, C.c_double))
    if rc < 0:
        raise AcsError(rc, "acs_polish")
    return rc, info


def acs_set_state(h, s, O, w, l: int, step=None):
    s = np.ascontiguousarray(s, dtype=np.float64)
    O = np.ascontiguousarray(O, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    st = None if step is None else np.ascontiguousarray(step, dtype=np.float64)
    _check_shape(h, w.size, s.size, "acs_set_state")
    if O.size != s.size or (st is not None and st.size < 3):
        raise AcsError(ERR_ARG, "acs_set_state: array lengths do not match the problem's m and n")
    rc = lib().acs_set_state(C.c_void_p(h), _ptr(s, C.c_double), _ptr(O, C.c_double),
                             _ptr(w, C.c_double), int(l), _ptr(st, C.c_double))
    if rc != 0:
        raise AcsError(rc, "acs_set_state")


def acs_problem_destroy(h) -> None:
    if h:
        lib().acs_problem_destroy(C.c_void_p(h))


def acs_debug_counters(h) -> np.ndarray:
    out = np.zeros(6, dtype=np.int64)
    rc = lib().acs_debug_counters(C.c_void_p(h), out.ctypes.data_as(C.POINTER(C.c_longlong)))
    if rc != 0:
        raise AcsError(rc, "acs_debug_counters")
    return out


PHASES = ("rescale_o", "rescale_apply", "b_tilde", "q_refresh", "abs_K", "cg_rhs", "cg_At",
          "cg_A", "cg_vec", "update", "kkt", "dense_factor", "dense_solve", "cg_tcomb", "rhs_comb",
          "update_comb", "dense_assemble", "dense_inverse")


def acs_debug_phase_times(h) -> dict:
    ms = np.zeros(len(PHASES))
    cnt = np.zeros(len(PHASES), dtype=np.int64)
    rc = lib().acs_debug_phase_times(C.c_void_p(h), _ptr(ms, C.c_double),
                                     cnt.ctypes.data_as(C.POINTER(C.c_longlong)), len(PHASES))
    if rc < 0:
        raise AcsError(rc, "acs_debug_phase_times")
    return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(PHASES)}


def acs_debug_barrier_ns(h, n: int = 1000) -> float:
    ns = C.c_double()
    rc = lib().acs_debug_barrier_ns(C.c_void_p(h), int(n), C.byref(ns))
    if rc != 0:
        raise AcsError(rc, "acs_debug_barrier_ns")
    return ns.value


def acs_debug_barrier_timeout(h):
    """(status recorded by the device, ms waited) of a barrier one CTA never reaches."""
    ms = C.c_double()
    rc = lib().acs_debug_barrier_timeout(C.c_void_p(h), C.byref(ms))
    return rc, ms.value


def acs_last_launch_ms(h) -> float:
    ms = C.c_double()
    rc = lib().acs_last_launch_ms(C.c_void_p(h), C.byref(ms))
    if rc != 0:
        raise AcsError(rc, "acs_last_launch_ms")
    return ms.value


def acs_last_polish_ms(h) -> float:
    ms = C.c_double()
    rc = lib().acs_last_polish_ms(C.c_void_p(h), C.byref(ms))
    if rc != 0:
        raise AcsError(rc, "acs_last_polish_ms")
    return ms.value


def acs_problem_info(h) -> dict:
    out = np.zeros(8, dtype=np.int32)
    rc = lib().acs_problem_info(C.c_void_p(h), _ptr(out, C.c_int32))
    if rc != 0:
        raise AcsError(rc, "acs_problem_info")
    keys = ("m", "n", "nnz", "padded_A", "padded_AT", "grid32", "grid64", "threads")
    return dict(zip(keys, out.tolist()))


def acs_kkt_residuals_noalloc(m, n, row_ptr, col, val, b, c, x, y, z, n_orthant, n_soc,
                              soc_offsets, residuals, stream=0) -> int:
    """All array arguments are DEVICE addresses (ints, e.g. torch tensor data_ptr())."""
    return lib().acs_kkt_residuals_noalloc(int(m), int(n), row_ptr, col, val, b, c, x, y, z,
                                           int(n_orthant), int(n_soc), soc_offsets, residuals, stream)


class Solver:
    """Convenience owner of one problem handle."""

    def __init__(self, inst=None, *, m=None, n=None, row_ptr=None, col=None, val=None, b=None,
                 c=None, n_orth=None, soc_dims=(), settings=None, **overrides):
        if inst is not None:
            m, n, row_ptr, col, val, b, c = inst.m, inst.n, inst.row_ptr, inst.col, inst.val, inst.b, inst.c
            n_orth, soc_dims = inst.n_orth, inst.soc_dims
        if settings is None:
            settings = acs_settings_default(**overrides)
        self.m, self.n = int(m), int(n)
        self.h = acs_problem_create(m, n, row_ptr, col, val, b, c, n_orth, soc_dims, settings)

    def solve(self, tol=1e-6, max_iter=10000) -> int:
        return acs_solve(self.h, tol, max_iter)

    def solve_async(self, tol=1e-6, max_iter=10000) -> int:
        return acs_solve_async(self.h, tol, max_iter)

    def get(self):
        return acs_get(self.h, self.m, self.n)

    def polish(self, rounds: int = 3):
        return acs_polish(self.h, rounds)

    def residuals(self):
        return acs_get_residuals(self.h)

    def close(self):
        acs_problem_destroy(self.h)
        self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            if self.h:
                self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# batched solves
# ---------------------------------------------------------------------------

def acs_batch_create(instances, settings=None, mapping=None, share=None):
    """instances: objects with m, n, row_ptr, col, val, b, c, n_orth, soc_dims.
    share[i] = index of an earlier member whose A member i reuses, or -1.
    Returns an opaque handle; raises AcsError (with .member) on failure."""
    count = len(instances)
    arr = (acs_instance * count)()
    keep = []
    for i, inst in enumerate(instances):
        j = -1 if share is None else int(share[i])
        a = arr[i]
        a.m, a.n = int(inst.m), int(inst.n)
        b = np.ascontiguousarray(inst.b, dtype=np.float64)
        c = np.ascontiguousarray(inst.c, dtype=np.float64)
        d = np.ascontiguousarray(inst.soc_dims, dtype=np.int32)
        rp = np.ascontiguousarray(inst.row_ptr, dtype=np.int64) if j < 0 else np.zeros(int(inst.m) + 1, np.int64)
        try:
            if j < 0:
                cl = np.ascontiguousarray(inst.col, dtype=np.int32)
                vl = np.ascontiguousarray(inst.val, dtype=np.float64)
                _check_lengths(inst.m, inst.n, rp, cl, vl, b, c, f"acs_batch_create (member {i})")
                keep += [rp, cl, vl]
                a.row_ptr, a.col, a.val = _ptr(rp, C.c_int64), _ptr(cl, C.c_int32), _ptr(vl, C.c_double)
            else:
                _check_lengths(inst.m, inst.n, rp, None, None, b, c, f"acs_batch_create (member {i})")
        except AcsError as err:
            err.member = i
            raise
        keep += [b, c, d]
        a.b, a.c = _ptr(b, C.c_double), _ptr(c, C.c_double)
        a.n_orthant, a.n_soc = int(inst.n_orth), int(d.size)
        a.soc_dims = _ptr(d, C.c_int32)
        a.share_A_with = j
    h = C.c_void_p()
    bad = C.c_int32(-1)
    mp = None
    if mapping is not None:
        mp = acs_batch_mapping(int(mapping[0]), int(mapping[1]))
    rc = lib().acs_batch_create(count, arr, C.byref(settings) if settings is not None else None,
                                C.byref(mp) if mp is not None else None, C.byref(h), C.byref(bad))
    if rc != 0:
        err = AcsError(rc, f"acs_batch_create (member {bad.value})")
        err.member = bad.value
        raise err
    return h.value


def acs_batch_solve(h, tol: float, max_iter: int) -> int:
    return lib().acs_batch_solve(C.c_void_p(h), float(tol), int(max_iter))


def acs_batch_solve_async(h, tol: float, max_iter: int) -> int:
    rc = lib().acs_batch_solve_async(C.c_void_p(h), float(tol), int(max_iter))
    if rc < 0:
        raise AcsError(rc, "acs_batch_solve_async")
    return rc


def acs_batch_get(h, i: int, m: int, n: int):
    """(status, x, y, s, iters, residuals[8]) of member i."""
    x, y, s, res = np.empty(n), np.empty(m), np.empty(n), np.empty(8)
    it = C.c_int32()
    rc = lib().acs_batch_get(C.c_void_p(h), int(i), _ptr(x, C.c_double), _ptr(y, C.c_double),
                             _ptr(s, C.c_double), C.byref(it), _ptr(res, C.c_double))
    return rc, x, y, s, it.value, res


def acs_batch_results(h, count: int):
    """(worst status, status[count], iters[count], residuals[count, 8])."""
    st = np.empty(count, np.int32)
    it = np.empty(count, np.int32)
    res = np.empty((count, 8))
    rc = lib().acs_batch_results(C.c_void_p(h), _ptr(st, C.c_int32), _ptr(it, C.c_int32),
                                 _ptr(res, C.c_double))
    return rc, st, it, res


def acs_batch_autotune(h, max_iter: int = 30):
    """(chosen (threads, team), ms[3, 3]: rows threads 256/512/1024, cols team 1/2/4)."""
    m = acs_batch_mapping()
    ms = np.empty(9)
    rc = lib().acs_batch_autotune(C.c_void_p(h), int(max_iter), C.byref(m), _ptr(ms, C.c_double))
    if rc != 0:
        raise AcsError(rc, "acs_batch_autotune")
    return (m.threads_per_cta, m.team_ctas), ms.reshape(3, 3)


def acs_batch_set_mapping(h, threads: int, team: int) -> None:
    m = acs_batch_mapping(int(threads), int(team))
    rc = lib().acs_batch_set_mapping(C.c_void_p(h), C.byref(m))
    if rc != 0:
        raise AcsError(rc, "acs_batch_set_mapping")


def acs_batch_last_ms(h) -> float:
    ms = C.c_double()
    rc = lib().acs_batch_last_ms(C.c_void_p(h), C.byref(ms))
    if rc != 0:
        raise AcsError(rc, "acs_batch_last_ms")
    return ms.value


def acs_batch_info(h) -> dict:
    out = np.zeros(8, dtype=np.int64)
    cnt = np.zeros(6, dtype=np.int64)
    llp = C.POINTER(C.c_longlong)
    rc = lib().acs_batch_info(C.c_void_p(h), out.ctypes.data_as(llp), cnt.ctypes.data_as(llp))
    if rc != 0:
        raise AcsError(rc, "acs_batch_info")
    keys = ("members", "matrices", "sum_m", "sum_n", "stored_nnz", "teams", "ctas", "graph")
    d = dict(zip(keys, out.tolist()))
    d["counters"] = cnt
    return d


def acs_batch_counters(h, count: int) -> np.ndarray:
    """int64 [count, 8]: see include/acs.h."""
    out = np.zeros((count, 8), dtype=np.int64)
    rc = lib().acs_batch_counters(C.c_void_p(h), out.ctypes.data_as(C.POINTER(C.c_longlong)))
    if rc != 0:
        raise AcsError(rc, "acs_batch_counters")
    return out


def acs_batch_member_ms(h, count: int) -> np.ndarray:
    ms = np.zeros(count)
    rc = lib().acs_batch_member_ms(C.c_void_p(h), _ptr(ms, C.c_double))
    if rc != 0:
        raise AcsError(rc, "acs_batch_member_ms")
    return ms


def acs_batch_phase_ms(h, i: int = -1) -> dict:
    """{phase: (ms, count)} of member i's last solve, or summed over members (i = -1)."""
    ms = np.zeros(len(PHASES))
    cnt = np.zeros(len(PHASES), dtype=np.int64)
    rc = lib().acs_batch_phase_ms(C.c_void_p(h), int(i), _ptr(ms, C.c_double),
                                  cnt.ctypes.data_as(C.POINTER(C.c_longlong)), len(PHASES))
    if rc < 0:
        raise AcsError(rc, "acs_batch_phase_ms")
    return {k: (float(ms[j]), int(cnt[j])) for j, k in enumerate(PHASES)}


def acs_batch_destroy(h) -> None:
    if h:
        lib().acs_batch_destroy(C.c_void_p(h))


def shared_A_index(instances):
    """share[i] for acs_batch_create: the first earlier member whose A has the
    same shape, pattern and values (compared exactly), else -1."""
    share = [-1] * len(instances)
    seen = {}
    for i, inst in enumerate(instances):
        key = (inst.m, inst.n, inst.row_ptr[-1])
        for j in seen.get(key, ()):
            o = instances[j]
            if (np.array_equal(o.row_ptr, inst.row_ptr) and np.array_equal(o.col, inst.col)
                    and np.array_equal(o.val, inst.val)):
                share[i] = j
                break
        else:
            seen.setdefault(key, []).append(i)
    return share


class Batch:
    """Owner of one batch handle."""

    def __init__(self, instances, settings=None, mapping=None, share="auto", **overrides):
        if settings is None:
            settings = acs_settings_default(**overrides)
        if share == "auto":
            share = shared_A_index(instances)
        self.count = len(instances)
        self.shapes = [(int(i.m), int(i.n)) for i in instances]
        self.h = acs_batch_create(instances, settings, mapping, share)

    def solve(self, tol=1e-6, max_iter=10000) -> int:
        return acs_batch_solve(self.h, tol, max_iter)

    def solve_async(self, tol=1e-6, max_iter=10000) -> int:
        return acs_batch_solve_async(self.h, tol, max_iter)

    def get(self, i):
        m, n = self.shapes[i]
        return acs_batch_get(self.h, i, m, n)

    def results(self):
        return acs_batch_results(self.h, self.count)

    def close(self):
        acs_batch_destroy(self.h)
        self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            if self.h:
                self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# serving loop
# ---------------------------------------------------------------------------

def acs_server_config_default(**overrides) -> acs_server_config:
    c = acs_server_config()
    rc = lib().acs_server_config_default(C.byref(c))
    if rc != 0:
        raise AcsError(rc, "acs_server_config_default")
    for k, v in overrides.items():
        if not hasattr(c, k):
            raise KeyError(k)
        setattr(c, k, v)
    return c


def acs_server_create(settings=None, config=None):
    h = C.c_void_p()
    rc = lib().acs_server_create(C.byref(settings) if settings is not None else None,
                                 C.byref(config) if config is not None else None, C.byref(h))
    if rc != 0:
        raise AcsError(rc, "acs_server_create")
    return h.value


def acs_server_submit(h, inst, tol: float = 1e-6, max_iter: int = 10000, settings=None) -> int:
    """Queue one request (host arrays are copied during the call); returns its id.
    settings: per-request mu, t, schedule and check period (acs_settings), or None."""
    rp = np.ascontiguousarray(inst.row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(inst.col, dtype=np.int32)
    vl = np.ascontiguousarray(inst.val, dtype=np.float64)
    b = np.ascontiguousarray(inst.b, dtype=np.float64)
    c = np.ascontiguousarray(inst.c, dtype=np.float64)
    d = np.ascontiguousarray(inst.soc_dims, dtype=np.int32)
    _check_lengths(inst.m, inst.n, rp, cl, vl, b, c, "acs_server_submit")
    a = acs_instance()
    a.m, a.n = int(inst.m), int(inst.n)
    a.row_ptr, a.col, a.val = _ptr(rp, C.c_int64), _ptr(cl, C.c_int32), _ptr(vl, C.c_double)
    a.b, a.c = _ptr(b, C.c_double), _ptr(c, C.c_double)
    a.n_orthant, a.n_soc, a.soc_dims = int(inst.n_orth), int(d.size), _ptr(d, C.c_int32)
    a.share_A_with = -1
    rid = C.c_int64()
    rc = lib().acs_server_submit(C.c_void_p(h), C.byref(a), float(tol), int(max_iter),
                                 C.byref(settings) if settings is not None else None, C.byref(rid))
    if rc != 0:
        raise AcsError(rc, "acs_server_submit")
    return rid.value


def acs_server_poll(h, rid: int) -> bool:
    done = C.c_int32()
    rc = lib().acs_server_poll(C.c_void_p(h), int(rid), C.byref(done))
    if rc != 0:
        raise AcsError(rc, "acs_server_poll")
    return bool(done.value)


def acs_server_wait(h, rid: int, timeout_s: float = -1.0) -> int:
    return lib().acs_server_wait(C.c_void_p(h), int(rid), float(timeout_s))


def acs_server_result(h, rid: int, m: int, n: int):
    """(status, x, y, s, iters, residuals[8], latency_ms) of a finished request."""
    x, y, s, res = np.empty(n), np.empty(m), np.empty(n), np.empty(8)
    it = C.c_int32()
    lat = C.c_double()
    rc = lib().acs_server_result(C.c_void_p(h), int(rid), _ptr(x, C.c_double), _ptr(y, C.c_double),
                                 _ptr(s, C.c_double), C.byref(it), _ptr(res, C.c_double), C.byref(lat))
    return rc, x, y, s, it.value, res, lat.value


def acs_server_stats(h) -> dict:
    out = np.zeros(10)
    rc = lib().acs_server_stats(C.c_void_p(h), _ptr(out, C.c_double))
    if rc != 0:
        raise AcsError(rc, "acs_server_stats")
    keys = ("rounds", "admitted", "finished", "active", "pool_bytes", "pool_peak_bytes", "large",
            "waiting", "round_ms_mean", "active_mean")
    return dict(zip(keys, out.tolist()))


def acs_server_destroy(h) -> None:
    if h:
        lib().acs_server_destroy(C.c_void_p(h))


LP_SCHEDULE = dict(t=9.2, cond_first=300, cond_period=100)      # Section V-A experiments
SOCP_SCHEDULE = dict(t=1.7, cond_first=200, cond_period=100)    # Section V-C experiments


def schedule_for(inst) -> acs_settings:
    """Per-request settings with the paper's schedule for the request's cone type."""
    return acs_settings_default(**(SOCP_SCHEDULE if len(inst.soc_dims) else LP_SCHEDULE))


class Server:
    """Owner of one serving loop."""

    def __init__(self, settings=None, config=None, **cfg):
        if config is None:
            config = acs_server_config_default(**cfg)
        self.h = acs_server_create(settings, config)
        self.shapes = {}

    def submit(self, inst, tol=1e-6, max_iter=10000, settings="auto") -> int:
        """settings="auto": the paper's LP schedule (t = 9.2, L = {300, 400, ...})
        for an LP, its SOCP schedule (t = 1.7, L = {200, 300, ...}) for a
        request with Lorentz cones."""
        if isinstance(settings, str) and settings == "auto":
            settings = schedule_for(inst)
        rid = acs_server_submit(self.h, inst, tol, max_iter, settings)
        self.shapes[rid] = (int(inst.m), int(inst.n))
        return rid

    def wait(self, rid, timeout_s=-1.0) -> int:
        return acs_server_wait(self.h, rid, timeout_s)

    def result(self, rid):
        m, n = self.shapes.pop(rid)
        return acs_server_result(self.h, rid, m, n)

    def stats(self) -> dict:
        return acs_server_stats(self.h)

    def close(self):
        acs_server_destroy(self.h)
        self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            if self.h:
                self.close()
        except Exception:
            pass


def acs_debug_assign_teams(work, grid: int) -> np.ndarray:
    """int32 [3, grid]: position, rank, team size per CTA (host-only check)."""
    w = np.ascontiguousarray(work, dtype=np.float64)
    out = np.zeros(3 * grid, dtype=np.int32)
    rc = lib().acs_debug_assign_teams(int(w.size), _ptr(w, C.c_double), int(grid), _ptr(out, C.c_int32))
    if rc != 0:
        raise AcsError(rc, "acs_debug_assign_teams")
    return out.reshape(3, grid)


def acs_debug_arena(cap: int, ops):
    """(offsets, used, peak) of a first-fit pool run (host-only check)."""
    o = np.ascontiguousarray(ops, dtype=np.int64)
    off = np.zeros(max(1, o.size), dtype=np.int64)
    up = np.zeros(2, dtype=np.int64)
    rc = lib().acs_debug_arena(int(cap), int(o.size), _ptr(o, C.c_int64), _ptr(off, C.c_int64),
                               _ptr(up, C.c_int64))
    if rc != 0:
        raise AcsError(rc, "acs_debug_arena")
    return off[:o.size], int(up[0]), int(up[1])


def acs_debug_sell(m, n, row_ptr, col, val, which: int, warps: int) -> dict:
    """The relabelling and sliced-ELLPACK image of A (which=0) or A' (which=1)
    as acs_problem_create prepares them (host-only check)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col, dtype=np.int32)
    va = np.ascontiguousarray(val, dtype=np.float64)
    info = np.zeros(4, dtype=np.int32)
    args = (int(m), int(n), _ptr(rp, C.c_int64), _ptr(ci, C.c_int32), _ptr(va, C.c_double), int(which), int(warps))
    rc = lib().acs_debug_sell(*args, _ptr(info, C.c_int32), None, None, None, None, None)
    if rc != 0:
        raise AcsError(rc, "acs_debug_sell")
    rows, slices, g, stored = (int(v) for v in info)
    perm = np.zeros(m, dtype=np.int32)
    sptr = np.zeros(slices + 1, dtype=np.int32)
    slen = np.zeros(max(slices, 1), dtype=np.int32)
    oc = np.zeros(max(stored, 1), dtype=np.int32)
    ov = np.zeros(max(stored, 1), dtype=np.float64)
    rc = lib().acs_debug_sell(*args, _ptr(info, C.c_int32), _ptr(perm, C.c_int32), _ptr(sptr, C.c_int32),
                              _ptr(slen, C.c_int32), _ptr(oc, C.c_int32), _ptr(ov, C.c_double))
    if rc != 0:
        raise AcsError(rc, "acs_debug_sell")
    return dict(rows=rows, slices=slices, g=g, stored=stored, perm=perm, sptr=sptr, slen=slen[:slices],
                col=oc[:stored], val=ov[:stored])


def acs_device_cache_trim(device: int = -1) -> None:
    """Return the device-memory cache's kept blocks to the driver."""
    rc = lib().acs_device_cache_trim(int(device))
    if rc != 0:
        raise AcsError(rc, "acs_device_cache_trim")


def acs_device_cache_stats(device: int = 0) -> dict:
    out = np.zeros(3, dtype=np.int64)
    rc = lib().acs_device_cache_stats(int(device), _ptr(out, C.c_int64))
    if rc != 0:
        raise AcsError(rc, "acs_device_cache_stats")
    return {"bytes": int(out[0]), "hits": int(out[1]), "misses": int(out[2])}


def acs_debug_images(h, which: int) -> dict:
    """The sliced-ELLPACK image of A (which=0) or A' (which=1) held on the device."""
    info = np.zeros(4, dtype=np.int32)
    rc = lib().acs_debug_images(C.c_void_p(h), int(which), _ptr(info, C.c_int32), None, None, None, None, None)
    if rc != 0:
        raise AcsError(rc, "acs_debug_images")
    rows, slices, g, stored = (int(v) for v in info)
    sptr = np.zeros(slices + 1, dtype=np.int32)
    slen = np.zeros(max(slices, 1), dtype=np.int32)
    oc = np.zeros(max(stored, 1), dtype=np.int32)
    ov = np.zeros(max(stored, 1), dtype=np.float64)
    o32 = np.full(max(stored, 1), np.nan, dtype=np.float32)
    rc = lib().acs_debug_images(C.c_void_p(h), int(which), _ptr(info, C.c_int32), _ptr(sptr, C.c_int32),
                                _ptr(slen, C.c_int32), _ptr(oc, C.c_int32), _ptr(ov, C.c_double),
                                _ptr(o32, C.c_float))
    if rc != 0:
        raise AcsError(rc, "acs_debug_images")
    return dict(rows=rows, slices=slices, g=g, stored=stored, sptr=sptr, slen=slen[:slices], col=oc[:stored],
                val=ov[:stored], v32=o32[:stored])


def acs_debug_cbsell(m, n, row_ptr, col, val, which: int, width_limit: int, ctas: int) -> dict:
    """The column-blocked image of the relabelled A (which=0) or of A'
    (which=1) that acs_problem_create builds for the FP32 passes (host-only
    check)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col, dtype=np.int32)
    va = np.ascontiguousarray(val, dtype=np.float64)
    info = np.zeros(6, dtype=np.int64)
    args = (int(m), int(n), _ptr(rp, C.c_int64), _ptr(ci, C.c_int32), _ptr(va, C.c_double), int(which),
            int(width_limit), int(ctas))
    rc = lib().acs_debug_cbsell(*args, _ptr(info, C.c_int64), None, None, None, None, None, None, None, None)
    if rc != 0:
        raise AcsError(rc, "acs_debug_cbsell")
    rows, cols, width, nblocks, nsl, stored = (int(v) for v in info)
    items = nblocks * nsl
    perm = np.zeros(m, dtype=np.int32)
    sptr = np.zeros(items + 1, dtype=np.int32)
    rowid = np.zeros(items * 32, dtype=np.uint16)
    oc = np.zeros(max(stored, 1), dtype=np.uint16)
    ov = np.zeros(max(stored, 1), dtype=np.float32)
    cta = np.zeros(ctas + 1, dtype=np.int32)
    cend = np.zeros(stored // 1024 + 2, dtype=np.uint32)
    ipos = np.zeros(items * 32, dtype=np.uint16)
    rc = lib().acs_debug_cbsell(*args, _ptr(info, C.c_int64), _ptr(perm, C.c_int32), _ptr(sptr, C.c_int32),
                                _ptr(rowid, C.c_uint16), _ptr(oc, C.c_uint16), _ptr(ov, C.c_float),
                                _ptr(cta, C.c_int32), _ptr(cend, C.c_uint32), _ptr(ipos, C.c_uint16))
    if rc != 0:
        raise AcsError(rc, "acs_debug_cbsell")
    return dict(rows=rows, cols=cols, width=width, nblocks=nblocks, nsl=nsl, stored=stored, perm=perm,
                sptr=sptr, rowid=rowid, col=oc[:stored], val=ov[:stored], cta_beg=cta, cend=cend, ipos=ipos)


PASS_COUNTS = ("cg_A", "cg_At", "fp64_A", "fp64_At", "rescalings", "checks", "fp32_outer_A",
               "fp32_outer_At", "outer32_end", "iterations", "cg_iterations", "cg_switch_at",
               "polish_attempts", "polish_taken", "polish_corrections", "polish_factored",
               "polish_support", "polish_support_entries")


def acs_debug_pass_counts(h) -> dict:
    out = np.zeros(len(PASS_COUNTS), dtype=np.int64)
    rc = lib().acs_debug_pass_counts(C.c_void_p(h), _ptr(out, C.c_int64), len(PASS_COUNTS))
    if rc < 0:
        raise AcsError(rc, "acs_debug_pass_counts")
    return {k: int(out[i]) for i, k in enumerate(PASS_COUNTS)}


LAYOUT = ("col_blocked", "A_blocks", "A_width", "A_stored", "At_blocks", "At_width", "At_stored",
          "dyn_smem", "sell_A_stored", "sell_At_stored", "sell_A_slices", "sell_At_slices",
          "create_h2d_bytes", "create_d2h_bytes")


def acs_debug_layout(h) -> dict:
    out = np.zeros(16, dtype=np.int64)
    rc = lib().acs_debug_layout(C.c_void_p(h), _ptr(out, C.c_int64), 16)
    if rc < 0:
        raise AcsError(rc, "acs_debug_layout")
    return {k: int(out[i]) for i, k in enumerate(LAYOUT)}


def acs_debug_batch_image(instances, settings=None, share=None):
    """(FNV-1a hash, bytes) of the host image acs_batch_create would upload
    (host-only check); raises AcsError (with .member) like acs_batch_create."""
    count = len(instances)
    arr = (acs_instance * count)()
    keep = []
    for i, inst in enumerate(instances):
        j = -1 if share is None else int(share[i])
        a = arr[i]
        a.m, a.n = int(inst.m), int(inst.n)
        if j < 0:
            rp = np.ascontiguousarray(inst.row_ptr, dtype=np.int64)
            cl = np.ascontiguousarray(inst.col, dtype=np.int32)
            vl = np.ascontiguousarray(inst.val, dtype=np.float64)
            keep += [rp, cl, vl]
            a.row_ptr, a.col, a.val = _ptr(rp, C.c_int64), _ptr(cl, C.c_int32), _ptr(vl, C.c_double)
        b = np.ascontiguousarray(inst.b, dtype=np.float64)
        c = np.ascontiguousarray(inst.c, dtype=np.float64)
        d = np.ascontiguousarray(inst.soc_dims, dtype=np.int32)
        keep += [b, c, d]
        a.b, a.c = _ptr(b, C.c_double), _ptr(c, C.c_double)
        a.n_orthant, a.n_soc, a.soc_dims = int(inst.n_orth), int(d.size), _ptr(d, C.c_int32)
        a.share_A_with = j
    h, nbytes, bad = C.c_uint64(), C.c_int64(), C.c_int32(-1)
    rc = lib().acs_debug_batch_image(count, arr, C.byref(settings) if settings is not None else None,
                                     C.byref(h), C.byref(nbytes), C.byref(bad))
    if rc != 0:
        err = AcsError(rc, f"acs_debug_batch_image (member {bad.value})")
        err.member = bad.value
        raise err
    return h.value, nbytes.value


def acs_debug_to_bf16(v) -> np.ndarray:
    """uint16 BF16 patterns the library stores for the values v (host-only check)."""
    a = np.ascontiguousarray(v, dtype=np.float64)
    out = np.zeros(a.size, dtype=np.uint16)
    rc = lib().acs_debug_to_bf16(int(a.size), _ptr(a, C.c_double), _ptr(out, C.c_uint16))
    if rc != 0:
        raise AcsError(rc, "acs_debug_to_bf16")
    return out


BENCH_KINDS = ("cb_At", "cb_tcomb", "cb_A", "cb_vec", "l2_At", "l2_A", "l2_vec", "fp64_rhs", "fp64_At",
               "barrier", "abs_K", "kkt", "o32_rhs", "o32_rhs_comb", "o32_upd", "o32_upd_comb",
               "cb_stage32", "cb_stage64", "cb_At_nogather", "cb_At_nostage",
               "stream_At", "stream_At_val")


def acs_bench_passes(h, kind, reps: int = 50, smem_bytes: int = -1) -> float:
    """Device microseconds of one phase (+ one grid barrier) on the problem's data."""
    k = BENCH_KINDS.index(kind) if isinstance(kind, str) else int(kind)
    us = C.c_double()
    rc = lib().acs_bench_passes(C.c_void_p(h), k, int(reps), int(smem_bytes), C.byref(us))
    if rc != 0:
        raise AcsError(rc, "acs_bench_passes")
    return us.value


def acs_bench_gather(entries: int, mode: int, steps: int = 64, device: int = 0) -> float:
    """Random 4-byte gathers per second (mode 0 default, 1 .cg, 2 .nc, 3 shared memory)."""
    g = C.c_double()
    rc = lib().acs_bench_gather(int(device), int(entries), int(mode), int(steps), C.byref(g))
    if rc != 0:
        raise AcsError(rc, "acs_bench_gather")
    return g.value

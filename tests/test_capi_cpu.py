"""Host-only checks of the C ABI: the library builds, loads, exports every
symbol include/acs.h declares, and rejects malformed input before touching
the device."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def capi():
    from paper_2103_00736_gb300 import capi as c, build
    if not os.path.exists(c.LIB_PATH):
        build.build()
    c.lib()
    return c


def _declared():
    txt = open(os.path.join(ROOT, "include", "acs.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(acs_[a-z0-9_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(capi):
    names = _declared()
    assert "acs_problem_create" in names and "acs_solve" in names and "acs_get" in names
    L = capi.lib()
    for name in names:
        assert hasattr(L, name), name


def test_settings_defaults(capi):
    s = capi.acs_settings_default()
    assert s.mu == 1.0 and s.t == 9.2 and s.cond_first == 300 and s.cond_period == 100
    assert s.check_every == 10 and s.precision == capi.PREC_MIXED and s.splitting == capi.SPLIT_DR
    assert capi.acs_status_string(0) == "solved"
    assert "CSR" in capi.acs_status_string(capi.ERR_CSR)


def _create(capi, m, n, rp, col, val, b, c, n_orth, dims=(), **kw):
    return capi.acs_problem_create(m, n, rp, col, val, b, c, n_orth, dims,
                                   capi.acs_settings_default(**kw) if kw else None)


@pytest.mark.parametrize("case,code", [
    ("empty_row", -2), ("col_range", -2), ("unsorted", -2), ("duplicate", -2), ("rowptr0", -2),
    ("cones_sum", -3), ("cone_small", -3), ("nan", -1), ("mu", -1), ("m0", -1),
])
def test_validation_errors(capi, case, code):
    rp = np.array([0, 2, 4], np.int64)
    col = np.array([0, 1, 1, 2], np.int32)
    val = np.array([1.0, 2.0, 3.0, 4.0])
    b, c = np.ones(2), np.ones(3)
    args = dict(m=2, n=3, rp=rp, col=col, val=val, b=b, c=c, n_orth=3, dims=())
    kw = {}
    if case == "empty_row":
        args["rp"] = np.array([0, 0, 4], np.int64)
    elif case == "col_range":
        args["col"] = np.array([0, 1, 1, 3], np.int32)
    elif case == "unsorted":
        args["col"] = np.array([1, 0, 1, 2], np.int32)
    elif case == "duplicate":
        args["col"] = np.array([1, 1, 1, 2], np.int32)
    elif case == "rowptr0":
        args["rp"] = np.array([1, 2, 4], np.int64)
    elif case == "cones_sum":
        args["n_orth"] = 2
    elif case == "cone_small":
        args["n_orth"], args["dims"] = 2, [1]
    elif case == "nan":
        args["val"] = np.array([1.0, np.nan, 3.0, 4.0])
    elif case == "mu":
        kw["mu"] = -1.0
    elif case == "m0":
        args["m"] = 0
    with pytest.raises(capi.AcsError) as e:
        _create(capi, args["m"], args["n"], args["rp"], args["col"], args["val"], args["b"],
                args["c"], args["n_orth"], args["dims"], **kw)
    assert e.value.code == code


def test_build_flags_target_sm103a():
    from paper_2103_00736_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_batch_rejects_malformed_members_before_the_device(capi):
    from paper_2103_00736_gb300 import instances as I
    good = I.bernoulli_lp(11, 6, 15, density=0.3)
    bad = I.bernoulli_lp(12, 6, 15, density=0.3)
    bad.row_ptr = bad.row_ptr.copy()
    bad.row_ptr[2] = bad.row_ptr[1]            # empty row 1
    with pytest.raises(capi.AcsError) as e:
        capi.acs_batch_create([good, good, bad])
    assert e.value.code == capi.ERR_CSR and e.value.member == 2
    with pytest.raises(capi.AcsError) as e:      # share index must point at an earlier member
        capi.acs_batch_create([good, good], share=[1, -1])
    assert e.value.code == capi.ERR_ARG and e.value.member == 0
    cones = I.bernoulli_lp(13, 6, 15, density=0.3)
    cones.n_orth = 10                           # 10 + 0 cones != n = 15
    with pytest.raises(capi.AcsError) as e:
        capi.acs_batch_create([good, cones])
    assert e.value.code == capi.ERR_CONES and e.value.member == 1
    with pytest.raises(capi.AcsError) as e:      # mapping outside the supported set
        capi.acs_batch_create([good], mapping=(384, 1))
    assert e.value.code == capi.ERR_ARG


def test_shared_A_detection(capi):
    from paper_2103_00736_gb300 import instances as I
    mem = I.batch(count=8, m_shared=60, mmin=20, mmax=80)
    share = capi.shared_A_index(mem)
    assert share[:2] == [-1, 0] and all(s == -1 for s in share[2:])


def test_server_rejects_bad_configurations_before_the_device(capi):
    bad = [dict(budget_bytes=1000), dict(max_active=0), dict(round_ms=0.0), dict(large_nnz=-1),
           dict(long_nnz=-1), dict(threads_per_cta=384), dict(team_ctas=3)]
    for kw in bad:
        with pytest.raises(capi.AcsError) as e:
            capi.acs_server_create(None, capi.acs_server_config_default(**kw))
        assert e.value.code == capi.ERR_ARG, kw
    s = capi.acs_settings_default(mu=-1.0)
    with pytest.raises(capi.AcsError) as e:
        capi.acs_server_create(s, capi.acs_server_config_default())
    assert e.value.code == capi.ERR_ARG
    c = capi.acs_server_config_default()
    assert (c.round_ms, c.max_active, c.threads_per_cta, c.team_ctas, c.adaptive_teams) == (2.0, 2048, 256, 1, 1)


def test_settings_of_the_projection_are_validated(capi):
    from paper_2103_00736_gb300 import instances as I
    inst = I.bernoulli_lp(21, 6, 15, density=0.3)
    for kw in (dict(projection=7), dict(dense_max_m=5000), dict(a_storage=3), dict(extrapolation=-0.5),
               dict(dense_switch_cg=-1), dict(splitting=2), dict(splitting=-1),
               dict(splitting=1), dict(splitting=1, cond_first=0, cond_list=[5])):
        with pytest.raises(capi.AcsError) as e:
            capi.acs_problem_create(inst.m, inst.n, inst.row_ptr, inst.col, inst.val, inst.b, inst.c,
                                    inst.n_orth, inst.soc_dims, capi.acs_settings_default(**kw))
        assert e.value.code == capi.ERR_ARG, kw


def test_polish_rejects_a_null_handle(capi):
    with pytest.raises(capi.AcsError) as e:
        capi.acs_polish(None)
    assert e.value.code == capi.ERR_ARG
    assert capi.acs_status_string(capi.POLISH_KEPT).startswith("polish")


def test_missing_library_fails_loudly(capi, monkeypatch, tmp_path):
    """No CPU fallback: without the CUDA library every entry point raises."""
    monkeypatch.setattr(capi, "LIB_PATH", str(tmp_path / "libacs.so"))
    monkeypatch.setattr(capi, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        capi.acs_settings_default()
    with pytest.raises(RuntimeError, match="not built"):
        capi.acs_problem_create(1, 1, np.array([0, 1], np.int64), np.array([0], np.int32), [1.0], [1.0],
                                [1.0], 1, [], None)


def test_product_path_does_not_load_the_oracle():
    """The package and the benchmark's GPU arms import nothing from oracle/
    (only the CPU-baseline leg does, inside its own subprocess)."""
    import subprocess
    import sys
    code = ("import sys; import paper_2103_00736_gb300.capi, paper_2103_00736_gb300.instances, bench; "
            "bad = [m for m in sys.modules if m == 'oracle' or m.startswith('oracle.')]; "
            "assert not bad, bad")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr


def test_binding_refuses_short_arrays(capi):
    """Arrays shorter than m, n and row_ptr[m] say are refused by the binding,
    before the C side would read past their ends."""
    rp = np.array([0, 2, 4], np.int64)
    col = np.array([0, 1, 1, 2], np.int32)
    val = np.array([1.0, 2.0, 3.0, 4.0])
    for args in ((2, 3, rp, col[:3], val, np.ones(2), np.ones(3)),
                 (2, 3, rp, col, val[:3], np.ones(2), np.ones(3)),
                 (2, 3, rp[:2], col, val, np.ones(2), np.ones(3)),
                 (2, 3, rp, col, val, np.ones(1), np.ones(3)),
                 (2, 3, rp, col, val, np.ones(2), np.ones(2))):
        with pytest.raises(capi.AcsError) as e:
            capi.acs_problem_create(*args, 3, [])
        assert e.value.code == capi.ERR_ARG and "array lengths" in str(e.value)
    from paper_2103_00736_gb300 import instances as I
    good = I.bernoulli_lp(11, 6, 15, density=0.3)
    short = I.bernoulli_lp(12, 6, 15, density=0.3)
    short.c = short.c[:-1]
    with pytest.raises(capi.AcsError) as e:
        capi.acs_batch_create([good, good, short])
    assert e.value.code == capi.ERR_ARG and e.value.member == 2


def test_abi_rejects_more_than_2_31_stored_entries(capi):
    """The C ABI's own check (called without the binding): row_ptr[m] >= 2^31
    is refused from the row pointers alone, before col or val are read."""
    import ctypes as C
    L = capi.lib()
    rp = np.array([0, 1, 1 << 31], np.int64)
    col = np.zeros(1, np.int32)
    val = np.ones(1)
    b, c = np.ones(2), np.ones(2)
    h = C.c_void_p()
    rc = L.acs_problem_create(2, 2, rp.ctypes.data_as(C.POINTER(C.c_int64)), col.ctypes.data_as(C.POINTER(C.c_int32)),
                              val.ctypes.data_as(C.POINTER(C.c_double)), b.ctypes.data_as(C.POINTER(C.c_double)),
                              c.ctypes.data_as(C.POINTER(C.c_double)), 2, 0, None, None, C.byref(h))
    assert rc == capi.ERR_CSR and not h.value


def test_batch_host_image_is_deterministic_and_checked(capi):
    """The batch's host preparation runs on several threads that take members
    as they come: the image is the same on every call, changes with any
    value of the input, and malformed members are reported as by
    acs_batch_create (first failing member, its code)."""
    from paper_2103_00736_gb300 import instances as I
    mem = I.batch(count=96, m_shared=200, mmin=50, mmax=400)
    share = capi.shared_A_index(mem)
    h0 = capi.acs_debug_batch_image(mem, share=share)
    for _ in range(3):
        assert capi.acs_debug_batch_image(mem, share=share) == h0
    mem[70].val = mem[70].val.copy()
    mem[70].val[5] += 1.0
    h1 = capi.acs_debug_batch_image(mem, share=share)
    assert h1[0] != h0[0] and h1[1] == h0[1]
    good = I.bernoulli_lp(11, 6, 15, density=0.3)
    bad = I.bernoulli_lp(12, 6, 15, density=0.3)
    bad.row_ptr = bad.row_ptr.copy()
    bad.row_ptr[2] = bad.row_ptr[1]
    nan = I.bernoulli_lp(13, 6, 15, density=0.3)
    nan.val = nan.val.copy()
    nan.val[3] = np.nan
    for members, code, where in (([good] * 70 + [nan] + [bad], capi.ERR_ARG, 70),
                                 ([good] * 65 + [bad] + [good] * 10 + [nan], capi.ERR_CSR, 65)):
        for fn in (capi.acs_debug_batch_image, capi.acs_batch_create):
            with pytest.raises(capi.AcsError) as e:
                fn(members)
            assert (e.value.code, e.value.member) == (code, where), fn


def test_batch_share_chains_through_invalid_members(capi):
    """A member that shares the A of an invalid member: the invalid one is
    reported (it comes first), and its arrays are never read."""
    from paper_2103_00736_gb300 import capi as c
    import ctypes as C
    from paper_2103_00736_gb300 import instances as I
    good = I.bernoulli_lp(11, 6, 15, density=0.3)
    count = 80
    arr = (c.acs_instance * count)()
    keep = []
    for i in range(count):
        rp = np.ascontiguousarray(good.row_ptr, np.int64)
        cl = np.ascontiguousarray(good.col, np.int32)
        vl = np.ascontiguousarray(good.val, np.float64)
        b = np.ascontiguousarray(good.b, np.float64)
        cc = np.ascontiguousarray(good.c, np.float64)
        keep += [rp, cl, vl, b, cc]
        a = arr[i]
        a.m, a.n = good.m, good.n
        a.row_ptr, a.col, a.val = c._ptr(rp, C.c_int64), c._ptr(cl, C.c_int32), c._ptr(vl, C.c_double)
        a.b, a.c = c._ptr(b, C.c_double), c._ptr(cc, C.c_double)
        a.n_orthant, a.n_soc, a.soc_dims = good.n, 0, None
        a.share_A_with = -1
    # member 40: an invalid share index and a row pointer that must not be read
    arr[40].share_A_with = -7
    arr[40].row_ptr = C.cast(C.c_void_p(16), C.POINTER(C.c_int64))
    arr[70].share_A_with = 40                 # shares with the invalid member
    h, bad = C.c_void_p(), C.c_int32(-1)
    hh, nb = C.c_uint64(), C.c_int64()
    rc = c.lib().acs_debug_batch_image(count, arr, None, C.byref(hh), C.byref(nb), C.byref(bad))
    assert (rc, bad.value) == (c.ERR_ARG, 40)
    rc = c.lib().acs_batch_create(count, arr, None, None, C.byref(h), C.byref(bad))
    assert (rc, bad.value) == (c.ERR_ARG, 40) and not h.value


_CHAIN_CHILD = r"""
import ctypes as C, mmap, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2103_00736_gb300 import capi as c, instances as I
small = I.bernoulli_lp(11, 5, 12, density=0.4)          # m = 5: row_ptr has 6 entries
big = I.bernoulli_lp(12, 10, 12, density=0.4)           # m = 10, same n
PAGE = mmap.PAGESIZE
buf = mmap.mmap(-1, 2 * PAGE, prot=mmap.PROT_READ | mmap.PROT_WRITE)
base = C.addressof(C.c_char.from_buffer(buf))
libc = C.CDLL(None)
libc.mprotect.argtypes = [C.c_void_p, C.c_size_t, C.c_int]
# member 0's row pointer ends where a page that must not be read begins
rp_addr = base + PAGE - 8 * (small.m + 1)
C.memmove(rp_addr, np.ascontiguousarray(small.row_ptr, np.int64).ctypes.data, 8 * (small.m + 1))
assert libc.mprotect(base + PAGE, PAGE, 0) == 0
keep = []
arr = (c.acs_instance * 3)()
for i, x in enumerate((small, big, big)):
    cl = np.ascontiguousarray(x.col, np.int32); vl = np.ascontiguousarray(x.val, np.float64)
    b = np.ascontiguousarray(x.b, np.float64); cc = np.ascontiguousarray(x.c, np.float64)
    rp = np.ascontiguousarray(x.row_ptr, np.int64)
    keep += [cl, vl, b, cc, rp]
    a = arr[i]
    a.m, a.n = x.m, x.n
    a.row_ptr = C.cast(C.c_void_p(rp_addr), C.POINTER(C.c_int64)) if i == 0 else c._ptr(rp, C.c_int64)
    a.col, a.val = c._ptr(cl, C.c_int32), c._ptr(vl, C.c_double)
    a.b, a.c = c._ptr(b, C.c_double), c._ptr(cc, C.c_double)
    a.n_orthant, a.n_soc, a.soc_dims = x.n, 0, None
    a.share_A_with = -1
arr[1].share_A_with = 0      # invalid: member 0 has other dimensions
arr[2].share_A_with = 1      # passes the direct check; the chain leads to member 0
bad = C.c_int32(-1)
hh, nb = C.c_uint64(), C.c_int64()
rc = c.lib().acs_debug_batch_image(3, arr, None, C.byref(hh), C.byref(nb), C.byref(bad))
print("RESULT", rc, bad.value)
"""


def test_batch_share_chain_of_other_dimensions(capi):
    """A chain 2 -> 1 -> 0 whose middle link has other dimensions than its
    ends: member 1 is reported, and member 2's check stops at the link
    instead of reading member 0's arrays with member 2's sizes (member 0's
    row pointer ends at a page that may not be read; the check runs in a
    child process, so a read past it would show as a crash)."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _CHAIN_CHILD, root], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stderr[-2000:])
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT")][-1].split()
    assert (int(line[1]), int(line[2])) == (capi.ERR_ARG, 1)


def _bf16_value(t):
    """The float value of BF16 pattern(s) t (upper half of an FP32)."""
    return (np.asarray(t, np.uint32) << 16).view(np.float32).astype(np.float64)


def test_bf16_storage_rounds_to_nearest_even(capi):
    """The stored BF16 value of x is the BF16 value nearest to its FP32 value,
    ties to the even pattern (checked against both neighbours, not by
    repeating the bit trick)."""
    rng = np.random.default_rng(17)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.uniform(-30, 30, 20000),
                        [0.0, -0.0, 1.0, -1.0, 3.0, 1e-40, -1e-40]])
    f = x.astype(np.float32)
    lo = (f.view(np.uint32) >> 16).astype(np.uint32)         # truncation toward zero in magnitude
    hi = lo + 1
    d_lo = np.abs(_bf16_value(lo) - f.astype(np.float64))
    d_hi = np.abs(_bf16_value(hi) - f.astype(np.float64))
    want = np.where(d_lo < d_hi, lo, np.where(d_hi < d_lo, hi, np.where(lo % 2 == 0, lo, hi)))
    got = capi.acs_debug_to_bf16(x)
    assert np.array_equal(got, want.astype(np.uint16))
    # exact ties (low half 0x8000) go to the even pattern, both ways
    ties = (np.array([0x3F808000, 0x3F818000, 0xBF808000, 0xC0418000], np.uint32)).view(np.float32)
    got = capi.acs_debug_to_bf16(ties.astype(np.float64))
    assert list(got) == [0x3F80, 0x3F82, 0xBF80, 0xC042]


def test_device_cache_api_on_the_host(capi):
    """The cache's bookkeeping needs no GPU: nothing kept, trim is a no-op,
    a negative device is an argument error for the statistics."""
    st = capi.acs_device_cache_stats(0)
    assert st["bytes"] == 0
    capi.acs_device_cache_trim(-1)
    with pytest.raises(capi.AcsError) as e:
        capi.acs_device_cache_stats(-1)
    assert e.value.code == capi.ERR_ARG

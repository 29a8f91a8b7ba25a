"""GPU: the sliced-ELLPACK images of A and A' that acs_problem_create builds
on the device equal, entry for entry, the host builder's images
(acs_debug_sell, itself checked against the input in tests/test_sell_host.py):
relabelling, slice tables, columns, FP64 values, and the FP32 copy is the
FP64 value rounded to nearest."""
import numpy as np
import pytest
import scipy.sparse as sp

pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2103_00736_gb300 import capi, instances as I  # noqa: E402


def _long_column_lp():
    """A sparse LP whose column 0 holds 5000 entries (above the device sort's
    4096: the host builder takes over) and column 1 holds 600 (CTA sort)."""
    rng = np.random.default_rng(11)
    m, n = 6000, 9000
    A = sp.random(m, n, density=0.001, random_state=rng, format="lil")
    A[:5000, 0] = rng.standard_normal((5000, 1))
    A[:600, 1] = rng.standard_normal((600, 1))
    A = A.tocsr()
    A.sort_indices()
    empty = np.flatnonzero(np.diff(A.indptr) == 0)
    if empty.size:
        A = (A + sp.csr_matrix((np.ones(empty.size), (empty, np.full(empty.size, 5))), shape=(m, n))).tocsr()
        A.sort_indices()
    return I.planted_lp(A.indptr, A.indices, A.data, m, n, seed=3)


CASES = {
    "small_lp": lambda: I.small_lp(),
    "large_lp_2pct": lambda: I.large_lp(scale=0.02),
    "socp": lambda: I.socp(scale=0.002),
    "dense_lp_400": lambda: I.dense_lp(400),
    "long_columns": _long_column_lp,
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_device_images_equal_the_host_builder(name):
    inst = CASES[name]()
    with capi.Solver(inst) as s:
        info = capi.acs_problem_info(s.h)
        warps = info["grid32"] * info["threads"] // 32
        for which in (0, 1):
            dev = capi.acs_debug_images(s.h, which)
            host = capi.acs_debug_sell(inst.m, inst.n, inst.row_ptr, inst.col, inst.val, which, warps)
            assert (dev["rows"], dev["slices"], dev["g"], dev["stored"]) == \
                (host["rows"], host["slices"], host["g"], host["stored"])
            np.testing.assert_array_equal(dev["sptr"], host["sptr"])
            np.testing.assert_array_equal(dev["slen"], host["slen"])
            np.testing.assert_array_equal(dev["col"], host["col"])
            np.testing.assert_array_equal(dev["val"], host["val"])
            np.testing.assert_array_equal(dev["v32"], host["val"].astype(np.float32))


def test_device_cache_reuses_the_blocks_of_a_destroyed_handle():
    """Create/solve/destroy twice: the second create's buffers come from the
    cache, its result equals the first; trim returns the blocks."""
    capi.acs_device_cache_trim(-1)
    inst = I.large_lp(scale=0.02)
    out = []
    for k in range(2):
        before = capi.acs_device_cache_stats(0)
        with capi.Solver(inst) as s:
            st = s.solve(tol=1e-6, max_iter=20000)
            _, x, y, z, iters, res = s.get()
        after = capi.acs_device_cache_stats(0)
        out.append((st, x, iters, after["hits"] - before["hits"], after["misses"] - before["misses"]))
    assert out[0][0] == capi.SOLVED and out[1][0] == capi.SOLVED and out[0][2] == out[1][2]
    np.testing.assert_array_equal(out[0][1], out[1][1])
    assert out[1][3] > 0 and out[1][4] < out[0][4], out
    assert capi.acs_device_cache_stats(0)["bytes"] > 0
    capi.acs_device_cache_trim(-1)
    assert capi.acs_device_cache_stats(0)["bytes"] == 0

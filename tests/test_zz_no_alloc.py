"""The allocation-free residual entry point (acs_kkt_residuals_noalloc).

Callers that cannot allocate device memory (code running inside another
framework's memory pool, under a fixed memory budget, or in a loop that must
not enter the allocator) pass every input and the output in device memory
they own; the entry point keeps its temporaries in a fixed device array.  This
file checks it through the C ABI, on several calls in a row (a call that
failed to clear the shared array would show up), against the residuals the
solver itself reports (acs_get) and against the FP64 CPU oracle's residual
function evaluated on the same point.  It is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2103_00736_gb300 import capi, instances as I  # noqa: E402
from oracle import kkt  # noqa: E402


def _dev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _solve_and_compare(inst, **settings):
    with capi.Solver(inst, **settings) as s:
        st = s.solve(tol=1e-6, max_iter=20000)
        rc, x, y, z, iters, res = s.get()
    assert st == capi.SOLVED
    dims = np.asarray(inst.soc_dims, dtype=np.int64)
    off = (inst.n_orth + np.concatenate([[0], np.cumsum(dims)])).astype(np.int32)
    keep = [_dev(inst.row_ptr.astype(np.int32), torch.int32), _dev(inst.col, torch.int32),
            _dev(inst.val, torch.float64), _dev(inst.b, torch.float64), _dev(inst.c, torch.float64),
            _dev(x, torch.float64), _dev(y, torch.float64), _dev(z, torch.float64),
            _dev(off, torch.int32)]
    out = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    ptr = [t.data_ptr() for t in keep]
    rc = capi.acs_kkt_residuals_noalloc(inst.m, inst.n, ptr[0], ptr[1], ptr[2], ptr[3], ptr[4],
                                        ptr[5], ptr[6], ptr[7], inst.n_orth, len(dims), ptr[8],
                                        out.data_ptr(), stream.cuda_stream)
    assert rc == capi.SOLVED, capi.acs_status_string(rc)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for k in range(4):                      # r_p, r_d, r_gap, r_cone
        assert abs(got[k] - res[k]) <= 1e-9 + 1e-6 * res[k], (k, got[k], res[k])
    for k in (4, 5):                        # c'x, b'y
        assert abs(got[k] - res[k]) <= 1e-9 * (1.0 + abs(res[k])), (k, got[k], res[k])
    ref = kkt.residuals(inst.to_scipy(), inst.b, inst.c, x, y, z, inst.n_orth, inst.soc_dims)
    for k, key in enumerate(("r_p", "r_d", "r_gap", "r_cone")):
        # FP64 sums in another order: the residuals are differences of large
        # terms, so their last few digits are rounding
        assert abs(got[k] - ref[key]) <= 1e-12 + 1e-6 * ref[key], (key, got[k], ref[key])
    for k, key in ((4, "obj_p"), (5, "obj_d")):
        assert abs(got[k] - ref[key]) <= 1e-12 * (1.0 + abs(ref[key])), (key, got[k], ref[key])
    return got


def test_noalloc_residuals_match_solver_on_consecutive_calls():
    lp = I.small_lp()
    socp = I.socp(scale=0.002)
    first = _solve_and_compare(lp, cond_first=300, cond_period=100)
    _solve_and_compare(socp, t=1.7, cond_first=200, cond_period=100)
    again = _solve_and_compare(lp, cond_first=300, cond_period=100)
    # the shared array was cleared between the calls: same point, same values
    np.testing.assert_allclose(again, first, rtol=1e-12, atol=1e-15)


def test_noalloc_rejects_n_above_its_limit():
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = dummy.data_ptr()
    rc = capi.acs_kkt_residuals_noalloc(1, (1 << 20) + 1, p, p, p, p, p, p, p, p, 1, 0, 0, p, 0)
    assert rc == capi.ERR_LIMIT

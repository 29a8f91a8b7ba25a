"""Host-only checks of the sliced-ELLPACK preparation every device product
reads (through acs_debug_sell; no device involved).

Bit-exact bars (index and byte work): the row relabelling is a permutation
that sorts rows by decreasing length, stably, within windows of 2048; the
matrix rebuilt from the lane layout (entry k of local row r of slice q at
sptr[q] + 32 (k / g) + r g + k mod g) is the relabelled A, respectively A',
entry for entry and in each row's order; padding is column 0, value 0; every
slice is as long as its longest row needs.
"""
import os

import numpy as np
import pytest

WINDOW = 2048


@pytest.fixture(scope="module")
def capi():
    from paper_2103_00736_gb300 import capi as c, build
    if not os.path.exists(c.LIB_PATH):
        build.build()
    c.lib()
    return c


def _ragged_csr(rng, m, n, long_rows=3):
    """Row lengths from 1 to ~n/4 (mostly short, a few long), sorted distinct
    columns, some empty columns."""
    lens = np.minimum(rng.geometric(0.15, m), n)
    lens[rng.choice(m, size=min(long_rows, m), replace=False)] = max(1, n // 4)
    cols = [np.sort(rng.choice(n - 3, size=min(k, n - 3), replace=False)) for k in lens]  # last 3 columns empty
    row_ptr = np.zeros(m + 1, np.int64)
    row_ptr[1:] = np.cumsum([len(c) for c in cols])
    col = np.concatenate(cols).astype(np.int32)
    val = rng.standard_normal(col.size)
    return row_ptr, col, val


def _rows_from_sell(S):
    """Every row rebuilt from the lane layout: (columns, values) over the
    slice's full length, the row's entries first, then its padding."""
    g, h = S["g"], 32 // S["g"]
    rows = []
    for q in range(S["slices"]):
        for lr in range(h):
            r = q * h + lr
            if r >= S["rows"]:
                break
            cs, vs = [], []
            for k in range(S["slen"][q] * g):
                idx = S["sptr"][q] + 32 * (k // g) + lr * g + (k % g)
                cs.append(S["col"][idx])
                vs.append(S["val"][idx])
            rows.append((np.array(cs, np.int64), np.array(vs)))
    return rows


def _check_layout(S):
    g = S["g"]
    assert g in (1, 2, 4, 8, 16, 32)
    h = 32 // g
    assert S["slices"] == -(-S["rows"] // h)
    assert S["sptr"][0] == 0 and np.array_equal(np.diff(S["sptr"]), 32 * S["slen"])
    assert S["stored"] == S["sptr"][-1]


def _check_rows(S, want_rows):
    """want_rows[r] = (columns, values) of row r in order."""
    got = _rows_from_sell(S)
    assert len(got) == len(want_rows)
    g, h = S["g"], 32 // S["g"]
    for r, ((gc, gv), (wc, wv)) in enumerate(zip(got, want_rows)):
        k = len(wc)
        assert np.array_equal(gc[:k], wc) and np.array_equal(gv[:k], wv), r
        assert not gc[k:].any() and not gv[k:].any(), r          # padding: column 0, value 0
    for q in range(S["slices"]):                                   # no slice longer than needed
        longest = max(len(want_rows[r][0]) for r in range(q * h, min(S["rows"], q * h + h)))
        assert S["slen"][q] == -(-longest // g), q


@pytest.mark.parametrize("m,n,warps,seed", [(37, 60, 1, 0), (300, 500, 8, 1), (4500, 900, 4864, 2),
                                            (5000, 200, 64, 3)])
def test_sell_image_of_A_and_At(capi, m, n, warps, seed):
    rng = np.random.default_rng(seed)
    row_ptr, col, val = _ragged_csr(rng, m, n)
    lens = np.diff(row_ptr)
    A = capi.acs_debug_sell(m, n, row_ptr, col, val, 0, warps)
    perm = A["perm"]
    assert np.array_equal(np.sort(perm), np.arange(m))
    for w0 in range(0, m, WINDOW):                   # stable sort by decreasing length per window
        seg = perm[w0:w0 + WINDOW]
        assert np.all(seg >= w0) and np.all(seg < w0 + WINDOW)
        key = list(zip(-lens[seg], seg))
        assert key == sorted(key)
    _check_layout(A)
    assert A["rows"] == m
    _check_rows(A, [(col[row_ptr[i]:row_ptr[i + 1]], val[row_ptr[i]:row_ptr[i + 1]]) for i in perm])

    At = capi.acs_debug_sell(m, n, row_ptr, col, val, 1, warps)
    assert np.array_equal(At["perm"], perm)
    _check_layout(At)
    assert At["rows"] == n
    # row j of A' lists the relabelled rows r with A[perm[r], j] != 0, increasing
    inv = np.empty(m, np.int64)
    inv[perm] = np.arange(m)
    rows_of = [[] for _ in range(n)]
    for i in range(m):
        for k in range(row_ptr[i], row_ptr[i + 1]):
            rows_of[col[k]].append((inv[i], val[k]))
    want = []
    for j in range(n):
        e = sorted(rows_of[j])
        want.append((np.array([r for r, _ in e], np.int64), np.array([v for _, v in e])))
    _check_rows(At, want)
    assert all(len(want[j][0]) == 0 for j in range(n - 3, n))   # empty columns are empty rows of A'


def test_lanes_per_row(capi):
    """g is a power of two, grows with the team (more warps want more slices),
    and stays within the average row length."""
    rng = np.random.default_rng(9)
    m, n = 3000, 4000
    row_ptr, col, val = _ragged_csr(rng, m, n, long_rows=0)
    avg = col.size / m
    gs = [capi.acs_debug_sell(m, n, row_ptr, col, val, 0, w)["g"] for w in (1, 16, 256, 4864)]
    assert gs == sorted(gs)
    for g in gs:
        assert g == 1 or g <= avg
    assert gs[0] == 1 and gs[-1] > 1


def test_sell_rejects_malformed_csr(capi):
    row_ptr = np.array([0, 2, 3], np.int64)
    with pytest.raises(capi.AcsError) as e:
        capi.acs_debug_sell(2, 3, row_ptr, np.array([1, 0, 2], np.int32), np.ones(3), 0, 8)   # unsorted row
    assert e.value.code == capi.ERR_CSR
    with pytest.raises(capi.AcsError) as e:
        capi.acs_debug_sell(2, 3, row_ptr, np.array([0, 1, 2], np.int32), np.ones(3), 2, 8)   # which
    assert e.value.code == capi.ERR_ARG


def _decode(S, indptr):
    """Positions in the image of every entry of the CSR rows given by
    indptr (row r's k-th entry), and a mask of the padding positions."""
    g, h = S["g"], 32 // S["g"]
    lens = np.diff(indptr)
    r = np.repeat(np.arange(lens.size), lens)
    k = np.arange(indptr[-1]) - np.repeat(indptr[:-1], lens)
    idx = S["sptr"][r // h].astype(np.int64) + 32 * (k // g) + (r % h) * g + (k % g)
    pad = np.ones(S["stored"], bool)
    pad[idx] = False
    return idx, pad


def test_sell_image_above_2_20_entries(capi):
    """Above 2^20 entries the preparation runs on several threads and sorts
    A' through column buckets; the image is the same exact layout."""
    import scipy.sparse as sp
    rng = np.random.default_rng(21)
    m, n, per = 20000, 150001, 8
    rows = np.concatenate([rng.choice(m, per, replace=False) for _ in range(n)])
    cols = np.repeat(np.arange(n), per)
    A = sp.csr_matrix((rng.standard_normal(rows.size), (rows, cols)), shape=(m, n))
    A.sort_indices()
    assert A.nnz >= 1 << 20
    rp, ci, va = A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data
    S = capi.acs_debug_sell(m, n, rp, ci, va, 0, 152 * 32)
    Ap = A[S["perm"]]
    idx, pad = _decode(S, Ap.indptr)
    assert np.array_equal(S["col"][idx], Ap.indices) and np.array_equal(S["val"][idx], Ap.data)
    assert not S["col"][pad].any() and not S["val"][pad].any()
    T = capi.acs_debug_sell(m, n, rp, ci, va, 1, 152 * 32)
    At = Ap.T.tocsr()
    At.sort_indices()                                  # relabelled rows increasing in every column
    idx, pad = _decode(T, At.indptr)
    assert np.array_equal(T["col"][idx], At.indices) and np.array_equal(T["val"][idx], At.data)
    assert not T["col"][pad].any() and not T["val"][pad].any()
    # the checks of the input run in parallel too, with the serial order's codes
    bad_v = va.copy()
    bad_v[-3] = np.nan
    with pytest.raises(capi.AcsError) as e:
        capi.acs_debug_sell(m, n, rp, ci, bad_v, 0, 152 * 32)
    assert e.value.code == capi.ERR_ARG
    bad_c = ci.copy()
    bad_c[-2] = n                                     # column out of range in the last row
    for v in (va, bad_v):                             # ... with or without a NaN as well: CSR first
        with pytest.raises(capi.AcsError) as e:
            capi.acs_debug_sell(m, n, rp, bad_c, v, 0, 152 * 32)
        assert e.value.code == capi.ERR_CSR

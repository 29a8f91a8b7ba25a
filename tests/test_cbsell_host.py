"""Host-only checks of the column-blocked image read by the FP32 passes of
the single-problem launch (through acs_debug_cbsell; no device involved).

Bit-exact bars (index and byte work):
  * the blocks cut the columns into nblocks runs of `width` columns (the
    last possibly shorter), width a multiple of 4 and at most the limit;
  * every row appears exactly once in every block, in the window of 2048
    rows it belongs to, and the rows of a window are ordered by decreasing
    count of entries in that block, stably (equal counts keep row order);
  * the matrix rebuilt from the lane layout (entry k of the row in lane r of
    an item at sptr[item] + 32 k + r, column = block * width + stored
    column) is the relabelled A, respectively A', entry for entry in each
    row's order, with FP32 values; padding is column 0, value 0; every item
    is as long as its longest row needs, and at least one chunk; the
    item-end marks flag exactly the last chunk of every item; ipos is the
    inverse of the row ids (the slot of every row in every block);
  * the items are dealt to the CTAs as contiguous ranges covering all items
    once, each range's work (chunks + 1 per item) within one item of an
    equal share.
"""
import os

import numpy as np
import pytest

WINDOW = 2048
SLICES_PER_WINDOW = WINDOW // 32
NO_ROW = 0xFFFF


@pytest.fixture(scope="module")
def capi():
    from paper_2103_00736_gb300 import capi as c, build
    if not os.path.exists(c.LIB_PATH):
        build.build()
    c.lib()
    return c


def _random_csr(rng, m, n, per_row_mean):
    lens = np.clip(rng.poisson(per_row_mean, m), 1, n)
    cols = [np.sort(rng.choice(n, size=k, replace=False)) for k in lens]
    row_ptr = np.zeros(m + 1, np.int64)
    row_ptr[1:] = np.cumsum(lens)
    return row_ptr, np.concatenate(cols).astype(np.int32), rng.standard_normal(int(row_ptr[-1]))


def _relabelled_rows(row_ptr, col, val, perm):
    return [(col[row_ptr[i]:row_ptr[i + 1]].astype(np.int64), val[row_ptr[i]:row_ptr[i + 1]]) for i in perm]


def _transpose_rows(row_ptr, col, val, perm, n):
    """Rows of A' of the relabelled A: for each column j, (relabelled row
    indices in increasing order, values)."""
    out = [([], []) for _ in range(n)]
    for r, i in enumerate(perm):
        for k in range(row_ptr[i], row_ptr[i + 1]):
            out[col[k]][0].append(r)
            out[col[k]][1].append(val[k])
    return [(np.array(a, np.int64), np.array(b)) for a, b in out]


def _check(S, rows, width_limit, ctas):
    R, ncols, W, nb, nsl = S["rows"], S["cols"], S["width"], S["nblocks"], S["nsl"]
    assert R == len(rows)
    assert W % 4 == 0 and 4 <= W <= max(4, width_limit - width_limit % 4)
    assert nb == -(-ncols // W) and (nb - 1) * W < ncols
    assert nsl == -(-R // 32)
    sptr, rowid = S["sptr"], S["rowid"]
    assert sptr[0] == 0 and np.all(np.diff(sptr) % 32 == 0) and S["stored"] == sptr[-1]
    lens = np.diff(sptr) // 32
    got = [[([], []) for _ in range(nb)] for _ in range(R)]
    for b in range(nb):
        seen = np.zeros(R, bool)
        for q in range(nsl):
            item = b * nsl + q
            counts = []
            for lane in range(32):
                rid = int(rowid[item * 32 + lane])
                if rid == NO_ROW:
                    counts.append(-1)
                    continue
                r = (q // SLICES_PER_WINDOW) * WINDOW + rid
                assert r < R and not seen[r], (b, q, lane)
                seen[r] = True
                cs, vs = [], []
                for k in range(lens[item]):
                    idx = sptr[item] + 32 * k + lane
                    cs.append(int(S["col"][idx]) + b * W)
                    vs.append(float(S["val"][idx]))
                got[r][b] = (cs, vs)
                counts.append(int(np.sum((rows[r][0] >= b * W) & (rows[r][0] < (b + 1) * W))))
            real = [c for c in counts if c >= 0]
            assert lens[item] == max(1, max(real) if real else 0), (b, q)   # at least one chunk
            # NO_ROW lanes only after the real ones
            assert counts == real + [-1] * (32 - len(real)), (b, q)
        assert seen.all(), b
        # stable order by decreasing count within every window
        for w in range(-(-R // WINDOW)):
            order = []
            for q in range(w * SLICES_PER_WINDOW, min(nsl, (w + 1) * SLICES_PER_WINDOW)):
                for lane in range(32):
                    rid = int(rowid[(b * nsl + q) * 32 + lane])
                    if rid != NO_ROW:
                        order.append(w * WINDOW + rid)
            cnt = [int(np.sum((rows[r][0] >= b * W) & (rows[r][0] < (b + 1) * W))) for r in order]
            key = sorted(range(len(order)), key=lambda k: (-cnt[k], order[k]))
            assert key == list(range(len(order))), (b, w)
    for r in range(R):
        wc, wv = rows[r]
        for b in range(nb):
            sel = (wc >= b * W) & (wc < (b + 1) * W)
            k = int(sel.sum())
            cs, vs = got[r][b]
            assert cs[:k] == list(wc[sel]), (r, b)
            assert np.array_equal(np.array(vs[:k], np.float32), wv[sel].astype(np.float32)), (r, b)
            assert all(c == b * W for c in cs[k:]) and not any(vs[k:]), (r, b)   # padding: column 0, value 0
    # ipos is the inverse of rowid: the slot of every row of a window in every block
    ipos = S["ipos"]
    for b in range(nb):
        for q in range(nsl):
            for lane in range(32):
                rid = int(rowid[(b * nsl + q) * 32 + lane])
                if rid != NO_ROW:
                    r = (q // SLICES_PER_WINDOW) * WINDOW + rid
                    assert ipos[b * nsl * 32 + r] == (q % SLICES_PER_WINDOW) * 32 + lane, (b, r)
    # item-end marks: exactly the last chunk of every item
    marks = np.unpackbits(S["cend"].view(np.uint8), bitorder="little").astype(bool)
    want = np.zeros(marks.size, bool)
    want[sptr[1:] // 32 - 1] = True
    assert np.array_equal(marks, want)
    cta = S["cta_beg"]
    assert cta[0] == 0 and cta[-1] == nb * nsl and np.all(np.diff(cta) >= 0)
    work = lens + 1
    share = work.sum() / ctas
    for c in range(ctas):
        w = work[cta[c]:cta[c + 1]].sum()
        assert w <= share + work.max() + 1e-9, (c, w, share)


@pytest.mark.parametrize("m,n,per_row,limit,ctas", [
    (300, 500, 6.0, 64, 7),       # several blocks, a ragged last block, one partial window
    (2500, 300, 9.0, 40, 16),     # two windows, the last partial; many blocks
    (70, 41, 3.0, 4, 3),          # the smallest block width
    (40, 1000, 30.0, 100000, 5),  # one block (limit above the column count)
])
def test_cbsell_layout_A_and_At(capi, m, n, per_row, limit, ctas):
    rng = np.random.default_rng(20210301 + m + n)
    row_ptr, col, val = _random_csr(rng, m, n, per_row)
    SA = capi.acs_debug_cbsell(m, n, row_ptr, col, val, 0, limit, ctas)
    rows_A = _relabelled_rows(row_ptr, col, val, SA["perm"])
    _check(SA, rows_A, limit, ctas)
    ST = capi.acs_debug_cbsell(m, n, row_ptr, col, val, 1, limit, ctas)
    assert np.array_equal(ST["perm"], SA["perm"])
    _check(ST, _transpose_rows(row_ptr, col, val, SA["perm"], n), limit, ctas)


def test_cbsell_product_matches_dense(capi):
    """Emulating the pass on the host (partials per block added in block
    order, FP32) gives A x to FP32 accuracy: the image describes A."""
    rng = np.random.default_rng(7)
    m, n = 400, 700
    row_ptr, col, val = _random_csr(rng, m, n, 8.0)
    S = capi.acs_debug_cbsell(m, n, row_ptr, col, val, 0, 96, 5)
    x = rng.standard_normal(n).astype(np.float32)
    part = np.zeros((S["nblocks"], m), np.float32)
    lens = np.diff(S["sptr"]) // 32
    for item in range(S["nblocks"] * S["nsl"]):
        b, q = divmod(item, S["nsl"])
        for lane in range(32):
            rid = int(S["rowid"][item * 32 + lane])
            if rid == NO_ROW:
                continue
            acc = np.float32(0)
            for k in range(lens[item]):
                idx = S["sptr"][item] + 32 * k + lane
                acc = np.float32(acc + S["val"][idx] * x[b * S["width"] + S["col"][idx]])
            part[b, (q // SLICES_PER_WINDOW) * WINDOW + rid] = acc
    y = part.sum(axis=0, dtype=np.float64)
    A = np.zeros((m, n))
    for r, i in enumerate(S["perm"]):
        A[r, col[row_ptr[i]:row_ptr[i + 1]]] = val[row_ptr[i]:row_ptr[i + 1]]
    want = A @ x.astype(np.float64)
    assert np.max(np.abs(y - want)) <= 1e-5 * (np.abs(A) @ np.abs(x)).max()


def test_cbsell_rejects_bad_arguments(capi):
    row_ptr, col, val = np.array([0, 1], np.int64), np.array([0], np.int32), np.array([1.0])
    for which, limit, ctas in ((2, 64, 1), (0, 3, 1), (0, 64, 0)):
        with pytest.raises(capi.AcsError):
            capi.acs_debug_cbsell(1, 1, row_ptr, col, val, which, limit, ctas)

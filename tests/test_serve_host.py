"""Host-only checks of the serving loop's bookkeeping, through the C ABI's
debug entry points (no device involved):

  * the first-fit pool that places admitted requests in one device
    allocation agrees offset for offset with a granule-bitmap model of first
    fit (lowest address with enough consecutive free 256-byte granules),
    which holds only if freed neighbours are coalesced;
  * the work-sized teams of a round: every request gets a power-of-two team
    of at least one CTA and at most its work cap, the teams are contiguous
    and fit the grid, and no team could still be doubled.
"""
import os

import numpy as np
import pytest

GRAN = 256
MAX_GRID = 256


@pytest.fixture(scope="module")
def capi():
    from paper_2103_00736_gb300 import capi as c, build
    if not os.path.exists(c.LIB_PATH):
        build.build()
    c.lib()
    return c


# ---------------------------------------------------------------- pool

class BitmapFirstFit:
    def __init__(self, cap):
        self.free = np.ones(cap // GRAN, dtype=bool)

    def alloc(self, nbytes):
        k = -(-nbytes // GRAN)
        run = 0
        for i, f in enumerate(self.free):
            run = run + 1 if f else 0
            if run == k:
                a = i - k + 1
                self.free[a:a + k] = False
                return a * GRAN
        return -1

    def release(self, off, nbytes):
        k = -(-nbytes // GRAN)
        a = off // GRAN
        assert not self.free[a:a + k].any()
        self.free[a:a + k] = True

    def used(self):
        return int((~self.free).sum()) * GRAN


def _random_ops(rng, nops, cap):
    ops, live = [], []
    for k in range(nops):
        if live and rng.random() < 0.45:
            j = live.pop(int(rng.integers(len(live))))
            ops.append(-j - 1)
        else:
            ops.append(int(rng.integers(1, cap // 6)))
            live.append(k)
    return ops


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_pool_is_first_fit_with_coalescing(capi, seed):
    rng = np.random.default_rng(seed)
    cap = 64 * 1024 + 100                       # rounded down to whole granules
    ops = _random_ops(rng, 400, cap)
    # frees may only name successful allocations: replay on the model first
    model, sizes, fixed = BitmapFirstFit(cap), {}, []
    for k, op in enumerate(ops):
        if op > 0:
            off = model.alloc(op)
            if off >= 0:
                sizes[k] = (off, op)
            fixed.append(op)
        else:
            j = -op - 1
            if j in sizes:
                model.release(*sizes.pop(j))
                fixed.append(op)
            else:
                fixed.append(1 + int(rng.integers(1, 4096)))   # an allocation instead
                off = model.alloc(fixed[-1])
                if off >= 0:
                    sizes[k] = (off, fixed[-1])
    offs, used, peak = capi.acs_debug_arena(cap, fixed)
    model, peak_m = BitmapFirstFit(cap), 0
    for k, op in enumerate(fixed):
        if op > 0:
            assert offs[k] == model.alloc(op), k
            peak_m = max(peak_m, model.used())
        else:
            j = -op - 1
            model.release(offs[j], fixed[j])
            assert offs[k] == -1
    assert used == model.used() and peak == peak_m
    assert (offs[offs >= 0] % GRAN == 0).all()
    assert (offs == -1).sum() > (np.array(fixed) < 0).sum()    # the pool did fill up


def test_pool_coalesces_freed_neighbours(capi):
    cap = 16 * GRAN
    quarter = 4 * GRAN
    # four quarters, free the middle two in either order, then half fits there
    for order in ((-2, -3), (-3, -2)):
        ops = [quarter] * 4 + list(order) + [2 * quarter]
        offs, used, peak = capi.acs_debug_arena(cap, ops)
        assert list(offs[:4]) == [0, quarter, 2 * quarter, 3 * quarter]
        assert offs[6] == quarter
        assert used == cap and peak == cap
    # everything freed in a scattered order leaves one block of the whole pool
    ops = [GRAN] * 16 + [-(j + 1) for j in (5, 0, 15, 7, 6, 1, 14, 2, 3, 9, 8, 4, 13, 10, 12, 11)] + [cap]
    offs, used, peak = capi.acs_debug_arena(cap, ops)
    assert offs[-1] == 0 and used == cap


def test_pool_rounds_to_granules_and_rejects_bad_frees(capi):
    offs, used, peak = capi.acs_debug_arena(10 * GRAN + 255, [1, GRAN + 1, 10 * GRAN])
    assert list(offs) == [0, GRAN, -1] and used == 3 * GRAN
    with pytest.raises(capi.AcsError):
        capi.acs_debug_arena(4 * GRAN, [GRAN, -1, -1])          # freed twice
    with pytest.raises(capi.AcsError):
        capi.acs_debug_arena(4 * GRAN, [-1])                     # frees a later op
    with pytest.raises(capi.AcsError):
        capi.acs_debug_arena(GRAN, [2 * GRAN, -1])               # frees a failed allocation


# ---------------------------------------------------------------- teams

def _pow2_floor(v):
    return 1 << (int(v).bit_length() - 1)


def _cap(w, grid):
    return min(_pow2_floor(max(1, int(w / 16384.0))), min(grid, MAX_GRID))


def _check_teams(work, grid, cta):
    pos, rank, size = cta
    n = len(work)
    g = np.zeros(n, dtype=int)
    b = 0
    for k in range(n):                           # contiguous, in request order
        assert pos[b] == k
        gk = int(size[b])
        assert gk >= 1 and gk & (gk - 1) == 0 and gk <= _cap(work[k], grid), (k, gk)
        assert list(pos[b:b + gk]) == [k] * gk
        assert list(rank[b:b + gk]) == list(range(gk))
        assert list(size[b:b + gk]) == [gk] * gk
        g[k] = gk
        b += gk
    assert (pos[b:] == -1).all()
    used = int(g.sum())
    assert used <= grid
    for k in range(n):                           # nothing left to double
        assert g[k] == _cap(work[k], grid) or used + g[k] > grid, (k, g[k], used)
    return g


@pytest.mark.parametrize("seed", range(6))
def test_teams_are_work_sized_and_fit(capi, seed):
    rng = np.random.default_rng(100 + seed)
    grid = int(rng.choice([152, 304, 76, 256]))
    n = int(rng.integers(1, min(grid, 60) + 1))
    work = np.exp(rng.uniform(np.log(2e3), np.log(5e7), n))
    g = _check_teams(work, grid, capi.acs_debug_assign_teams(work, grid))
    order = np.argsort(work)
    assert g[order[-1]] >= g[order[0]]          # the heaviest gets no fewer CTAs than the lightest


def test_teams_degenerate_cases(capi):
    grid = 152
    # as many requests as CTAs: one each
    cta = capi.acs_debug_assign_teams(np.full(grid, 1e7), grid)
    assert (cta[2] == 1).all() and list(cta[0]) == list(range(grid))
    # one heavy request: the largest power of two within the grid
    cta = capi.acs_debug_assign_teams([1e9], grid)
    assert (cta[2][:128] == 128).all() and (cta[0][128:] == -1).all()
    # small work is capped: w / 16384 CTAs at most
    cta = capi.acs_debug_assign_teams([3 * 16384.0, 100.0], grid)
    assert cta[2][0] == 2 and cta[2][2] == 1 and (cta[0][3:] == -1).all()
    # larger grids never give one team more than the persistent-launch maximum
    cta = capi.acs_debug_assign_teams([1e12], 1024)
    assert cta[2][0] == MAX_GRID
    for bad in (([], 152), ([1.0] * 5, 4), ([1.0, 0.0], 152), ([1.0, -2.0], 152), ([1.0], 0)):
        with pytest.raises(capi.AcsError):
            capi.acs_debug_assign_teams(*bad)

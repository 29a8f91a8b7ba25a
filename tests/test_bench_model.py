"""The byte models behind bench.py's roofline fractions (CPU only): the
fixed per-unit formula of the hot path, the implementation's own pass-count
models (single solve, batch member, crossover polish) and the roofline
object's arithmetic, so that a reported fraction can be recomputed from the
JSON line and these formulas."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

ZERO6 = [0, 0, 0, 0, 0, 0]


def test_path_bytes_of_the_large_lp_solve():
    """m = 2e5, n = 1e6, nnz = 1e7; 390 iterations, 1380 CG iterations, 39
    KKT checks, 2 rescalings: 390 x 182.4 MB + 1380 x 172 MB + 39 x 240 MB +
    2 x 80 MB = 318.016 GB, the figure of the formula worked by hand."""
    got = bench.path_bytes(200_000, 1_000_000, 10_000_000, 390, 1380, 39, 2)
    assert got == 390 * 182.4e6 + 1380 * 172e6 + 39 * 240e6 + 2 * 80e6
    assert got == pytest.approx(318.016e9, rel=1e-12)


@pytest.mark.parametrize("nnz", [1, 7, 10_000_000])
def test_the_models_count_the_same_matrix_stream(nnz):
    """With no vectors (m = n = 0) only the matrix bytes are left: an FP32
    outer iteration (one pass over A, one over A') is 16 nnz in both models,
    a CG iteration 16 nnz, a KKT check (one FP64 pass each way) 24 nnz."""
    assert bench.path_bytes(0, 0, nnz, 1, 0, 0, 0) == 16.0 * nnz
    assert bench.algorithmic_bytes(0, 0, nnz, ZERO6, 0, n32_A=1, n32_AT=1) == 16.0 * nnz
    assert bench.path_bytes(0, 0, nnz, 0, 1, 0, 0) == 16.0 * nnz
    assert bench.algorithmic_bytes(0, 0, nnz, [1, 1, 0, 0, 0, 0], 0) == 16.0 * nnz
    assert bench.path_bytes(0, 0, nnz, 0, 0, 1, 0) == 24.0 * nnz
    assert bench.algorithmic_bytes(0, 0, nnz, [0, 0, 1, 1, 0, 0], 0) == 24.0 * nnz


@pytest.mark.parametrize("counters", [[1380, 1380, 430, 431, 2, 39], [0, 0, 1, 1, 0, 0], [17, 17, 9, 12, 1, 2]])
def test_a_batch_member_is_a_single_solve_without_the_cached_operator(counters):
    """member_bytes takes the iteration count from its counters (one FP64 A'
    update pass per iteration besides the checks' and the rescalings');
    without dense corrections it equals algorithmic_bytes of that count."""
    m, n, nnz = 1000, 2500, 50_000
    iters = counters[3] - counters[5] - counters[4]
    assert bench.member_bytes(m, n, nnz, counters + [0, 0]) == pytest.approx(
        bench.algorithmic_bytes(m, n, nnz, counters, iters), rel=1e-15)
    # each dense correction reads the inverse factor twice: m^2 doubles
    assert bench.member_bytes(m, n, nnz, counters + [3, 1]) - bench.member_bytes(m, n, nnz, counters + [0, 0]) \
        == pytest.approx(3 * 8.0 * m * m, rel=1e-15)


def test_polish_bytes():
    m, n, nnz = 100_000, 500_000, 5_000_000
    # a support of every column and entry is the all-of-A count (the factored path)
    assert bench.polish_bytes(m, n, nnz, 171, 1, support=n, support_entries=nnz) == bench.polish_bytes(m, n, nnz, 171, 1)
    # FP32 corrections read 8 bytes an entry of A_B instead of 12, twice per CG iteration
    full = bench.polish_bytes(m, n, nnz, 171, 1, 480_000, 2_000_000, cg_entry_bytes=12.0)
    f32 = bench.polish_bytes(m, n, nnz, 171, 1, 480_000, 2_000_000, cg_entry_bytes=8.0)
    assert full - f32 == 171 * 2 * 4.0 * 2_000_000
    # a smaller support reads fewer bytes; no polish reads none
    assert bench.polish_bytes(m, n, nnz, 171, 1, 400_000, 1_500_000) < bench.polish_bytes(m, n, nnz, 171, 1, 480_000, 2_000_000)
    assert bench.polish_bytes(m, n, nnz, 0, 0, 480_000, 2_000_000) == 0.0


def test_roofline_entry_arithmetic():
    """achieved = bytes / launch time, frac = achieved / the measured copy
    bandwidth (the fallback figure when no measurement is present), and the
    own model reported beside it on the same time."""
    peak, kind = bench.measured_peak_hbm()
    assert peak > 0 and kind in ("measured", "fallback")
    r = bench.roofline_entry("k", 318.016e9, 240.0, traffic=350e9, own_bytes=400e9)
    assert r["achieved"] == pytest.approx(318.016e9 / 0.240 / 1e9, rel=1e-15)
    assert r["frac"] == pytest.approx(r["achieved"] / peak, rel=1e-15)
    assert r["peak"] == peak and r["peak_kind"] == kind and r["unit"] == "GB/s" and r["bound"] == "hbm"
    assert r["traffic"] == 350e9 and r["traffic_gbs"] == pytest.approx(350e9 / 0.240 / 1e9)
    assert r["own_model"]["frac"] == pytest.approx(400e9 / 0.240 / 1e9 / peak, rel=1e-15)
    assert bench.roofline_entry("k", 1e9, 1.0)["traffic_gbs"] is None

"""Host-side arithmetic of the benchmark (no GPU): the algorithmic work it charges to each kernel
of the blocked LU, and the roofline fractions it prints from a per-kernel profile.

The blocked LU performs exactly the multiply-adds of the unblocked one (Theorem thm:LU's dense LU
of U33, reorganised), so the bench's split of that work into sub-panel factorisations, in-panel
updates and trailing updates, plus the two triangular solves it does not charge (the unit-lower
solves for U12 inside and across the outer panels), must add up to the unblocked count:
for each pivot column k of an n x n matrix, (n - k - 1) multipliers and (n - k - 1)^2 updates."""
import json
import os

import pytest

pytest.importorskip("torch")
import bench  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _unblocked_flops(n):
    return 8.0 * sum((n - k - 1) ** 2 + (n - k - 1) for k in range(n))


def _uncharged_trsm_flops(n, NB, nbp):
    # unit-lower solves: rows j+1..j+ib-1 of a sub-panel against the rest of its outer panel, and
    # rows J+1..J+jb-1 of an outer panel against the trailing columns
    t = 0.0
    for J in range(0, n, NB):
        jb = min(NB, n - J)
        for j in range(J, J + jb, nbp):
            ib = min(nbp, J + jb - j)
            t += 8.0 * (J + jb - j - ib) * ib * (ib - 1) / 2
        t += 8.0 * (n - J - jb) * jb * (jb - 1) / 2
    return t


@pytest.mark.parametrize("n", [4096, 1000, 300, 32, 1])
def test_lu_work_adds_up_to_the_unblocked_lu(n):
    w = bench.lu_work(n)
    total = w["panel"] + w["inner"] + w["trailing"] + _uncharged_trsm_flops(n, 256, 32)
    assert total == pytest.approx(_unblocked_flops(n), rel=1e-12, abs=0.5)
    assert w["trailing"] >= 0 and w["inner"] >= 0 and (w["panel"] > 0) == (n > 1)


def test_lu_work_at_the_bench_size():
    # N = 4096: the trailing updates carry almost all of the (8/3) N^3 flops of the LU
    n = 4096
    w = bench.lu_work(n)
    assert w["trailing"] / _unblocked_flops(n) > 0.85
    # every outer panel moves its 2 NB rows across the other columns and its U12 block once
    assert w["swap_bytes"] == sum(16.0 * (2.0 * min(256, n - J) * (n - min(256, n - J))
                                          + min(256, n - J) * (n - J - min(256, n - J)))
                                  for J in range(0, n, 256))


def test_roofline_fractions_recompute_from_the_profile():
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else \
        {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}
    N, nrhs, iters = 4096, 65, 2
    prof = [("panel_lc_kernel", 128, 7.3), ("cgemm_tc_kernel (Schur complement)", 1, 3.5),
            ("resid_tc_kernel (+ split-K reduction)", 1, 1.2), ("trsv_flow_kernel", 4, 1.25),
            ("some_kernel_without_a_work_model", 3, 0.1)]
    roof, extra = bench.roofline_from_profile(prof, N, nrhs, 2, iters, peaks, "measured")
    # the dominant kernel is the one with the largest summed time, and the unmodelled one is left out
    assert roof["kernel"] == "panel_lc_kernel"
    assert [r["kernel"] for r in extra["kernels"]] == [p[0] for p in prof[1:4]]
    fp32 = 152 * 128 * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12
    tf32 = peaks["bf16_tflops"] * 1.1 / 2.25
    expect = {
        "panel_lc_kernel": (bench.lu_work(N)["panel"] / 7.3e-3 / 1e12, fp32),
        "cgemm_tc_kernel (Schur complement)": (16.0 * N ** 3 / 3.5e-3 / 1e12, tf32),
        "resid_tc_kernel (+ split-K reduction)": (16.0 * 4 * N * N / 1.2e-3 / 1e9, peaks["hbm_gbs"]),
        "trsv_flow_kernel": (iters * N * N * 8.0 / 1.25e-3 / 1e9, peaks["hbm_gbs"]),
    }
    for r in [roof] + extra["kernels"]:
        ach, peak = expect[r["kernel"]]
        assert r["achieved"] == pytest.approx(ach, rel=1e-12)
        assert r["peak"] == pytest.approx(peak, rel=1e-12)
        assert r["frac"] == pytest.approx(ach / peak, rel=1e-12)
        assert r["ms_per_launch"] * r["launches"] == pytest.approx(r["ms_total"], rel=1e-12)
        assert r["frac_note"]


def test_secondary_measurements_cannot_lose_the_headline():
    assert bench._guarded(lambda: {"ms": 1.0}) == {"ms": 1.0}

    def fails():
        raise RuntimeError("bm_solve: BM_ENOTCONV")

    assert bench._guarded(fails) == {"error": "RuntimeError: bm_solve: BM_ENOTCONV"}

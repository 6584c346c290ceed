"""Host-side arithmetic of bench.py (no GPU): the roofline rates from the per-category CUDA-event
times, the clock summary that decides whether a run is rejected, and the seeded batched workload."""
import importlib.util
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_kernel_rates_use_the_algorithmic_bytes(bench):
    N, n_pot, hbm = 1_000_000, 200_000, 6790.3
    prof = {"residual": (50.0, 10), "jvp": (30.0, 20)}   # total ms, calls
    r64 = bench.kernel_rates(prof, N, n_pot, hbm, "fp64")
    # residual: z, z^n, R for time-dependent unknowns (24 B), no z^n for potentials (16 B)
    res = r64["residual"]
    assert res["avg_ms"] == pytest.approx(5.0)
    assert res["bytes_per_dof"] == pytest.approx((24.0 * (N - n_pot) + 16.0 * n_pot) / N)
    assert res["gdof_s"] == pytest.approx(N / 5e-3 / 1e9)
    assert res["hbm_gbs"] == pytest.approx((24.0 * N - 8.0 * n_pot) / 5e-3 / 1e9)
    assert res["hbm_frac"] == pytest.approx(res["hbm_gbs"] / hbm)
    # product: z, v, J v at 8 B each in FP64, 4 B each in FP32
    assert r64["jvp"]["bytes_per_dof"] == 24.0
    assert r64["jvp"]["hbm_gbs"] == pytest.approx(24.0 * N / 1.5e-3 / 1e9)
    r32 = bench.kernel_rates(prof, N, n_pot, hbm, "mixed")
    assert r32["jvp"]["bytes_per_dof"] == 12.0
    assert r32["jvp"]["hbm_frac"] == pytest.approx(r64["jvp"]["hbm_frac"] / 2)
    # a category without calls is left out, not divided by zero
    assert "jvp" not in bench.kernel_rates({"residual": (1.0, 1), "jvp": (0.0, 0)}, N, n_pot, hbm, "fp64")


def test_clock_summary_reports_median_max_and_active_reasons(bench):
    cs = bench.ClockSampler(0)
    assert cs.summary()["reasons"] == ["unsampled"]
    not_active = "Not Active"
    cs.rows = [["2070", "2070", "900.1", not_active, not_active, not_active, not_active],
               ["1965", "2070", "1390.0", not_active, not_active, not_active, "Active"],
               ["2070", "2070", "1200.0", not_active, not_active, not_active, not_active],
               ["[N/A]", "[N/A]", "[N/A]", not_active, not_active, not_active, not_active]]
    s = cs.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 4
    assert s["reasons"] == ["sw_power_cap"]
    cs.rows.append(["1100", "2070", "1000", "Active", not_active, "Active", not_active])
    assert cs.summary()["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]


def test_batched_workload_is_seeded_and_in_range(bench):
    a, b = bench.batch_specs(64), bench.batch_specs(64)
    assert a == b
    sides = np.array([s["side"] for s in a])
    assert sides.min() >= 24 and sides.max() <= 96
    assert all(0.4 <= s["porosity"] <= 0.8 and 2.0 <= s["corr"] <= 8.0 for s in a)
    assert all(0.1 <= s["f_C"] <= 2.0 for s in a)
    assert [s["order"] for s in a].count(1) == 32          # DG0 / DG1 at 50/50
    assert len({s["seed"] for s in a}) == 64
    assert bench.batch_specs(64, seed=12) != a

"""Host logic of bench.py's roofline (no GPU): algorithmic work per backup
for each kernel family, the byte width of FP64 stored rows, and the choice
between the HBM, lane-load and FP64 FMA ceilings."""
import os
import sys
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
import workloads as W  # noqa: E402


def _args(workload, tmode, prec, v_store="native"):
    return SimpleNamespace(workload=workload, tmode=tmode, prec=prec, v_store=v_store)


def _info(n, window, nu_runs=0, span=0, kernel=0, wsum=None):
    slots = 1
    for wd in window:
        slots *= wd
    return {"n": n, "window": list(window), "window_slots": slots, "window_sum": wsum or sum(window),
            "backup_kernel": kernel, "input_runs": nu_runs, "inner_span": span}


LANES = {"shared": 9.6e12, "global_l1": 8.8e12}


def test_stored_full_fp64_counts_eight_bytes_per_mass(monkeypatch):
    monkeypatch.setattr(bench, "peaks", lambda: {"hbm_gbs": 6790.0, "source": "test"})
    w = W.robot_lin()
    nx, nu = w.problem.n_states, w.problem.n_inputs
    info = _info(2, [41, 41], kernel=6)
    r = bench.roofline(_args("robot", "stored_full", "fp64"), w, info, 1.0, nx, dict(LANES))
    per_pair = 8 * 41 * 41 + 2 * 2
    per_state = 8 + 8 + 2 + 1
    assert r["bound"] == "hbm"
    assert r["algorithmic_bytes_per_launch"] == nx * nu * per_pair + nx * per_state
    r32 = bench.roofline(_args("robot", "stored_full", "fp32"), w, info, 1.0, nx, dict(LANES))
    assert r32["algorithmic_bytes_per_launch"] == nx * nu * (4 * 41 * 41 + 4) + nx * (4 + 4 + 2 + 1)


def test_fp64_takes_the_closer_ceiling(monkeypatch):
    monkeypatch.setattr(bench, "peaks", lambda: {"hbm_gbs": 6790.0, "source": "test"})
    w = W.robot_lin()
    nx, nu = w.problem.n_states, w.problem.n_inputs
    info = _info(2, [41, 41], kernel=6)
    fmas = nx * nu * 41 * 41
    lanes = dict(LANES, fma_fp64=0.62e12)
    # FMA-bound: the FP64 rate is reached first
    r = bench.roofline(_args("robot", "stored_full", "fp64"), w, info, 0.3, nx, lanes)
    ach = fmas / 0.3e-3 / 1e12
    hbm_frac = (nx * nu * (8 * 41 * 41 + 4) + nx * 19) / 0.3e-3 / 1e9 / 6790.0
    assert r["algorithmic_fmas_per_backup"] == fmas
    if ach / 0.62 > hbm_frac:
        assert r["bound"] == "alu" and r["other_ceiling"]["bound"] == "hbm"
    else:
        assert r["bound"] == "hbm" and r["other_ceiling"]["bound"] == "alu"
    assert r["frac"] >= r["other_ceiling"]["frac"]
    # with a far faster FP64 unit the HBM ceiling binds instead
    r2 = bench.roofline(_args("robot", "stored_full", "fp64"), w, info, 0.3, nx, dict(LANES, fma_fp64=1e15))
    assert r2["bound"] == "hbm" and r2["other_ceiling"]["unit"].startswith("T FMA/s")


def test_per_run_kernel_counts_run_contractions(monkeypatch):
    monkeypatch.setattr(bench, "peaks", lambda: {"hbm_gbs": 6790.0, "source": "test"})
    monkeypatch.setattr(bench, "measured_traffic", lambda args, n: (None, None))
    w = W.unicycle()
    nx, nu = w.problem.n_states, w.problem.n_inputs
    free = nx - 1000
    info = _info(3, [3, 3, 3], nu_runs=5, span=4, kernel=5)
    r = bench.roofline(_args("unicycle", "stored_separable", "fp32"), w, info, 0.008, free, dict(LANES))
    assert r["bound"] == "alu" and r["unit"] == "G lane-loads/s"
    assert r["algorithmic_lane_loads_per_backup"] == free * 5 * 4 * 3 ** 2 + free * nu * 3
    assert r["peak"] == pytest.approx(9.6e3)
    gather = free * nu * 27
    assert r["window_slot_rate_vs_gather_ceiling"] == pytest.approx(gather / 0.008e-3 / 1e9 / 9.6e3)


def test_gather_kernels_use_their_load_path(monkeypatch):
    monkeypatch.setattr(bench, "peaks", lambda: {"hbm_gbs": 6790.0, "source": "test"})
    monkeypatch.setattr(bench, "measured_traffic", lambda args, n: (None, None))
    w = W.traffic6(n_per_dim=5, horizon=2)
    nx = w.problem.n_states
    info = _info(6, [5] * 6, kernel=1)
    r = bench.roofline(_args("traffic6", "stored_separable", "fp32_kahan"), w, info, 1.0, nx, dict(LANES))
    assert "global_l1" in r["peak_source"] and r["algorithmic_lane_loads_per_backup"] == nx * 4 * 5 ** 6
    info2 = _info(2, [3, 3], kernel=2)
    r2 = bench.roofline(_args("unicycle", "stored_separable", "fp32"), w, info2, 1.0, nx, dict(LANES))
    assert "shared" in r2["peak_source"]


def test_plane_kernel_roofline_from_counted_work(monkeypatch):
    """Kernel 7: stage-1 V values (4 bytes each, through L2), stage-2 box loads
    (shared lane-loads) and FP32 FMAs (one per value read plus W + 1 per
    second-stage row), each against its measured ceiling; the highest
    fraction is the bound, the other two are listed beside it."""
    monkeypatch.setattr(bench, "measured_traffic", lambda args, n: (None, None))
    w = W.traffic6()
    info = _info(6, [5] * 6, kernel=7)
    work = {"v_loads": 4_000_000_000, "box_loads": 30_000_000_000, "box_rows": 1_200_000_000}
    lanes = dict(LANES, fma_fp32=40e12, l2_bytes=20e12)
    r = bench.roofline(_args("traffic6", "stored_separable", "fp32_kahan"), w, info, 100.0, 0, lanes, work)
    l2 = 4e9 * 4 / 0.1 / 1e9 / 20e3
    sh = 30e9 / 0.1 / 1e9 / 9.6e3
    fma = (4e9 + 30e9 + 1.2e9 * 6) / 0.1 / 1e12 / 40.0
    fr = {"l2": l2, "shared": sh, "fma": fma}
    assert r["frac"] == pytest.approx(max(fr.values()))
    assert len(r["other_ceilings"]) == 2
    assert r["frac"] >= max(c["frac"] for c in r["other_ceilings"])
    assert r["nominal_window_slots_per_backup"] == w.problem.n_states * 4 * 5 ** 6
    r16 = bench.roofline(_args("traffic6", "stored_separable", "fp32", "bf16"), w, info, 100.0, 0, lanes, work)
    l2c = [c for c in [r16] + r16["other_ceilings"] if c["bound"] == "l2"][0]
    assert l2c["achieved"] == pytest.approx(4e9 * 2 / 0.1 / 1e9)


def test_on_the_fly_counts_erfc_edges(monkeypatch):
    """Rows on the fly: sum_i (W_i + 1) erfc edge values per (free state,
    input) pair against the measured erfc rate; the closest ceiling binds."""
    monkeypatch.setattr(bench, "peaks", lambda: {"hbm_gbs": 6790.0, "source": "test"})
    w = W.robot_lin()
    nx, nu = w.problem.n_states, w.problem.n_inputs
    info = _info(2, [41, 41], kernel=6)
    evals = nx * nu * (41 + 1 + 41 + 1)
    slow = dict(LANES, fma_fp64=0.62e12, erfc_fp64=1e9)
    r = bench.roofline(_args("robot", "otf", "fp64"), w, info, 2.0, nx, slow)
    assert r["unit"] == "G erfc/s (FP64)" and r["algorithmic_erfc_per_backup"] == evals
    assert r["achieved"] == pytest.approx(evals / 2.0e-3 / 1e9)
    assert len(r["other_ceilings"]) == 2 and r["frac"] >= max(c["frac"] for c in r["other_ceilings"])
    fast = dict(LANES, fma_fp64=0.62e12, erfc_fp64=1e15)
    r2 = bench.roofline(_args("robot", "otf", "fp64"), w, info, 2.0, nx, fast)
    assert not r2["unit"].startswith("G erfc") and r2["other_ceilings"][-1]["unit"] == "G erfc/s (FP64)"
    r32 = bench.roofline(_args("robot", "otf", "fp32"), w, info, 0.1, nx, dict(LANES, fma_fp32=38e12, erfc_fp32=1e9))
    assert r32["unit"] == "G erfc/s (FP32)"
    # stored rows and non-Gaussian noise take no erfc ceiling
    r3 = bench.roofline(_args("robot", "stored_full", "fp64"), w, info, 2.0, nx, slow)
    assert "other_ceilings" not in r3

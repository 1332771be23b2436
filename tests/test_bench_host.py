"""Host-side arithmetic of bench.py's roofline records (no GPU): the algorithmic
byte and operation counts the bench line reports are the ones its docstrings
state, so a figure in a committed bench line can be recomputed by hand."""
import pytest

import bench


def test_hbm_roofline_counts():
    info = {"force_path": 0, "threads_per_particle": 1, "force_block": 128}
    r = bench.hbm_roofline(1_000_000, 92.0, "mixed", 0.2, 0.4, info, "ka1m")
    assert r["alg_bytes_per_launch"] == 1_000_000 * (148 + 4 * 92)
    assert r["k5_only"]["alg_bytes_per_launch"] == 1_000_000 * (36 + 4 * 92)
    assert r["achieved"] == pytest.approx(516e6 / 0.2e-3 / 1e9, rel=1e-6)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-3)
    assert r["force_share_of_step"] == pytest.approx(0.5)
    r64 = bench.hbm_roofline(64_000, 80.0, "fp64", 0.3, 0.3, info, "lj64k")
    assert r64["alg_bytes_per_launch"] == 64_000 * (196 + 4 * 80)


def test_fp64_roofline_counts():
    peaks = {"dfma": {"ops_per_s": 5e11}, "drcp_in_dfma_slots": 6.0}
    r = bench.fp64_roofline(64_000, 80.0, 0.25, peaks, 2.5, 2.9)
    f_cut = (2.5 / 2.9) ** 3
    per_pair = f_cut * (14 + 6.0)
    assert r["ops_per_listed_pair"] == pytest.approx(per_pair, abs=0.01)
    ops = 64_000 * (80.0 * per_pair + 13)
    assert r["ops_per_launch"] == int(ops)
    assert r["frac"] == pytest.approx(ops / 0.25e-3 / 5e11, rel=1e-3)
    assert r["bound"] == "fp64"

"""gbmd_get_thermo_noalloc gives what gbmd_get_thermo gives.

The allocation-free readout is for callers that must not allocate GPU memory:
programs whose memory manager has already reserved the device's memory, and
code that runs while CUDA work is captured in a mode where cudaMalloc is an
error.  It keeps its scratch (per-tile partial sums and a descriptor copy) in
static device arrays shared by every call, so the checks below call it twice in
a row on one system, then on a second system of another size and type count,
then again after more steps, and compare each result with the allocating entry
point, within the tolerances of the parity tests.  It also checks the size
limit.  This file is collected last on purpose.
"""
import math

import numpy as np
import pytest

from paper_1308_5587_gb300 import gbmd, workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1308_5587_gb300 import _build
    _build.build()


def _same(a, b, prec):
    rel = 1e-12 if prec == "fp64" else 2e-6
    assert a["step"] == b["step"]
    assert a["n_rebuilds"] == b["n_rebuilds"]
    for k in ("pe", "ke", "temperature", "pressure", "w"):
        assert math.isclose(a[k], b[k], rel_tol=rel, abs_tol=1e-12), k
    va, vb = np.array(a["virial"]), np.array(b["virial"])
    assert np.allclose(va, vb, rtol=rel, atol=rel * np.abs(vb).max())


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_thermo_matches_allocating_thermo(prec):
    w1 = wl.lj_fluid(3000, 0.84, 1.2, seed=501)
    w2 = wl.lj_fluid(2000, 1.2, 1.0, seed=502, binary=True, r_buff=0.3)
    s1 = gbmd.System.from_workload(w1, precision=prec)
    s2 = gbmd.System.from_workload(w2, precision=prec)
    s1.step(40)
    s2.step(25)
    ref1 = gbmd.gbmd_get_thermo(s1.handle)
    ref2 = gbmd.gbmd_get_thermo(s2.handle)
    first = gbmd.gbmd_get_thermo_noalloc(s1.handle)
    second = gbmd.gbmd_get_thermo_noalloc(s1.handle)      # two calls in a row
    _same(first, ref1, prec)
    _same(second, ref1, prec)
    other = gbmd.gbmd_get_thermo_noalloc(s2.handle)       # shared scratch, other system
    _same(other, ref2, prec)
    s1.step(15)
    again = gbmd.gbmd_get_thermo_noalloc(s1.handle)
    _same(again, gbmd.gbmd_get_thermo(s1.handle), prec)
    assert again["step"] == 55
    s1.close()
    s2.close()


def test_noalloc_thermo_rejects_systems_over_the_limit():
    # global force path: 128 particles per energy tile, so 4,194,304 particles at most
    w = wl.lj_fluid(4_200_000, 0.84, 1.2, seed=503)
    s = gbmd.System.from_workload(w, precision="mixed", force_path="global")
    with pytest.raises(gbmd.GbmdError) as e:
        gbmd.gbmd_get_thermo_noalloc(s.handle)
    assert e.value.status == "BAD_ARG"
    assert "allocation-free limit" in str(e.value)
    t = gbmd.gbmd_get_thermo(s.handle)          # the allocating readout still works
    assert math.isfinite(t["pe"]) and t["pe"] < 0
    s.close()


def test_noalloc_thermo_does_not_depend_on_the_force_tuning():
    # the energy launch has its own fixed tiles: the FP64 sums are bitwise the same
    # for every block size at one threads-per-particle setting
    w = wl.lj_fluid(5000, 0.84, 1.2, seed=504)
    s = gbmd.System.from_workload(w, precision="fp64")
    s.step(10)
    ref = gbmd.gbmd_get_thermo_noalloc(s.handle)
    for block in (64, 128, 256, 512):
        s.set_tuning(2, block)
        t = gbmd.gbmd_get_thermo_noalloc(s.handle)
        assert t["pe"] == ref["pe"] and t["virial"] == ref["virial"]
        t2 = gbmd.gbmd_get_thermo(s.handle)
        assert t2["pe"] == ref["pe"]
    s.close()

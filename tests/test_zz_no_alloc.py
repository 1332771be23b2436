"""gbmd_get_thermo_noalloc gives what gbmd_get_thermo gives.

The allocation-free readout is for callers that must not allocate GPU memory:
programs whose memory manager has already reserved the device's memory, and
code that runs while CUDA work is captured in a mode where cudaMalloc is an
error.  It keeps its scratch (per-tile partial sums and a descriptor copy) in
static device arrays shared by every call, so the checks below call it twice in
a row on one system, then on a second system of another size and type count,
then again after more steps, and compare each result with the allocating entry
point.  Both run the same kernels over the same fixed energy tiles and sum in
the same order, so the two readouts must agree exactly, on the global and the
staged force path and on the tree neighbour list alike.  It also checks the size
limit and the refusal to run while a neighbour-list overflow is still pending
(recovering from one grows the list, which allocates).  This file is collected
last on purpose.
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


def _same(a, b):
    # same kernels, same tiles, same order: equal to the last bit
    assert a["step"] == b["step"]
    assert a["n_rebuilds"] == b["n_rebuilds"]
    for k in ("pe", "ke", "temperature", "pressure", "w"):
        assert a[k] == b[k], (k, a[k], b[k])
    assert list(a["virial"]) == list(b["virial"])
    assert math.isfinite(a["pe"])


CASES = [("fp64", "global", "cell"), ("mixed", "global", "cell"), ("mixed", "staged", "cell"),
         ("fp64", "global", "tree"), ("mixed", "global", "tree")]


@pytest.mark.parametrize("prec,path,nlist", CASES)
def test_noalloc_thermo_matches_allocating_thermo(prec, path, nlist):
    w1 = wl.lj_fluid(3000, 0.84, 1.2, seed=501)
    w2 = wl.lj_fluid(2000, 1.2, 1.0, seed=502, binary=True, r_buff=0.3)
    if path == "staged":   # at least 4 cells per axis, windows well inside shared memory
        w1 = wl.lj_fluid(6000, 0.84, 1.2, seed=501)
        w2 = wl.lj_fluid(4000, 1.2, 1.0, seed=502, binary=True, r_buff=0.3)
    s1 = gbmd.System.from_workload(w1, precision=prec, force_path=path, nlist=nlist)
    s2 = gbmd.System.from_workload(w2, precision=prec, force_path=path, nlist=nlist)
    if path == "staged":
        assert s1.info()["force_path"] == 1 and s2.info()["force_path"] == 1
    s1.step(40)
    s2.step(25)
    ref1 = gbmd.gbmd_get_thermo(s1.handle)
    ref2 = gbmd.gbmd_get_thermo(s2.handle)
    first = gbmd.gbmd_get_thermo_noalloc(s1.handle)
    second = gbmd.gbmd_get_thermo_noalloc(s1.handle)      # two calls in a row
    _same(first, ref1)
    _same(second, ref1)
    other = gbmd.gbmd_get_thermo_noalloc(s2.handle)       # shared scratch, other system
    _same(other, ref2)
    s1.step(15)
    again = gbmd.gbmd_get_thermo_noalloc(s1.handle)
    _same(again, gbmd.gbmd_get_thermo(s1.handle))
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
    s.set_tuning(2, 128)   # the reference at the lane count every block size below uses
    s.step(10)
    ref = gbmd.gbmd_get_thermo_noalloc(s.handle)
    for block in (64, 128, 256, 512):
        s.set_tuning(2, block)
        t = gbmd.gbmd_get_thermo_noalloc(s.handle)
        assert t["pe"] == ref["pe"] and t["virial"] == ref["virial"]
        t2 = gbmd.gbmd_get_thermo(s.handle)
        assert t2["pe"] == ref["pe"]
    s.close()


def test_noalloc_thermo_refuses_a_pending_overflow_then_matches_after_sync():
    # a dilute lattice gas flowing inward: neighbour counts outgrow the initial
    # capacity mid-run, which freezes the system until the host grows the list
    g = (np.arange(12) - 5.5) * 1.5
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    box = np.full(3, 18.0)
    vel = -0.6 * pos / 9.0
    roomy = gbmd.System(pos, vel, box, precision="mixed", nlist_capacity=400)
    c0 = int(roomy.neighbors(cap=400)[0].max())
    roomy.close()
    tight = gbmd.System(pos, vel, box, precision="mixed", nlist_capacity=c0)
    tight.step(400)                          # enqueued; the overflow happens on the device
    with pytest.raises(gbmd.GbmdError) as e:
        gbmd.gbmd_get_thermo_noalloc(tight.handle)
    assert e.value.status == "STATE"
    tight.sync()                             # grows the list and finishes the steps
    assert tight.info()["nlist_capacity"] > c0
    t = gbmd.gbmd_get_thermo_noalloc(tight.handle)
    assert t["step"] == 400
    _same(t, gbmd.gbmd_get_thermo(tight.handle))
    tight.close()

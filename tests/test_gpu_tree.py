"""The tree neighbour list (gbmd_desc.nlist = GBMD_NLIST_TREE) on the GPU, through the
C ABI: the same neighbour set as the definition (brute force in the oracle) for
one-type, two-type and size-disperse systems, forces and trajectories against the
oracle, batches mixing tree and cell lists, overflow recovery and edge sizes.

Tolerances as for the cell list: neighbour sets identical outside a 1e-9 band of
r_list; FP64 forces 1e-12 relative; mixed 1e-5 relative L2; FP64 trajectories 1e-9
over 100 steps.  The tree lists a particle's neighbours in another order than the
cell list, so FP32 sums may differ in the last bits between the two lists, never
beyond these bounds.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1308_5587_gb300 import gbmd, workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    from paper_1308_5587_gb300 import _build
    _build.build()
    oracle.build()
    oracle.set_threads(os.cpu_count() or 1)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def check_neighbors(s, w):
    pos = s.state()[0]
    counts, idx = s.neighbors(cap=int(s.info()["nlist_capacity"]) + 8)
    rl = oracle.cutoffs(w.pairs.as_dict()) + w.r_buff
    pairs, r = oracle.neighbors(pos, w.box, w.types, rl)
    ok = np.abs(r - rl[w.types[pairs[:, 0]], w.types[pairs[:, 1]]]) > 1e-9
    ref = {(int(a), int(b)) for a, b in pairs[ok]}
    band = {(int(a), int(b)) for a, b in pairs[~ok]}
    mine = set()
    for i in range(w.n):
        row = idx[i, :counts[i]]
        assert np.all(np.diff(row) > 0)   # no duplicates
        mine.update((min(i, int(j)), max(i, int(j))) for j in row)
    assert ref <= mine, len(ref - mine)
    assert mine - ref <= band
    return len(ref)


def check_verlet(s, w):
    """Between builds: the list was built at earlier positions, and no particle has
    moved r_buff/2 since, so it holds every pair now within r_cut and none now
    beyond r_list + r_buff."""
    pos = s.state()[0]
    counts, idx = s.neighbors(cap=int(s.info()["nlist_capacity"]) + 8)
    rc = oracle.cutoffs(w.pairs.as_dict())
    pairs, r = oracle.neighbors(pos, w.box, w.types, rc)
    inner = r < rc[w.types[pairs[:, 0]], w.types[pairs[:, 1]]] - 1e-9
    must = {(int(a), int(b)) for a, b in pairs[inner]}
    pairs, r = oracle.neighbors(pos, w.box, w.types, rc + 2 * w.r_buff + 1e-9)
    may = {(int(a), int(b)) for a, b in pairs}
    mine = set()
    for i in range(w.n):
        mine.update((min(i, int(j)), max(i, int(j))) for j in idx[i, :counts[i]])
    assert must <= mine, len(must - mine)
    assert mine <= may


def check_forces(s, w, prec):
    pos = s.state()[0]
    F = s.forces()
    Fo, Uo, Wo, _, _ = oracle.forces(pos, w.box, w.types, w.pairs.as_dict())
    th = s.thermo()
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert rel_l2(F, Fo) <= tol
    assert th["pe"] == pytest.approx(Uo, rel=tol if prec == "fp64" else 1e-5)
    assert np.allclose(th["virial"], Wo, rtol=tol, atol=tol * np.abs(Wo).max())


WORKLOADS = {
    "lj1500": lambda: wl.lj_fluid(1500, 0.84, 1.2, seed=91),
    "ka1200": lambda: wl.lj_fluid(1200, 1.2, 1.0, seed=92, binary=True, r_buff=0.3),
    "lj256_small_box": lambda: wl.lj_fluid(256, 0.9, 1.2, seed=93),
    "colloid_1to5": lambda: wl.colloid_mixture(3000, ratio=5.0, seed=94),
    "colloid_1to3": lambda: wl.colloid_mixture(4000, ratio=3.0, seed=95),
}


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("case", list(WORKLOADS))
def test_tree_neighbor_sets_and_forces(case, prec):
    w = WORKLOADS[case]()
    s = gbmd.System.from_workload(w, precision=prec, nlist="tree")
    assert s.info()["nlist"] == gbmd.GBMD_NLIST_TREE
    assert s.info()["force_path"] == 0
    check_neighbors(s, w)
    check_forces(s, w, prec)
    s.step(150)   # rebuilds at the GPU's own positions (no re-sort: cell order changes)
    assert s.info()["n_rebuilds"] >= 1
    check_verlet(s, w)
    check_forces(s, w, prec)
    pos, vel, img, step = s.state()   # a rebuild at these positions, then the exact set
    s.set_state(pos, vel, img, step)
    check_neighbors(s, w)
    s.close()


@pytest.mark.parametrize("case", ["ka1200", "colloid_1to5"])
def test_tree_fp64_trajectory_matches_the_oracle(case):
    w = WORKLOADS[case]()
    o = oracle.vv_run(w.pos, w.vel, w.box, w.types, w.pairs.as_dict(), w.mass, w.dt, 100)
    s = gbmd.System.from_workload(w, precision="fp64", nlist="tree", sort_period=40)
    s.step(100)
    pos, vel, img, step = s.state()
    assert step == 100
    assert np.abs(pos + img * w.box - (o["pos"] + o["image"] * w.box)).max() <= 1e-9
    assert np.abs(vel - o["vel"]).max() <= 1e-8
    s.close()


def test_tree_and_cell_lists_step_alike():
    """Mixed precision: the two lists differ only in each row's order."""
    w = WORKLOADS["colloid_1to3"]()
    out = []
    for nl in ("cell", "tree"):
        s = gbmd.System.from_workload(w, precision="mixed", nlist=nl, sort_period=50)
        s.step(200)
        out.append((s.state(), s.thermo(), s.info()))
        s.close()
    (a, ta, ia), (b, tb, ib) = out
    assert ta["step"] == tb["step"] == 200
    assert abs(ia["n_rebuilds"] - ib["n_rebuilds"]) <= 1   # the same trajectory to ~1e-6
    assert np.abs(a[0] + a[2] * w.box - b[0] - b[2] * w.box).max() < 1e-3
    assert ta["pe"] == pytest.approx(tb["pe"], rel=1e-4)


def test_batch_mixing_tree_and_cell_members_matches_alone():
    ws = [WORKLOADS["colloid_1to5"](), wl.lj_fluid(2000, 0.84, 1.2, seed=96),
          wl.colloid_mixture(2000, ratio=4.0, seed=97)]
    kinds = ["tree", "cell", "tree"]
    ws[1].pairs = wl.wca_single()   # one evaluator for the batch (WCA)
    alone = []
    for w, nl in zip(ws, kinds):
        s = gbmd.System.from_workload(w, precision="mixed", nlist=nl)
        s.set_tuning(2, 128)
        s.step(80)
        alone.append((s.state(), s.thermo()))
        s.close()
    b = gbmd.Batch("mixed")
    b.set_tuning(2, 128)
    ss = [gbmd.System.from_workload(w, precision="mixed", nlist=nl) for w, nl in zip(ws, kinds)]
    for s in ss:
        b.add(s)
    b.step(80)
    b.sync()
    for s, (st, th) in zip(ss, alone):
        st2 = s.state()
        for x, y in zip(st2[:3], st[:3]):
            assert np.array_equal(x, y)
        assert s.thermo()["pe"] == th["pe"]
    b.close()
    for s in ss:
        s.close()


def test_tree_overflow_is_recovered_bitwise():
    w = WORKLOADS["colloid_1to5"]()
    ref = gbmd.System.from_workload(w, precision="mixed", nlist="tree")
    ref.step(60)
    small = gbmd.System.from_workload(w, precision="mixed", nlist="tree", nlist_capacity=8)
    small.step(60)
    for x, y in zip(small.state()[:3], ref.state()[:3]):
        assert np.array_equal(x, y)
    assert small.info()["nlist_capacity"] > 8
    ref.close()
    small.close()


@pytest.mark.parametrize("n", [1, 3, 17])
def test_tree_tiny_systems_and_empty_types(n):
    w = wl.lj_fluid(n, 0.05, 1.0, seed=98)
    w.box = np.maximum(w.box, 6.0)
    w.pos = w.pos * 0.5
    # two types, the second one empty: a tree of one empty leaf
    p = wl.PairTable(np.ones((2, 2)), np.ones((2, 2)), np.full((2, 2), 2.5))
    s = gbmd.System(w.pos, w.vel, w.box, np.zeros(n, np.int32), p.eps, p.sigma, p.rcut,
                    precision="fp64", nlist="tree")
    s.step(20)
    pos = s.state()[0]
    F = s.forces()
    Fo, *_ = oracle.forces(pos, w.box, np.zeros(n, np.int32), p.as_dict())
    assert np.allclose(F, Fo, rtol=1e-12, atol=1e-12)
    s.close()


def test_tree_with_nvt():
    w = WORKLOADS["colloid_1to3"]()
    s = gbmd.System.from_workload(w, precision="mixed", nlist="tree", integrator="nvt",
                                  kT=1.0, tau=0.5)
    s.step(200)
    th = s.thermo()
    assert th["step"] == 200 and np.isfinite(th["h_ext"])
    check_verlet(s, w)
    check_forces(s, w, "mixed")
    s.close()


def test_tree_autotune_and_cell_scale_keep_results():
    """The autotuner's cell-width sweep regrids the tree list's sort cells (type-major
    bins); the lists and forces stay those of the definition."""
    w = WORKLOADS["colloid_1to3"]()
    s = gbmd.System.from_workload(w, precision="mixed", nlist="tree")
    s.step(20)
    s.autotune(None)
    info = s.info()
    assert info["nlist"] == gbmd.GBMD_NLIST_TREE
    assert info["cell_scale"] in (1.0, 1.1, 1.2, 1.35)
    s.step(20)
    check_verlet(s, w)
    check_forces(s, w, "mixed")
    s.set_cell_scale(1.35)
    s.set_state(*s.state())   # a rebuild at the current positions, then the exact set
    check_neighbors(s, w)
    check_forces(s, w, "mixed")
    s.close()

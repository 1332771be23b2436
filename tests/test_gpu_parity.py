"""CUDA path vs the FP64 CPU oracle, element by element, through the C ABI.

Tolerances (from the arithmetic; global relative L2 = ||F_gpu - F_ref|| / ||F_ref||):
* FP64 forces, energy, virial: <= 1e-12 relative (every operation is FP64; the only
  differences are summation order and fused multiply-adds, ~1e-15 per pair);
* mixed forces: <= 1e-5 relative L2 (FP32 pair arithmetic, ~1e-7 per operation,
  summed over ~55 pairs with cancellation); per particle <= 1e-4 F_rms;
* neighbour sets: identical, excluding pairs within 1e-9 sigma of r_list;
* trajectories (FP64): <= 1e-9 sigma over 100 steps.
Particles with a pair within a band of r_cut are left out of per-particle maxima
(a pair exactly at the cut may be decided either way by different rounding).
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


def mi(d, box):
    return d - box * np.rint(d / box)


def near_cut(pos, box, types, rcut, band):
    """Particles with some pair within `band` of its r_cut."""
    rl = np.asarray(rcut, np.float64)
    pairs, r = oracle.neighbors(pos, box, types, rl + band)
    rc = rl[types[pairs[:, 0]], types[pairs[:, 1]]]
    hit = pairs[np.abs(r - rc) < band]
    return np.unique(hit.ravel())


def check_forces(sysm, w, prec, where=""):
    pos, vel, img, step = sysm.state()
    F = sysm.forces()
    p = w.pairs.as_dict()
    Fo, Uo, Wo, uo, Wio = oracle.forces(pos, w.box, w.types, p)
    err = rel_l2(F, Fo)
    frms = np.sqrt(np.mean(Fo ** 2))
    band = 1e-9 if prec == "fp64" else 1e-5
    skip = near_cut(pos, w.box, w.types, w.pairs.rcut, band)
    mask = np.ones(len(F), bool)
    mask[skip] = False
    dmax = np.abs(F - Fo)[mask].max() / frms
    th = sysm.thermo()
    if prec == "fp64":
        assert err <= 1e-12, (where, err)
        assert dmax <= 1e-11, (where, dmax)
        assert th["pe"] == pytest.approx(Uo, rel=1e-12), where
        assert np.allclose(th["virial"], Wo, rtol=1e-12, atol=1e-9 * np.abs(Wo).max()), where
    else:
        assert err <= 1e-5, (where, err)
        assert dmax <= 1e-4, (where, dmax)
        assert th["pe"] == pytest.approx(Uo, rel=2e-6), where
        assert np.allclose(th["virial"], Wo, rtol=2e-5, atol=2e-5 * np.abs(Wo).max()), where
    return err


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["lj1000", "lj_ragged_777", "ka2000", "ortho_small"])
def test_forces_energy_virial_at_creation(prec, case):
    if case == "lj1000":
        w = wl.lj_fluid(1000, 0.84, 1.2, seed=31)
    elif case == "lj_ragged_777":
        w = wl.lj_fluid(777, 0.84, 1.2, seed=32)
    elif case == "ka2000":
        w = wl.lj_fluid(2000, 1.2, 1.0, seed=33, binary=True, r_buff=0.3)
    else:   # orthorhombic box with 2 cells on one axis (deduplicated stencil)
        w = wl.lj_fluid(600, 0.84, 1.2, seed=34)
        w.box = np.array([w.box[0] * 0.75, w.box[1], w.box[2] / 0.75])
    s = gbmd.System.from_workload(w, precision=prec)
    check_forces(s, w, prec, case)
    u, Wi = s.per_particle()
    pos = s.state()[0]
    _, _, _, uo, Wio = oracle.forces(pos, w.box, w.types, w.pairs.as_dict())
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert np.abs(u - uo).max() <= tol * (1 + np.abs(uo).max()) * 10
    assert np.abs(Wi - Wio).max() <= tol * (1 + np.abs(Wio).max()) * 10
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_neighbor_sets_match_brute_force(prec):
    for w in (wl.lj_fluid(1500, 0.84, 1.2, seed=41),
              wl.lj_fluid(1200, 1.2, 1.0, seed=42, binary=True, r_buff=0.3),
              wl.lj_fluid(256, 0.9, 1.2, seed=43),            # 2 cells per axis
              wl.lj_fluid(5000, 0.84, 1.2, seed=44),          # 6 cells: two-cell warps
              wl.lj_fluid(5000, 1.2, 1.0, seed=45, binary=True, r_buff=0.3)):  # 5: odd
        s = gbmd.System.from_workload(w, precision=prec)
        for rnd in range(2):
            pos = s.state()[0]
            counts, idx = s.neighbors(cap=512)
            rl = w.pairs.rcut + w.r_buff
            pairs, r = oracle.neighbors(pos, w.box, w.types, rl)
            rlp = rl[w.types[pairs[:, 0]], w.types[pairs[:, 1]]]
            ok = np.abs(r - rlp) > 1e-9
            ref = {(int(a), int(b)) for a, b in pairs[ok]}
            band = {(int(a), int(b)) for a, b in pairs[~ok]}
            mine = set()
            for i in range(w.n):
                row = idx[i, :counts[i]]
                assert np.all(np.diff(row) > 0)
                for j in row:
                    mine.add((min(i, int(j)), max(i, int(j))))
            # full list: every pair appears from both sides
            assert counts.sum() == 2 * len(mine)
            assert mine - band == ref
            # move everything and rebuild through set_state
            pos2 = pos + np.random.default_rng(rnd).normal(scale=0.1, size=pos.shape)
            s.set_state(pos2, s.state()[1])
        s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_neighbor_sets_of_dense_cells_span_several_segments(prec):
    """r_buff 1.5 at rho 1.2: cells 4 sigma wide hold ~77 particles (three passes of a
    warp), about 1,200 candidates per pass survive the culling (several segments of 14
    tested chunks, appended with rows left mid slot group between segments), ~320
    neighbours per particle, and exactly 3 cells per axis (the smallest grid of the
    relative-coordinate path).  Neighbour sets equal the brute-force pairs and the
    forces match the oracle, before and after a rebuild from moved positions."""
    base = wl.lj_fluid(4000, 1.2, 1.0, seed=46)
    w = wl.Workload(base.pos, base.vel, base.types, base.box, base.pairs, r_buff=1.5)
    assert int(w.box[0] // (float(w.pairs.rcut.max()) + 1.5)) == 3
    s = gbmd.System.from_workload(w, precision=prec)
    for rnd in range(2):
        pos = s.state()[0]
        counts, idx = s.neighbors(cap=512)
        assert counts.max() < 512 and counts.mean() > 250
        rl = w.pairs.rcut + w.r_buff
        pairs, r = oracle.neighbors(pos, w.box, w.types, rl)
        rlp = rl[w.types[pairs[:, 0]], w.types[pairs[:, 1]]]
        ok = np.abs(r - rlp) > 1e-9
        ref = {(int(a), int(b)) for a, b in pairs[ok]}
        band = {(int(a), int(b)) for a, b in pairs[~ok]}
        mine = set()
        for i in range(w.n):
            row = idx[i, :counts[i]]
            assert np.all(np.diff(row) > 0)
            mine.update((min(i, int(j)), max(i, int(j))) for j in row)
        assert counts.sum() == 2 * len(mine)
        assert mine - band == ref
        F = s.forces()
        Fo, *_ = oracle.forces(pos, w.box, w.types, w.pairs.as_dict())
        assert rel_l2(F, Fo) <= (1e-12 if prec == "fp64" else 1e-5)
        pos2 = pos + np.random.default_rng(10 + rnd).normal(scale=0.1, size=pos.shape)
        s.set_state(pos2, s.state()[1])
    s.close()


def test_trajectory_plain_fp64_4000_100_steps():
    """The plain FP64 configuration: N=4,000 LJ, 100 NVE steps, vs the oracle."""
    w = wl.plain_fp64_4k()
    ref = oracle.vv_run(w.pos, w.vel, w.box, w.types, w.pairs.as_dict(), w.mass, w.dt, 100)
    s = gbmd.System.from_workload(w, precision="fp64")
    s.step(100)
    pos, vel, img, step = s.state()
    assert step == 100
    dx = np.abs(mi(pos - ref["pos"], w.box)).max()
    dv = np.abs(vel - ref["vel"]).max()
    assert dx <= 1e-9 and dv <= 1e-9, (dx, dv)
    unwrapped = pos + img * w.box
    ref_unwrapped = ref["pos"] + ref["image"] * w.box
    assert np.abs(unwrapped - ref_unwrapped).max() <= 1e-9
    assert s.info()["n_rebuilds"] >= 1
    F = s.forces()
    assert rel_l2(F, ref["force"]) <= 1e-10
    s.close()


def test_trajectory_mixed_stays_close():
    w = wl.lj_fluid(2000, 0.84, 1.2, seed=51)
    ref = oracle.vv_run(w.pos, w.vel, w.box, w.types, w.pairs.as_dict(), w.mass, w.dt, 50)
    s = gbmd.System.from_workload(w, precision="mixed")
    s.step(50)
    pos, vel, _, _ = s.state()
    assert np.abs(mi(pos - ref["pos"], w.box)).max() < 1e-5
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_overflow_is_recovered_bitwise(prec):
    w = wl.lj_fluid(3000, 0.84, 1.5, seed=61)
    big = gbmd.System.from_workload(w, precision=prec)
    counts, _ = big.neighbors(cap=512)
    tight = gbmd.System.from_workload(w, precision=prec, nlist_capacity=int(counts.max()))
    small = gbmd.System.from_workload(w, precision=prec, nlist_capacity=8)   # overflows at once
    assert small.info()["nlist_capacity"] > 8
    for s in (big, tight, small):
        s.step(300)
    a, b, c = big.state(), tight.state(), small.state()
    for k in range(3):
        assert np.array_equal(a[k], b[k]) and np.array_equal(a[k], c[k])
    assert a[3] == b[3] == c[3] == 300
    for s in (big, tight, small):
        s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_overflow_mid_run_compression(prec):
    """A dilute lattice gas flowing inward: neighbour counts grow past the initial
    capacity during stepping; the run is recovered and equals a roomy run bitwise."""
    g = (np.arange(12) - 5.5) * 1.5
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    box = np.full(3, 18.0)
    vel = -0.6 * pos / 9.0
    roomy = gbmd.System(pos, vel, box, precision=prec, nlist_capacity=400)
    c0 = int(roomy.neighbors(cap=400)[0].max())
    tight = gbmd.System(pos, vel, box, precision=prec, nlist_capacity=c0)
    roomy.step(400)
    tight.step(400)
    tight.sync()
    assert tight.info()["nlist_capacity"] > c0
    a, b = roomy.state(), tight.state()
    for k in range(4):
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k]))
    roomy.close()
    tight.close()


def test_morton_resort_changes_nothing_physical():
    w = wl.lj_fluid(4000, 0.84, 1.2, seed=71)
    a = gbmd.System.from_workload(w, precision="fp64", sort_period=0)
    b = gbmd.System.from_workload(w, precision="fp64", sort_period=10)
    a.step(100)
    b.step(100)
    assert b.info()["n_sorts"] > 1
    pa, va, ia, _ = a.state()
    pb, vb, ib, _ = b.state()
    assert np.abs(mi(pa - pb, w.box)).max() < 1e-10
    assert np.abs(va - vb).max() < 1e-10
    assert rel_l2(b.forces(), a.forces()) < 1e-12
    a.close()
    b.close()


def test_checkpoint_resume():
    w = wl.lj_fluid(2000, 0.84, 1.2, seed=81)
    a = gbmd.System.from_workload(w, precision="fp64")
    a.step(50)
    pos, vel, img, step = a.state()
    a.step(50)
    b = gbmd.System.from_workload(w, precision="fp64")
    b.set_state(pos, vel, img, step)
    b.step(50)
    pa, va, ia, sa = a.state()
    pb, vb, ib, sb = b.state()
    assert sa == sb == 100
    assert np.abs(mi(pa - pb, w.box)).max() < 1e-12 * 1e3
    assert np.abs(va - vb).max() < 1e-11
    a.close()
    b.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_set_state_keeps_types_and_refuses_non_finite_input(prec):
    """set_state on a binary mixture whose particles have been re-sorted (tags no
    longer equal to internal indices): the types stay with their tags, so the forces
    at the new state match the oracle's with the original types.  A NaN or inf in
    the new positions or velocities is refused (BAD_ARG) and leaves the system as it
    was: same state, same forces, and it keeps stepping."""
    w = wl.lj_fluid(3000, 1.2, 1.0, seed=82, binary=True, r_buff=0.3)
    s = gbmd.System.from_workload(w, precision=prec, sort_period=10)
    s.step(40)
    assert s.info()["n_sorts"] >= 2
    rng = np.random.default_rng(3)
    pos2 = w.pos + rng.normal(scale=0.05, size=w.pos.shape)
    vel2 = rng.normal(size=w.vel.shape)
    s.set_state(pos2, vel2, None, 7)
    pos, vel, img, step = s.state()
    assert step == 7
    assert np.abs(mi(pos - pos2, w.box)).max() < 1e-9
    F = s.forces()
    Fo, *_ = oracle.forces(pos, w.box, w.types, w.pairs.as_dict())
    assert rel_l2(F, Fo) <= (1e-12 if prec == "fp64" else 1e-5)
    before = s.state()
    for bad_pos, bad_vel in ((np.nan, 0.0), (0.0, np.inf), (-np.inf, 0.0)):
        p3, v3 = pos2.copy(), vel2.copy()
        p3[1234, 1] += bad_pos
        v3[17, 2] += bad_vel
        with pytest.raises(gbmd.GbmdError) as e:
            s.set_state(p3, v3, None, 9)
        assert e.value.status == "BAD_ARG"
        after = s.state()
        for x, y in zip(before, after):
            assert np.array_equal(np.asarray(x), np.asarray(y))
    assert np.array_equal(s.forces(), F)
    s.step(10)
    assert s.state()[3] == 17
    s.close()


def test_deterministic_reruns():
    w = wl.lj_fluid(5000, 0.84, 1.2, seed=91)
    out = []
    for _ in range(2):
        s = gbmd.System.from_workload(w, precision="mixed", sort_period=20)
        s.step(120)
        out.append(s.state() + (s.forces(),))
        s.close()
    for x, y in zip(out[0], out[1]):
        assert np.array_equal(np.asarray(x), np.asarray(y))


def test_edge_cases_one_and_two_particles_and_far_images():
    # N = 1: free flight, no forces
    box = np.full(3, 10.0)
    s = gbmd.System(np.zeros((1, 3)), np.array([[1.0, -2.0, 3.0]]), box, precision="fp64")
    s.step(1000)
    pos, vel, img, step = s.state()
    x = np.array([1.0, -2.0, 3.0]) * 1000 * 0.005
    k = np.floor((x + 5) / 10)
    assert np.allclose(pos[0], x - 10 * k, atol=1e-9) and np.array_equal(img[0], k)
    assert np.all(s.forces() == 0)
    s.close()
    # N = 2 at r = sigma across the periodic boundary: |F| = 24
    pos = np.array([[4.5, 0, 0], [-4.5, 0, 0]])
    s = gbmd.System(pos, np.zeros((2, 3)), box, precision="fp64")
    F = s.forces()
    assert F[0] == pytest.approx([-24, 0, 0], abs=1e-10)
    assert F[1] == pytest.approx([24, 0, 0], abs=1e-10)
    s.close()
    # positions given in far images: identical forces and energy
    w = wl.lj_fluid(500, 0.84, 1.2, seed=93)
    s1 = gbmd.System.from_workload(w, precision="fp64")
    shift = np.random.default_rng(0).integers(-3, 4, size=w.pos.shape)
    s2 = gbmd.System(w.pos + shift * w.box, w.vel, w.box, precision="fp64")
    assert rel_l2(s2.forces(), s1.forces()) < 1e-13
    assert np.array_equal(s2.state()[2] - s1.state()[2], shift)
    s1.close()
    s2.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_pairs_at_the_cutoff_inside_and_across_the_box(prec):
    """Two particles at r = r_cut (1 + delta), delta from -1e-5 to +1e-5, inside the
    box and across a box face.  The FP64 path rejects a pair beyond r_cut by an FP32
    test on the fixed-point shadow first, and corrects the minimum image only in
    warps where some pair crosses a face: inside r_cut the forces match the oracle
    (FP64 1e-12, mixed 1e-5), beyond it they are exactly zero.  Mixed precision
    decides the cut in FP32, so it is held to pairs 1e-5 from r_cut."""
    L = 12.0
    box = np.full(3, L)
    pairs = wl.lj_single().as_dict()
    rc = 2.5
    u = np.array([1.0, 0.3, -0.2])
    u /= np.linalg.norm(u)
    deltas = (-1e-5, -1e-6, -1e-7, -1e-9, 1e-9, 1e-7, 1e-6, 1e-5) if prec == "fp64" else (-1e-5, 1e-5)
    for delta in deltas:
        r = rc * (1.0 + delta)
        for across in (False, True):
            p0 = np.array([L / 2 - 0.4, 0.1, -0.2]) if across else np.array([-1.0, 0.5, 0.3])
            pos = np.stack([p0, p0 + r * u])
            s = gbmd.System(pos, np.zeros((2, 3)), box, precision=prec)
            p = s.state()[0]
            F = s.forces()
            Fo, *_ = oracle.forces(p, box, np.zeros(2, np.int32), pairs)
            if delta > 0:
                assert np.all(F == 0) and np.all(Fo == 0), (delta, across)
            else:
                tol = 1e-12 if prec == "fp64" else 1e-5
                assert rel_l2(F, Fo) <= tol, (delta, across, F, Fo)
            s.close()


def test_fp64_kob_andersen_at_the_one_lane_default():
    """FP64 from 32k particles runs one lane per particle in 64-thread blocks, with
    the two-type table of the FP32 pre-test and the FP64 coefficients in shared
    memory: a 40,000-particle Kob-Andersen mixture, sampled particles against the
    oracle at 1e-12, at creation and after 50 steps with rebuilds."""
    w = wl.lj_fluid(40_000, 1.2, 1.0, seed=47, binary=True, r_buff=0.3)
    s = gbmd.System.from_workload(w, precision="fp64")
    info = s.info()
    assert info["threads_per_particle"] == 1 and info["force_block"] == 64
    idx = np.random.default_rng(6).choice(w.n, 768, replace=False)
    for nsteps in (0, 50):
        s.step(nsteps)
        pos = s.state()[0]
        F = s.forces()
        Fo, *_ = oracle.forces_subset(pos, w.box, w.types, w.pairs.as_dict(), idx)
        assert rel_l2(F[idx], Fo) <= 1e-12, nsteps
    assert s.info()["n_rebuilds"] >= 1
    s.close()


def test_step_limit_and_async_steps():
    w = wl.lj_fluid(1000, 0.84, 1.2, seed=95)
    s = gbmd.System.from_workload(w, precision="mixed")
    s.set_step_limit(30)
    s.step(100)
    assert s.state()[3] == 30
    s.set_step_limit(-1)
    s.step(5)
    assert s.state()[3] == 105 or s.state()[3] == 35
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_alone_equals_in_mix(prec):
    params = wl.replica_params(6, seed=123, n_lo=300, n_hi=3000)
    ws = [wl.replica(*p) for p in params]
    alone = []
    for w in ws:
        s = gbmd.System.from_workload(w, precision=prec)
        s.set_tuning(2, 256)
        s.step(60)
        alone.append((s.state(), s.forces(), s.thermo()))
        s.close()
    b = gbmd.Batch(prec)
    b.set_tuning(2, 256)
    sys_ = [gbmd.System.from_workload(w, precision=prec) for w in ws]
    for s in sys_:
        b.add(s)
    b.step(60)
    b.sync()
    assert b.info()["members"] == len(ws)
    for s, (st, F, th) in zip(sys_, alone):
        st2 = s.state()
        for k in range(4):
            assert np.array_equal(np.asarray(st2[k]), np.asarray(st[k]))
        assert np.array_equal(s.forces(), F)
        assert s.thermo()["pe"] == th["pe"]
    b.close()
    for s in sys_:
        s.close()


def test_sampled_forces_full_size_lj64k():
    """The 64,000-particle LJ fluid, both precisions, sampled particles vs the oracle."""
    w = wl.lj_64k()
    idx = np.random.default_rng(5).choice(w.n, 1024, replace=False)
    for prec, tol in (("fp64", 1e-12), ("mixed", 1e-5)):
        s = gbmd.System.from_workload(w, precision=prec, sort_period=100)
        s.step(150)
        pos = s.state()[0]
        F = s.forces()
        Fo, uo, Wo = oracle.forces_subset(pos, w.box, w.types, w.pairs.as_dict(), idx)
        assert rel_l2(F[idx], Fo) <= tol, prec
        tot = np.abs(F).sum()
        assert np.linalg.norm(F.sum(0)) <= (1e-10 if prec == "fp64" else 1e-5) * tot
        s.close()


@pytest.mark.slow
def test_sampled_forces_full_size_ka_1m():
    """Kob-Andersen N=10^6, mixed, Morton re-sort every 100 steps, sampled vs the oracle."""
    w = wl.ka_1m()
    s = gbmd.System.from_workload(w, precision="mixed", sort_period=100)
    s.step(200)
    pos = s.state()[0]
    F = s.forces()
    idx = np.random.default_rng(6).choice(w.n, 256, replace=False)
    Fo, uo, Wo = oracle.forces_subset(pos, w.box, w.types, w.pairs.as_dict(), idx)
    assert rel_l2(F[idx], Fo) <= 1e-5
    info = s.info()
    assert info["n_sorts"] >= 2 and info["step"] == 200
    assert np.linalg.norm(F.sum(0)) <= 1e-5 * np.abs(F).sum()
    s.close()


def _system_with_path(w, staged, **kw):
    return gbmd.System.from_workload(w, precision="mixed",
                                     force_path="staged" if staged else "global", **kw)


@pytest.mark.parametrize("binary", [False, True])
def test_staged_and_global_force_paths_agree(binary):
    """The shared-memory (staged) force path and the global-index path give the same
    forces (to FP32 summation order) and the same neighbour sets."""
    w = (wl.lj_fluid(6000, 1.2, 1.0, seed=201, binary=True, r_buff=0.3) if binary
         else wl.lj_fluid(6000, 0.84, 1.2, seed=202))
    a = _system_with_path(w, True)
    b = _system_with_path(w, False)
    assert a.info()["force_path"] == 1 and b.info()["force_path"] == 0
    for s in (a, b):
        s.step(60)
    Fa, Fb = a.forces(), b.forces()
    pa, pb = a.state()[0], b.state()[0]
    assert np.abs(mi(pa - pb, w.box)).max() < 1e-4
    Fo, _, _, _, _ = oracle.forces(pa, w.box, w.types, w.pairs.as_dict())
    assert rel_l2(Fa, Fo) <= 1e-5
    st = a.state()
    a.set_state(*st)          # rebuild the lists at the positions compared below
    ca, ia = a.neighbors(cap=512)
    pos = a.state()[0]
    rl = w.pairs.rcut + w.r_buff
    pairs, r = oracle.neighbors(pos, w.box, w.types, rl)
    ok = np.abs(r - rl[w.types[pairs[:, 0]], w.types[pairs[:, 1]]]) > 1e-9
    ref = {(int(x), int(y)) for x, y in pairs[ok]}
    band = {(int(x), int(y)) for x, y in pairs[~ok]}
    mine = set()
    for i in range(w.n):
        for j in ia[i, :ca[i]]:
            mine.add((min(i, int(j)), max(i, int(j))))
    assert mine - band == ref
    ta, tb = a.thermo(), b.thermo()
    assert ta["pe"] == pytest.approx(tb["pe"], rel=1e-5)
    a.close()
    b.close()


def test_staged_window_overflow_falls_back():
    """A dense cluster in a large box: the staged windows exceed shared memory at the
    first build, the system falls back to global indices, and forces stay right."""
    blob = wl.lj_fluid(4000, 1.2, 1.0, seed=203)
    box = np.full(3, 60.0)
    s = _system_with_path(
        wl.Workload(blob.pos, blob.vel, blob.types, box, blob.pairs, r_buff=1.5), True)
    info = s.info()
    assert info["force_path"] == 0
    F = s.forces()
    Fo, *_ = oracle.forces(s.state()[0], box, None, blob.pairs.as_dict())
    assert rel_l2(F, Fo) <= 1e-5
    s.step(20)
    assert s.state()[3] == 20
    s.close()


def _pairs_of(s, n):
    counts, idx = s.neighbors(cap=512)
    out = set()
    for i in range(n):
        for j in idx[i, :counts[i]]:
            out.add((min(i, int(j)), max(i, int(j))))
    return out


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_cell_width_changes_nothing_physical(prec):
    """Wider cells (gbmd_set_cell_scale): a new grid, the same neighbour sets, the
    same forces up to summation order, and the same trajectory."""
    w = wl.lj_fluid(5000, 0.84, 1.2, seed=61)
    a = gbmd.System.from_workload(w, precision=prec)
    b = gbmd.System.from_workload(w, precision=prec)
    a.step(30)
    b.step(30)
    for x in (a, b):          # both rebuild their lists at the current positions
        x.set_state(*x.state())
    c0 = a.info()["cells"]
    before = _pairs_of(a, w.n)
    a.set_cell_scale(1.3)
    info = a.info()
    assert info["cell_scale"] == 1.3 and all(x < y for x, y in zip(info["cells"], c0))
    assert _pairs_of(a, w.n) == before
    tol = 1e-13 if prec == "fp64" else 1e-6
    assert rel_l2(a.forces(), b.forces()) <= tol
    a.step(40)
    b.step(40)
    pa, pb = a.state()[0], b.state()[0]
    assert np.abs(mi(pa - pb, w.box)).max() <= (1e-9 if prec == "fp64" else 1e-5)
    Fo, Uo, _, _, _ = oracle.forces(pa, w.box, w.types, w.pairs.as_dict())
    assert rel_l2(a.forces(), Fo) <= (1e-12 if prec == "fp64" else 1e-5)
    with pytest.raises(gbmd.GbmdError):
        a.set_cell_scale(0.5)
    a.close()
    b.close()


def test_autotune_picks_a_valid_cell_width_and_tuning():
    w = wl.lj_fluid(8000, 1.2, 1.0, seed=62, binary=True, r_buff=0.3)
    s = gbmd.System.from_workload(w, precision="mixed")
    s.step(20)
    s.autotune(None)
    info = s.info()
    assert info["cell_scale"] in (1.0, 1.1, 1.2, 1.35)
    assert info["threads_per_particle"] in (1, 2, 4) and info["force_block"] in (128, 256, 512)
    s.step(20)
    pos = s.state()[0]
    Fo, _, _, _, _ = oracle.forces(pos, w.box, w.types, w.pairs.as_dict())
    assert rel_l2(s.forces(), Fo) <= 1e-5
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_four_types_pair_table_path(prec):
    """Four particle types (the pair table read from shared memory rather than held in
    registers, in the force kernels and the list build): forces, energy and virial
    after stepping, and the neighbour sets, against the oracle."""
    base = wl.lj_fluid(1500, 0.9, 1.2, seed=35)
    rng = np.random.default_rng(35)
    types = rng.integers(0, 4, base.n).astype(np.int32)
    a = np.arange(4)
    eps = 0.6 + 0.2 * (a[:, None] + a[None, :])
    sigma = 0.85 + 0.05 * np.abs(a[:, None] - a[None, :])
    pairs = wl.PairTable(eps, sigma, 2.5 * sigma)
    w = wl.Workload(base.pos, base.vel, types, base.box, pairs, r_buff=0.4)
    s = gbmd.System.from_workload(w, precision=prec)
    s.step(25)
    check_forces(s, w, prec, "four types")
    s.set_state(*s.state())          # lists rebuilt at the current positions
    pos = s.state()[0]
    rl = pairs.rcut + w.r_buff
    pr, r = oracle.neighbors(pos, w.box, types, rl)
    ok = np.abs(r - rl[types[pr[:, 0]], types[pr[:, 1]]]) > 1e-9
    ref = {(int(x), int(y)) for x, y in pr[ok]}
    band = {(int(x), int(y)) for x, y in pr[~ok]}
    assert _pairs_of(s, w.n) - band == ref
    s.close()


def _four_type_workload(n, seed):
    base = wl.lj_fluid(n, 0.9, 1.2, seed=seed)
    types = np.random.default_rng(seed).integers(0, 4, base.n).astype(np.int32)
    a = np.arange(4)
    sigma = 0.85 + 0.05 * np.abs(a[:, None] - a[None, :])
    pairs = wl.PairTable(0.6 + 0.2 * (a[:, None] + a[None, :]), sigma, 2.5 * sigma)
    return wl.Workload(base.pos, base.vel, types, base.box, pairs, r_buff=0.4)


def test_batch_of_mixed_shapes_and_paths_equals_alone():
    """One batch holding a single-type system, a Kob-Andersen system, a four-type
    system and a system on the staged force path: two force launches share the
    step's last-block count, and the pair-table mode is the batch's widest.  Every
    member ends bitwise where it ends alone."""
    ws = [wl.lj_fluid(1200, 0.84, 1.2, seed=71),
          wl.lj_fluid(1500, 1.2, 1.0, seed=72, binary=True, r_buff=0.3),
          _four_type_workload(1000, 73),
          wl.lj_fluid(6000, 0.84, 1.2, seed=74)]
    paths = ["global", "global", "global", "staged"]
    alone = []
    for w, fp in zip(ws, paths):
        s = gbmd.System.from_workload(w, precision="mixed", force_path=fp)
        s.set_tuning(2, 128)
        s.step(60)
        alone.append((s.state(), s.forces()))
        s.close()
    b = gbmd.Batch("mixed")
    b.set_tuning(2, 128)
    sys_ = [gbmd.System.from_workload(w, precision="mixed", force_path=fp)
            for w, fp in zip(ws, paths)]
    assert sys_[3].info()["force_path"] == 1
    for s in sys_:
        b.add(s)
    b.step(60)
    b.sync()
    for s, (st, F) in zip(sys_, alone):
        st2 = s.state()
        assert st2[3] == 60
        for k in range(3):
            assert np.array_equal(np.asarray(st2[k]), np.asarray(st[k]))
        assert np.array_equal(s.forces(), F)
    b.close()
    for s in sys_:
        s.close()


def test_staged_path_four_types():
    w = _four_type_workload(6000, 75)
    a = gbmd.System.from_workload(w, precision="mixed", force_path="staged")
    g = gbmd.System.from_workload(w, precision="mixed", force_path="global")
    assert a.info()["force_path"] == 1
    a.step(30)
    g.step(30)
    pa, pg = a.state()[0], g.state()[0]
    assert np.abs(mi(pa - pg, w.box)).max() < 1e-4
    Fo, *_ = oracle.forces(pa, w.box, w.types, w.pairs.as_dict())
    assert rel_l2(a.forces(), Fo) <= 1e-5
    a.close()
    g.close()


def test_overflow_inside_a_batch_is_recovered_bitwise():
    """A batch member whose list overflows mid-run (the inflowing lattice gas) is
    frozen on the device while the others keep stepping, grown and caught up at the
    batch's sync; every member equals its roomy run alone."""
    g = (np.arange(12) - 5.5) * 1.5
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    box = np.full(3, 18.0)
    vel = -0.6 * pos / 9.0
    other = wl.lj_fluid(2000, 0.84, 1.2, seed=76)
    roomy = gbmd.System(pos, vel, box, precision="mixed", nlist_capacity=400)
    c0 = int(roomy.neighbors(cap=400)[0].max())
    roomy.set_tuning(2, 128)
    roomy.step(300)
    ref_gas = roomy.state()
    o = gbmd.System.from_workload(other, precision="mixed")
    o.set_tuning(2, 128)
    o.step(300)
    ref_other = o.state()
    roomy.close()
    o.close()
    b = gbmd.Batch("mixed")
    b.set_tuning(2, 128)
    tight = gbmd.System(pos, vel, box, precision="mixed", nlist_capacity=c0)
    o2 = gbmd.System.from_workload(other, precision="mixed")
    b.add(tight)
    b.add(o2)
    b.step(300)
    b.sync()
    assert tight.info()["nlist_capacity"] > c0
    for got, ref in ((tight.state(), ref_gas), (o2.state(), ref_other)):
        assert got[3] == 300
        for k in range(3):
            assert np.array_equal(np.asarray(got[k]), np.asarray(ref[k]))
    b.close()
    tight.close()
    o2.close()

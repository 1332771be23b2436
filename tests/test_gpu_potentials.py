"""The other pair potentials on the CUDA path (Mie, WCA, Yukawa, Gaussian) against
the FP64 CPU oracle, through the C ABI.

Tolerances:
* FP64 forces, energy, virial: <= 1e-12 relative (as for LJ: every operation is
  FP64, the libraries' pow / exp / sqrt are within an ulp or two);
* mixed forces: <= 1e-5 relative L2, per particle <= 1e-4 F_rms (as for LJ); the
  energy and virial sums <= 1e-5 relative: FP32 powers and exponentials carry a
  relative error of up to ~1e-6 (Mie: (n/2) times the logarithm's absolute error),
  and Mie's two powers cancel by up to a factor ~4 near the minimum;
* trajectories (FP64): <= 1e-9 sigma over 100 steps; NVT thermostat <= 1e-9.
Particles with a pair within a band of its r_cut are left out of per-particle
maxima.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1308_5587_gb300 import gbmd, workloads as wl

pytestmark = pytest.mark.gpu

KINDS = ["mie", "wca", "yukawa", "gauss"]


@pytest.fixture(scope="module", autouse=True)
def _setup():
    from paper_1308_5587_gb300 import _build
    _build.build()
    oracle.build()
    oracle.set_threads(os.cpu_count() or 1)


def pairs_single(kind):
    return {"mie": wl.mie_single(10.0, 6.0), "wca": wl.wca_single(),
            "yukawa": wl.yukawa_single(1.0, 1.0, 2.5), "gauss": wl.gauss_single(1.0, 1.0, 3.0)}[kind]


def pairs_mixture(kind):
    """Two types, every per-pair parameter different."""
    eps = np.array([[1.0, 1.2], [1.2, 0.8]])
    sig = np.array([[1.0, 0.9], [0.9, 0.85]])
    if kind == "mie":
        return wl.PairTable(eps, sig, 2.5 * sig, "mie", np.array([[12.0, 10.0], [10.0, 9.5]]),
                            np.array([[6.0, 6.0], [6.0, 5.5]]))
    if kind == "wca":
        return wl.PairTable(eps, sig, 2.0 ** (1 / 6) * sig, "wca")
    if kind == "yukawa":
        return wl.PairTable(eps, np.ones((2, 2)), np.array([[2.5, 2.2], [2.2, 2.0]]), "yukawa",
                            kappa=np.array([[1.0, 1.5], [1.5, 0.8]]))
    return wl.PairTable(eps, sig, 2.8 * sig, "gauss")


def fluid(kind, n, seed, binary=False, rho=0.84):
    p = pairs_mixture(kind) if binary else pairs_single(kind)
    return wl.lj_fluid(n, rho, 1.2, seed, pairs=p, binary=binary)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def near_cut(pos, box, types, rc, band):
    pairs, r = oracle.neighbors(pos, box, types, rc + band)
    hit = pairs[np.abs(r - rc[types[pairs[:, 0]], types[pairs[:, 1]]]) < band]
    return np.unique(hit.ravel())


def check(s, w, prec, where):
    pos = s.state()[0]
    p = w.pairs.as_dict()
    F = s.forces()
    Fo, Uo, Wo, uo, Wio = oracle.forces(pos, w.box, w.types, p)
    frms = np.sqrt(np.mean(Fo ** 2))
    mask = np.ones(w.n, bool)
    mask[near_cut(pos, w.box, w.types, oracle.cutoffs(p), 1e-9 if prec == "fp64" else 1e-5)] = False
    err, dmax = rel_l2(F, Fo), np.abs(F - Fo)[mask].max() / frms
    th = s.thermo()
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert err <= tol, (where, err)
    assert dmax <= (1e-11 if prec == "fp64" else 1e-4), (where, dmax)
    assert th["pe"] == pytest.approx(Uo, rel=tol), where
    assert np.allclose(th["virial"], Wo, rtol=tol, atol=tol * np.abs(Wo).max()), where
    u, Wi = s.per_particle()
    assert np.abs(u - uo).max() <= 10 * tol * (1 + np.abs(uo).max()), where
    assert np.abs(Wi - Wio).max() <= 10 * tol * (1 + np.abs(Wio).max()), where
    return err


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("binary", [False, True])
def test_forces_energy_virial(kind, prec, binary):
    # 4,999 particles: many tiles of every force launch and a ragged last one
    w = fluid(kind, 4999, seed=61, binary=binary, rho=1.0 if binary else 0.84)
    s = gbmd.System.from_workload(w, precision=prec)
    check(s, w, prec, f"{kind}/{prec}/binary={binary}")
    s.close()


@pytest.mark.parametrize("kind", KINDS)
def test_mixed_precision_after_steps(kind):
    """Forces at the GPU's own positions after 300 mixed steps (rebuilds included)."""
    w = fluid(kind, 3000, seed=62)
    s = gbmd.System.from_workload(w, precision="mixed", sort_period=50)
    s.step(300)
    assert s.info()["n_rebuilds"] >= 1
    check(s, w, "mixed", kind)
    s.close()


@pytest.mark.parametrize("kind", KINDS)
def test_fp64_trajectory_100_steps(kind):
    w = fluid(kind, 1000, seed=63, binary=(kind != "gauss"), rho=0.9)
    p = w.pairs.as_dict()
    o = oracle.vv_run(w.pos, w.vel, w.box, w.types, p, w.mass, w.dt, 100)
    s = gbmd.System.from_workload(w, precision="fp64")
    s.step(100)
    pos, vel, img, step = s.state()
    assert step == 100
    x_gpu = pos + img * w.box
    x_or = o["pos"] + o["image"] * w.box
    assert np.abs(x_gpu - x_or).max() <= 1e-9, kind
    assert np.abs(vel - o["vel"]).max() <= 1e-8, kind
    s.close()


def test_nvt_with_yukawa_matches_the_oracle():
    w = fluid("yukawa", 800, seed=64, binary=True, rho=0.9)
    p = w.pairs.as_dict()
    o = oracle.nvt_run(w.pos, w.vel, w.box, w.types, p, w.mass, w.dt, 1.5, 0.5, 100)
    s = gbmd.System.from_workload(w, precision="fp64", integrator="nvt", kT=1.5, tau=0.5)
    s.step(100)
    pos, vel, img, step = s.state()
    th = s.thermo()
    assert np.abs(pos + img * w.box - (o["pos"] + o["image"] * w.box)).max() <= 1e-9
    assert th["xi"] == pytest.approx(o["xi"], abs=1e-9)
    assert th["eta"] == pytest.approx(o["eta"], abs=1e-9)
    s.close()


@pytest.mark.parametrize("kind", KINDS)
def test_neighbor_set_uses_the_potential_cut(kind):
    w = fluid(kind, 2500, seed=65, binary=True, rho=1.0)
    s = gbmd.System.from_workload(w, precision="mixed")
    pos = s.state()[0]
    counts, idx = s.neighbors(cap=512)
    rl = oracle.cutoffs(w.pairs.as_dict()) + w.r_buff
    pairs, r = oracle.neighbors(pos, w.box, w.types, rl)
    ok = np.abs(r - rl[w.types[pairs[:, 0]], w.types[pairs[:, 1]]]) > 1e-9
    ref = {(int(a), int(b)) for a, b in pairs[ok]}
    band = {(int(a), int(b)) for a, b in pairs[~ok]}
    mine = {(min(i, int(j)), max(i, int(j))) for i in range(w.n) for j in idx[i, :counts[i]]}
    assert ref <= mine and mine - ref <= band
    s.close()


@pytest.mark.parametrize("kind", ["mie", "gauss"])
def test_batch_members_match_alone(kind):
    ws = [fluid(kind, n, seed=70 + k) for k, n in enumerate((900, 2100, 1500))]
    alone = []
    for w in ws:
        s = gbmd.System.from_workload(w, precision="mixed")
        s.step(60)
        alone.append((s.state(), s.thermo()))
        s.close()
    b = gbmd.Batch("mixed")
    sys_ = [gbmd.System.from_workload(w, precision="mixed") for w in ws]
    for s in sys_:
        b.add(s)
    b.step(60)
    b.sync()
    for s, (st, th) in zip(sys_, alone):
        st2 = s.state()
        for a, c in zip(st2[:3], st[:3]):
            assert np.array_equal(a, c)
        assert s.thermo()["pe"] == th["pe"]
    b.close()
    for s in sys_:
        s.close()


def test_batch_rejects_mixed_evaluators_and_staged_falls_back():
    b = gbmd.Batch("mixed")
    lj = gbmd.System.from_workload(wl.lj_fluid(1000, 0.84, 1.2, seed=80), precision="mixed")
    wca = gbmd.System.from_workload(fluid("wca", 1000, seed=81), precision="mixed")
    yuk = gbmd.System.from_workload(fluid("yukawa", 1000, seed=82), precision="mixed")
    b.add(lj)
    b.add(wca)          # LJ and WCA share the evaluator
    with pytest.raises(gbmd.GbmdError) as e:
        b.add(yuk)
    assert e.value.status == "BAD_ARG"
    b.close()
    for s in (lj, wca, yuk):
        s.close()
    # the staged path serves LJ / WCA only; a Mie system asking for it runs global
    w = fluid("mie", 40000, seed=83)
    s = gbmd.System.from_workload(w, precision="mixed", force_path="staged")
    assert s.info()["force_path"] == 0
    check(s, w, "mixed", "mie staged request")
    s.close()
    w = fluid("wca", 40000, seed=84)
    s = gbmd.System.from_workload(w, precision="mixed", force_path="staged")
    assert s.info()["force_path"] == 1
    check(s, w, "mixed", "wca staged")
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("kind", ["mie", "yukawa", "gauss"])
def test_potentials_on_the_tree_list(kind, prec):
    """The evaluators and the tree neighbour list together: two types, then after
    steps with rebuilds, against the oracle."""
    w = fluid(kind, 3000, seed=66, binary=True, rho=1.0)
    s = gbmd.System.from_workload(w, precision=prec, nlist="tree")
    assert s.info()["nlist"] == gbmd.GBMD_NLIST_TREE
    check(s, w, prec, f"{kind}/{prec}/tree")
    s.step(120)
    check(s, w, prec, f"{kind}/{prec}/tree after steps")
    s.close()


def test_mie_nvt_batch_members_match_alone():
    ws = [fluid("mie", n, seed=75 + k) for k, n in enumerate((800, 1700))]
    kw = dict(precision="mixed", integrator="nvt", kT=1.1, tau=0.7)
    alone = []
    for w in ws:
        s = gbmd.System.from_workload(w, **kw)
        s.set_tuning(2, 128)
        s.step(50)
        alone.append((s.state(), s.thermo()))
        s.close()
    b = gbmd.Batch("mixed")
    b.set_tuning(2, 128)
    ss = [gbmd.System.from_workload(w, **kw) for w in ws]
    for s in ss:
        b.add(s)
    b.step(50)
    b.sync()
    for s, (st, th) in zip(ss, alone):
        for x, y in zip(s.state()[:3], st[:3]):
            assert np.array_equal(x, y)
        t2 = s.thermo()
        assert t2["xi"] == th["xi"] and t2["pe"] == th["pe"]
    b.close()
    for s in ss:
        s.close()

"""NVT (Nose-Hoover in the MTK form) on the GPU against the oracle's integrator.

The FP64 path follows the oracle's trajectory to 1e-9 over 100 steps (positions,
velocities, thermostat); the mixed path stays close; the thermostat drives the
temperature to kT while the extended energy H = K + U + g kT (tau^2 xi^2/2 + eta)
stays conserved; batches and checkpoints behave as for NVE.
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


def mi(d, box):
    return d - box * np.rint(d / box)


def nvt_system(w, prec, kT, tau, **kw):
    return gbmd.System.from_workload(w, precision=prec, integrator="nvt", kT=kT, tau=tau, **kw)


def test_nvt_fp64_trajectory_follows_the_oracle():
    w = wl.lj_fluid(2000, 0.84, 1.0, seed=81)
    kT, tau, steps = 1.5, 0.5, 100
    s = nvt_system(w, "fp64", kT, tau)
    s.step(steps)
    pos, vel, img, st = s.state()
    th = s.thermo()
    o = oracle.nvt_run(w.pos, w.vel, w.box, w.types, w.pairs.as_dict(), w.mass, w.dt, kT, tau,
                       steps, series=True)
    assert st == steps
    assert np.abs(mi(pos - o["pos"], w.box)).max() <= 1e-9
    assert np.abs(vel - o["vel"]).max() <= 1e-9
    assert th["xi"] == pytest.approx(o["xi"], abs=1e-11)
    assert th["eta"] == pytest.approx(o["eta"], abs=1e-11)
    g = 3 * w.n - 3
    H = o["ke"][-1] + o["pe"][-1] + g * kT * (0.5 * tau * tau * o["xi"] ** 2 + o["eta"])
    assert th["h_ext"] == pytest.approx(H, rel=1e-11)
    assert abs(o["xi"]) > 1e-2          # the thermostat acted
    s.close()


def test_nvt_mixed_stays_close_to_fp64():
    w = wl.lj_fluid(3000, 0.84, 1.0, seed=82)
    a = nvt_system(w, "fp64", 1.4, 0.4)
    b = nvt_system(w, "mixed", 1.4, 0.4)
    a.step(100)
    b.step(100)
    pa, pb = a.state()[0], b.state()[0]
    assert np.abs(mi(pa - pb, w.box)).max() <= 1e-4
    assert b.thermo()["xi"] == pytest.approx(a.thermo()["xi"], abs=1e-4)
    a.close()
    b.close()


def test_nvt_drives_temperature_and_conserves_h_ext():
    """The temperature goes to kT; the extended energy fluctuates no more than the
    oracle's does on the same system (the trajectories part, so the comparison is of
    the size of the fluctuation: the integration error of a hot, dense liquid)."""
    w = wl.lj_fluid(1000, 0.84, 1.0, seed=83)
    kT, tau = 2.0, 0.5
    s = nvt_system(w, "mixed", kT, tau)
    h0 = s.thermo()["h_ext"]
    T, H = [], []
    for k in range(20):
        s.step(100)
        t = s.thermo()
        T.append(t["temperature"])
        H.append(t["h_ext"])
    s.close()
    assert abs(np.mean(T[10:]) - kT) < 0.25
    o = oracle.nvt_run(w.pos, w.vel, w.box, w.types, w.pairs.as_dict(), w.mass, w.dt, kT, tau,
                       2000, series=True)
    g = 3 * w.n - 3
    Ho = o["ke"] + o["pe"] + g * kT * (0.5 * tau * tau * o["xis"] ** 2 + o["etas"])
    dev_gpu = np.abs(np.array(H) - h0).max()
    dev_oracle = np.abs(Ho[100::100] - Ho[0]).max()
    assert h0 == pytest.approx(Ho[0], rel=1e-6)
    assert dev_gpu <= 3.0 * dev_oracle + 1e-6 * abs(h0), (dev_gpu, dev_oracle)


def test_nvt_batch_alone_equals_in_mix_and_no_mixing_with_nve():
    ws = [wl.lj_fluid(n, 0.8, 1.0, seed=84 + k) for k, n in enumerate((900, 1500, 2200))]
    alone = []
    for w in ws:
        s = nvt_system(w, "mixed", 1.3, 0.6)
        s.set_tuning(2, 128)
        s.step(80)
        alone.append((s.state(), s.thermo()))
        s.close()
    b = gbmd.Batch("mixed")
    b.set_tuning(2, 128)
    sys_ = [nvt_system(w, "mixed", 1.3, 0.6) for w in ws]
    for s in sys_:
        b.add(s)
    nve = gbmd.System.from_workload(ws[0], precision="mixed")
    with pytest.raises(gbmd.GbmdError) as e:
        b.add(nve)
    assert e.value.status == "BAD_ARG"
    b.step(80)
    b.sync()
    for s, (st, th) in zip(sys_, alone):
        st2 = s.state()
        for k in range(4):
            assert np.array_equal(np.asarray(st2[k]), np.asarray(st[k]))
        assert s.thermo()["xi"] == th["xi"]
    b.close()
    nve.close()
    for s in sys_:
        s.close()


def test_nvt_checkpoint_resume_and_setter_rules():
    w = wl.lj_fluid(2000, 0.84, 1.0, seed=87)
    ref = nvt_system(w, "fp64", 1.5, 0.5)
    ref.step(100)
    a = nvt_system(w, "fp64", 1.5, 0.5)
    a.step(50)
    pos, vel, img, st = a.state()
    th = a.thermo()
    with pytest.raises(gbmd.GbmdError) as e:       # mid-run: not a completed-step state
        a.set_thermostat(th["xi"], th["eta"])
    assert e.value.status == "STATE"
    b = nvt_system(w, "fp64", 1.5, 0.5)
    b.set_state(pos, vel, img, st)
    b.set_thermostat(th["xi"], th["eta"])
    b.step(50)
    p1, p2 = ref.state()[0], b.state()[0]
    assert np.abs(mi(p1 - p2, w.box)).max() <= 1e-9
    assert b.thermo()["xi"] == pytest.approx(ref.thermo()["xi"], abs=1e-11)
    nve = gbmd.System.from_workload(w, precision="fp64")
    with pytest.raises(gbmd.GbmdError) as e:
        nve.set_thermostat(0.1, 0.0)
    assert e.value.status == "BAD_ARG"
    for s in (ref, a, b, nve):
        s.close()

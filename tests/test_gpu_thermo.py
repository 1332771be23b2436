"""Temperature, kinetic energy and pressure of the CUDA path against the FP64 oracle.

Section 7.1 checks force, energy and virial against independently computed values;
gbmd_get_thermo also returns K, T and P = (N T + tr W / 3) / V built from them.
Each case reads the GPU's own state (tag order, full-step velocities), recomputes
K with ``oracle.kinetic``, the virial with ``oracle.forces`` and (T, P) with
``oracle.thermo``, and compares them with the GPU's readout:
* FP64: <= 1e-12 relative (FP64 throughout; only summation order differs);
* mixed: <= 2e-5 relative (FP32 pair forces enter the virial and the closing half
  kick of the velocities; the parity tests bound the force error by 1e-5).
The pressure is compared relative to the scale of its two terms, N T / V + |tr W| / (3 V),
so a state where they nearly cancel is not judged by a tiny denominator.
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


def _check(s, w, prec):
    rel = 1e-12 if prec == "fp64" else 2e-5
    pos, vel, _, step = s.state()
    th = s.thermo()
    assert th["step"] == step
    K = oracle.kinetic(vel, w.mass)
    _, U, W, _, _ = oracle.forces(pos, w.box, w.types, w.pairs.as_dict())
    T, P = oracle.thermo(w.n, w.box, K, W)
    vol = float(np.prod(w.box))
    assert th["ke"] == pytest.approx(K, rel=rel)
    assert th["temperature"] == pytest.approx(T, rel=rel)
    assert th["pe"] == pytest.approx(U, rel=rel)
    trw = W[0] + W[3] + W[5]
    assert th["w"] == pytest.approx(trw, rel=rel, abs=rel * np.abs(W).max())
    scale = w.n * T / vol + abs(trw) / (3 * vol)
    assert abs(th["pressure"] - P) <= rel * scale, (th["pressure"], P)
    return th


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_pressure_temperature_kinetic_at_creation_and_after_steps(prec):
    w = wl.lj_fluid(4000, 0.84, 1.2, seed=701)
    s = gbmd.System.from_workload(w, precision=prec)
    th0 = _check(s, w, prec)                  # full-step velocities as given
    assert th0["temperature"] == pytest.approx(1.2, rel=1e-12)
    s.step(60)                                # velocities half a kick behind on the device
    _check(s, w, prec)
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_pressure_of_a_binary_mixture_on_the_staged_and_global_paths(prec):
    # 4,000 particles at rho 1.2: 5 cells per axis, windows inside shared memory
    w = wl.lj_fluid(4000, 1.2, 1.0, seed=702, binary=True, r_buff=0.3)
    paths = ["global"] + (["staged"] if prec == "mixed" else [])
    for path in paths:
        s = gbmd.System.from_workload(w, precision=prec, force_path=path)
        assert s.info()["force_path"] == (1 if path == "staged" else 0)
        s.step(40)
        _check(s, w, prec)
        s.close()


def test_pressure_of_a_dilute_gas_is_near_ideal():
    # few pairs inside the cut: P is dominated by N T / V and the virial is small
    w = wl.lj_fluid(2000, 0.1, 2.0, seed=703)
    s = gbmd.System.from_workload(w, precision="fp64")
    th = _check(s, w, "fp64")
    vol = float(np.prod(w.box))
    ideal = w.n * th["temperature"] / vol
    assert abs(th["pressure"] - ideal) < 0.2 * ideal
    s.close()

"""Pins for the FP64 CPU oracle: what the physics and the mathematics fix.

None of these compares the oracle with itself.  Each pin is chosen so that a
plausible slip in ``oracle/lj_oracle.c`` (a dropped factor, a wrong sign or
index, a transposed operand, a wrong wrap) fails at least one of them:

* closed forms of the 12-6 potential at r = sigma and r = 2^(1/6) sigma, and the
  exact shift at r_cut = 2.5 sigma (two particles and the six-particle fixture
  of Section 7.1, including periodic images across every face);
* Newton's third law, F = -grad U by central differences, the virial as the
  strain derivative of U;
* the neighbour set against scipy's periodic k-d tree (independent search);
* velocity Verlet against an independent high-order ODE solver, its second
  order convergence, time reversibility, momentum conservation, free flight
  through the periodic boundary, energy conservation;
* the ideal-gas limit of the pressure;
* Nose-Hoover (MTK) NVT: the weak-coupling limit is velocity Verlet exactly, the
  extended energy is conserved at second order in dt, the splitting is time
  reversible under (v, xi) -> (-v, -xi), and the thermostat drives the
  temperature to kT where NVE would not.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_1308_5587_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
VLJ_CUT_25 = -0.016316891136        # 4 (0.4^12 - 0.4^6), exact decimal
F_CUT_25 = -0.0389994774528         # 24 (2*0.4^12 - 0.4^6) / 2.5, exact decimal
R_MIN = 2.0 ** (1.0 / 6.0)


def pair_params(eps=1.0, sigma=1.0, rcut=2.5):
    return {"eps": np.array([[eps]]), "sigma": np.array([[sigma]]),
            "rcut": np.array([[rcut]])}


def two_particles(r, axis=0, L=20.0):
    pos = np.zeros((2, 3))
    pos[1, axis] = -r        # d_01 = x0 - x1 = +r along axis
    return pos, np.full(3, L)


# --- closed forms ---------------------------------------------------------------

@pytest.mark.parametrize("eps,sigma", [(1.0, 1.0), (0.5, 1.0), (2.0, 1.25), (1.5, 0.8)])
def test_two_particle_closed_form(oracle, eps, sigma):
    p = pair_params(eps, sigma, 2.5 * sigma)
    # r = sigma: V_LJ = 0, so V = -V_LJ(rc); |F| = 24 eps / sigma, repulsive
    for axis in range(3):
        pos, box = two_particles(sigma, axis)
        F, U, W, ui, _ = oracle.forces(pos, box, None, p)
        assert U == pytest.approx(-eps * VLJ_CUT_25, rel=1e-12)
        assert F[0, axis] == pytest.approx(24 * eps / sigma, rel=1e-12)
        assert np.allclose(F[0], -F[1], atol=0)
        assert np.abs(np.delete(F[0], axis)).max() == 0
        assert W[[0, 3, 5][axis]] == pytest.approx(24 * eps, rel=1e-12)   # r |F|
        assert ui == pytest.approx([U / 2, U / 2], rel=1e-14)
    # r = 2^(1/6) sigma: minimum, F = 0, V = -eps - V_LJ(rc)
    pos, box = two_particles(R_MIN * sigma)
    F, U, W, _, _ = oracle.forces(pos, box, None, p)
    assert U == pytest.approx(-eps - eps * VLJ_CUT_25, rel=1e-12)
    assert np.abs(F).max() < 1e-12 * eps / sigma
    # just inside the cut: the shifted energy vanishes continuously, force does not
    pos, box = two_particles(2.5 * sigma * (1 - 1e-12))
    F, U, W, _, _ = oracle.forces(pos, box, None, p)
    assert abs(U) < 1e-10 * eps
    assert F[0, 0] == pytest.approx(eps / sigma * F_CUT_25, rel=1e-9)
    # at and beyond the cut: nothing (strict '<')
    for r in (2.5 * sigma, 2.5 * sigma * (1 + 1e-12), 3.0 * sigma):
        pos, box = two_particles(r)
        F, U, W, _, _ = oracle.forces(pos, box, None, p)
        assert U == 0 and np.all(F == 0) and np.all(W == 0)


def test_six_particle_fixture(oracle):
    """Section 7.1's six-particle LJ unit test, values from the calculator script."""
    doc = json.load(open(os.path.join(GOLDEN, "lj_six_particle.json")))
    assert len(doc["cases"]) >= 5
    for c in doc["cases"]:
        params = {k: np.array(c[k]) for k in ("eps", "sigma", "rcut")}
        F, U, W, ui, _ = oracle.forces(np.array(c["pos"]), np.array(c["box"]),
                                       np.array(c["types"], np.int32), params)
        assert U == pytest.approx(c["energy"], rel=1e-12, abs=1e-14), c["name"]
        assert np.allclose(F, np.array(c["force"]), rtol=0, atol=1e-11), c["name"]
        assert np.allclose(W, np.array(c["virial"]), rtol=0, atol=1e-11), c["name"]
        assert np.allclose(ui, np.array(c["per_energy"]), rtol=0, atol=1e-13), c["name"]


def test_periodic_image_invariance(oracle):
    """Shifting any particle by a box vector changes nothing (min image)."""
    w = wl.lj_fluid(256, 0.84, 1.2, seed=11)
    F0, U0, W0, _, _ = oracle.forces(w.pos, w.box, None, w.pairs.as_dict())
    rng = np.random.default_rng(3)
    shifted = w.pos + rng.integers(-2, 3, size=w.pos.shape) * w.box
    F1, U1, W1, _, _ = oracle.forces(shifted, w.box, None, w.pairs.as_dict())
    assert U1 == pytest.approx(U0, rel=1e-12)
    assert np.allclose(F1, F0, rtol=0, atol=1e-10 * np.abs(F0).max())
    assert np.allclose(W1, W0, rtol=1e-12, atol=1e-10)


# --- invariants and derivatives -------------------------------------------------

@pytest.mark.parametrize("binary", [False, True])
def test_newton_third_law(oracle, binary):
    w = wl.lj_fluid(500, 1.2 if binary else 0.84, 1.0, seed=5, binary=binary)
    F, *_ = oracle.forces(w.pos, w.box, w.types, w.pairs.as_dict())
    assert np.linalg.norm(F.sum(0)) <= 1e-10 * np.linalg.norm(F, axis=1).sum()


def _clear_of_cut(pos, box, types, rcut, margin):
    d = pos[:, None, :] - pos[None, :, :]
    d -= box * np.rint(d / box)
    r = np.sqrt((d * d).sum(-1))
    rc = rcut[types[:, None], types[None, :]]
    np.fill_diagonal(r, 10 * rc.max())
    return np.abs(r - rc).min() > margin


@pytest.mark.parametrize("binary", [False, True])
def test_force_is_minus_energy_gradient(oracle, binary):
    for seed in range(100, 200):
        w = wl.lj_fluid(64, 0.6, 1.0, seed=seed, binary=binary, jitter=0.2)
        if _clear_of_cut(w.pos, w.box, w.types, w.pairs.rcut, 1e-4):
            break
    p = w.pairs.as_dict()
    F, U, *_ = oracle.forces(w.pos, w.box, w.types, p)
    h = 1e-6
    grad = np.zeros_like(F)
    for i in range(w.n):
        for a in range(3):
            xp = w.pos.copy(); xp[i, a] += h
            xm = w.pos.copy(); xm[i, a] -= h
            grad[i, a] = (oracle.forces(xp, w.box, w.types, p)[1]
                          - oracle.forces(xm, w.box, w.types, p)[1]) / (2 * h)
    frms = math.sqrt(np.mean(F ** 2))
    assert np.abs(F + grad).max() <= 1e-6 * frms


def test_virial_is_strain_derivative(oracle):
    """W_aa = -dU/d(lambda_a) under axis scaling; W_ab = -dU/d(gamma_ab) under shear."""
    for seed in range(300, 400):
        w = wl.lj_fluid(64, 0.6, 1.0, seed=seed, binary=True, jitter=0.2)
        if _clear_of_cut(w.pos, w.box, w.types, w.pairs.rcut, 1e-4):
            break
    p = w.pairs.as_dict()
    _, U, W, *_ = oracle.forces(w.pos, w.box, w.types, p)
    h = 1e-7
    comp = {(0, 0): 0, (0, 1): 1, (0, 2): 2, (1, 1): 3, (1, 2): 4, (2, 2): 5}
    for a in range(3):
        s = np.ones(3); s[a] += h
        up = oracle.forces(w.pos * s, w.box * s, w.types, p)[1]
        s[a] -= 2 * h
        dn = oracle.forces(w.pos * s, w.box * s, w.types, p)[1]
        assert -(up - dn) / (2 * h) == pytest.approx(W[comp[(a, a)]], rel=1e-6, abs=1e-6)
    # shear: an isolated cluster in the middle of a large box (no boundary pairs)
    cl = wl.lj_fluid(27, 0.8, 1.0, seed=7, jitter=0.1)
    big = np.full(3, 60.0)
    _, U, W, *_ = oracle.forces(cl.pos, big, None, cl.pairs.as_dict())
    for (a, b) in [(0, 1), (0, 2), (1, 2)]:
        def energy(g):
            x = cl.pos.copy(); x[:, a] += g * cl.pos[:, b]
            return oracle.forces(x, big, None, cl.pairs.as_dict())[1]
        dU = (energy(h) - energy(-h)) / (2 * h)
        assert -dU == pytest.approx(W[comp[(a, b)]], rel=1e-6, abs=1e-6)


def test_per_particle_halves_and_subset(oracle):
    w = wl.lj_fluid(300, 1.2, 1.0, seed=9, binary=True)
    p = w.pairs.as_dict()
    F, U, W, ui, Wi = oracle.forces(w.pos, w.box, w.types, p)
    assert ui.sum() == pytest.approx(U, rel=1e-12)
    assert np.allclose(Wi.sum(0), W, rtol=1e-12, atol=1e-10)
    idx = np.array([0, 17, 299, 5, 5])
    Fs, us, Ws = oracle.forces_subset(w.pos, w.box, w.types, p, idx)
    assert np.array_equal(Fs, F[idx]) and np.array_equal(us, ui[idx])
    assert np.array_equal(Ws, Wi[idx])


# --- neighbour set against an independent search --------------------------------

@pytest.mark.parametrize("binary", [False, True])
def test_neighbors_match_periodic_kdtree(oracle, binary):
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(21 + binary)
    L = np.array([15.0, 13.0, 17.0])
    n = 2500
    pos = (rng.random((n, 3)) - 0.5) * L
    types = (rng.random(n) < 0.3).astype(np.int32) if binary else np.zeros(n, np.int32)
    rl = np.array([[2.8, 2.3], [2.3, 2.5]]) if binary else np.array([[2.9]])
    pairs, r = oracle.neighbors(pos, L, types, rl)
    tree = cKDTree(pos + 0.5 * L, boxsize=L)
    sdm = tree.sparse_distance_matrix(tree, rl.max(), output_type="ndarray")
    sdm = sdm[sdm["i"] < sdm["j"]]
    keep = sdm["v"] < rl[types[sdm["i"]], types[sdm["j"]]]
    ref = sdm[keep]
    band = 1e-9
    rl_mine = rl[types[pairs[:, 0]], types[pairs[:, 1]]]
    mine = {(int(i), int(j)) for (i, j), d, c in zip(pairs, r, rl_mine) if abs(d - c) > band}
    rl_ref = rl[types[ref["i"]], types[ref["j"]]]
    theirs = {(int(i), int(j)) for i, j, d, c in zip(ref["i"], ref["j"], ref["v"], rl_ref)
              if abs(d - c) > band}
    assert len(mine) > 1000
    assert mine == theirs
    assert np.all(pairs[:, 0] < pairs[:, 1])
    assert np.all(np.diff(pairs[:, 0]) >= 0)


# --- velocity Verlet ------------------------------------------------------------

def test_free_flight_through_boundary(oracle):
    """No interactions: x(t) = x0 + v t, wrapped, with exact image counts."""
    L = np.array([30.0, 31.0, 32.0])
    # three lanes at least 10 apart in two coordinates: they never meet
    pos = np.array([[0.0, 0.0, 0.0], [10.0, 3.0, 10.0], [-10.0, -10.0, -12.0]])
    vel = np.array([[37.0, 0.0, 0.0], [0.0, -41.0, 0.0], [0.0, 0.0, 45.5]])
    dt, n = 0.01, 400
    out = oracle.vv_run(pos, vel, L, None, pair_params(), 1.0, dt, n)
    x = pos + n * dt * vel
    k = np.floor((x + 0.5 * L) / L)
    assert np.array_equal(out["image"], k.astype(np.int32))
    assert np.allclose(out["pos"], x - k * L, rtol=0, atol=1e-11)
    assert np.array_equal(out["vel"], vel)


def _vv_cluster():
    pos = np.array([[0.0, 0.0, 0.0], [1.12, 0.05, 0.0], [0.5, 0.95, 0.1], [0.4, 0.4, 0.9]])
    vel = np.array([[0.3, -0.2, 0.1], [-0.1, 0.4, 0.0], [0.0, -0.3, 0.2], [-0.2, 0.1, -0.3]])
    return pos, vel, np.full(3, 40.0)


def test_verlet_matches_ode_solver_second_order(oracle):
    from scipy.integrate import solve_ivp
    pos, vel, L = _vv_cluster()
    p = pair_params()
    T = 0.4

    def rhs(t, y):
        x = y[:12].reshape(4, 3)
        F = oracle.forces(x, L, None, p)[0]
        return np.concatenate([y[12:], F.ravel()])

    sol = solve_ivp(rhs, (0, T), np.concatenate([pos.ravel(), vel.ravel()]), method="DOP853",
                    rtol=1e-12, atol=1e-12)
    x_ref = sol.y[:12, -1].reshape(4, 3)
    errs = []
    for dt in (0.004, 0.002, 0.001):
        out = oracle.vv_run(pos, vel, L, None, p, 1.0, dt, int(round(T / dt)))
        errs.append(np.abs(out["pos"] - x_ref).max())
    assert errs[-1] < 2e-5
    for a, b in zip(errs, errs[1:]):
        assert 3.5 < a / b < 4.5        # O(dt^2)


def test_time_reversibility_and_momentum(oracle):
    w = wl.lj_fluid(108, 0.84, 1.2, seed=2)
    p = w.pairs.as_dict()
    fwd = oracle.vv_run(w.pos, w.vel, w.box, None, p, 1.0, 0.005, 100)
    back = oracle.vv_run(fwd["pos"], -fwd["vel"], w.box, None, p, 1.0, 0.005, 100,
                         image=fwd["image"])
    x0, _ = oracle.wrap(w.pos, w.box)
    d = back["pos"] - x0
    d -= w.box * np.rint(d / w.box)
    assert np.abs(d).max() < 1e-9
    assert np.allclose(back["vel"], -w.vel, rtol=0, atol=1e-9)
    assert np.abs(fwd["vel"].sum(0)).max() < 1e-12 * np.abs(w.vel).sum()


def test_nve_energy_conservation(oracle):
    w = wl.lj_fluid(256, 0.84, 1.2, seed=4)
    out = oracle.vv_run(w.pos, w.vel, w.box, None, w.pairs.as_dict(), 1.0, 0.005, 1000,
                        series=True)
    e = out["pe"] + out["ke"]
    assert np.abs(e - e[0]).max() < 2e-3 * abs(e[0])
    # halving dt shrinks the energy error roughly fourfold (second order)
    w2 = wl.lj_fluid(256, 0.84, 1.2, seed=4)
    out2 = oracle.vv_run(w2.pos, w2.vel, w2.box, None, w2.pairs.as_dict(), 1.0, 0.0025, 40,
                         series=True)
    out1 = oracle.vv_run(w2.pos, w2.vel, w2.box, None, w2.pairs.as_dict(), 1.0, 0.005, 20,
                         series=True)
    e1 = out1["pe"] + out1["ke"]
    e2 = out2["pe"] + out2["ke"]
    assert np.abs(e2 - e2[0]).max() < np.abs(e1 - e1[0]).max()


def test_ideal_gas_pressure(oracle):
    """No pair inside the cut: W = 0 and P = rho T, T = 2K / (3N - 3)."""
    g = np.arange(4) * 5.0 - 7.5
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    vel = np.random.default_rng(1).normal(size=pos.shape)
    L = np.full(3, 20.0)
    _, U, W, _, _ = oracle.forces(pos, L, None, pair_params())
    assert U == 0 and np.all(W == 0)
    K = oracle.kinetic(vel, 2.0)
    assert K == pytest.approx(float((vel ** 2).sum()), rel=1e-14)   # m = 2
    T, P = oracle.thermo(len(pos), L, K, W)
    assert T == pytest.approx(2 * K / (3 * len(pos) - 3), rel=1e-14)
    assert P == pytest.approx(len(pos) / 8000.0 * T, rel=1e-14)


def test_virial_pressure_is_minus_volume_derivative_of_energy(oracle):
    """At K = 0 the pressure is the configurational one, P = -dU/dV, with U(V) taken
    under uniform scaling of the box and every position (V = lambda^3 V0): a
    central difference in lambda fixes the sign, the 1/3 and the 1/V of the
    virial term independently of how the oracle writes P."""
    for seed in range(300, 400):
        w = wl.lj_fluid(64, 0.6, 1.0, seed=seed, binary=True, jitter=0.2)
        if _clear_of_cut(w.pos, w.box, w.types, w.pairs.rcut, 1e-4):
            break
    p = w.pairs.as_dict()
    _, U, W, *_ = oracle.forces(w.pos, w.box, w.types, p)
    h = 1e-7
    up = oracle.forces(w.pos * (1 + h), w.box * (1 + h), w.types, p)[1]
    dn = oracle.forces(w.pos * (1 - h), w.box * (1 - h), w.types, p)[1]
    vol = float(np.prod(w.box))
    dU_dV = (up - dn) / (2 * h) / (3 * vol)          # dV/dlambda = 3 V0 at lambda = 1
    _, P = oracle.thermo(w.n, w.box, 0.0, W)
    assert abs(W[0] + W[3] + W[5]) > 1.0              # a real virial, not the W = 0 case
    assert P == pytest.approx(-dU_dV, rel=1e-6, abs=1e-9)


def test_pair_pressure_closed_form(oracle):
    """Two particles at r = sigma in an otherwise empty box: the pair virial is
    r |F(r)| = 24 eps (Clausius), so at K = 0 P = 24 eps / (3 V) = 8 eps / V; adding
    kinetic energy adds the ideal-gas part N T / V and nothing else."""
    for eps in (1.0, 0.7):
        pos, box = two_particles(1.0, axis=1, L=12.0)
        _, _, W, _, _ = oracle.forces(pos, box, None, pair_params(eps=eps))
        vol = 12.0 ** 3
        T0, P0 = oracle.thermo(2, box, 0.0, W)
        assert T0 == 0.0
        assert P0 == pytest.approx(8.0 * eps / vol, rel=1e-12)
        K = 1.7
        T, P = oracle.thermo(2, box, K, W)
        assert T == pytest.approx(2 * K / 3, rel=1e-14)        # 3N - 3 = 3 degrees of freedom
        assert P == pytest.approx(P0 + 2 * T / vol, rel=1e-12)


def test_oracle_thread_count_independent(oracle):
    w = wl.lj_fluid(400, 0.84, 1.2, seed=8)
    old = oracle.get_threads()
    try:
        oracle.set_threads(1)
        a = oracle.forces(w.pos, w.box, None, w.pairs.as_dict())
        oracle.set_threads(4)
        b = oracle.forces(w.pos, w.box, None, w.pairs.as_dict())
    finally:
        oracle.set_threads(old)
    assert np.array_equal(a[0], b[0]) and a[1] == b[1]


# --- Nose-Hoover (MTK) NVT -------------------------------------------------------

def _h_ext(r, n, kT, tau):
    g = 3 * n - 3
    return r["ke"] + r["pe"] + g * kT * (0.5 * tau * tau * r["xis"] ** 2 + r["etas"])


def test_nvt_weak_coupling_is_velocity_verlet(oracle):
    w = wl.lj_fluid(108, 0.84, 1.2, seed=5)
    p = w.pairs.as_dict()
    a = oracle.nvt_run(w.pos, w.vel, w.box, None, p, 1.0, 0.005, 1.2, 1e12, 60)
    b = oracle.vv_run(w.pos, w.vel, w.box, None, p, 1.0, 0.005, 60)
    assert np.array_equal(a["pos"], b["pos"]) and np.array_equal(a["vel"], b["vel"])
    assert abs(a["xi"]) < 1e-20


def _nvt_cluster():
    # four particles near the pair minimum, far from every cut-off and image
    pos = np.array([[0.0, 0.0, 0.0], [1.12, 0.0, 0.0], [0.56, 0.97, 0.0], [0.56, 0.32, 0.91]])
    vel = np.random.default_rng(8).normal(scale=0.3, size=(4, 3))
    vel -= vel.mean(0)
    return pos, vel, np.full(3, 30.0)


def test_nvt_extended_energy_is_conserved_at_second_order(oracle):
    pos, vel, box = _nvt_cluster()
    p = pair_params()
    kT, tau, t_end = 0.5, 0.2, 0.4
    drift = []
    for dt in (0.004, 0.002):
        r = oracle.nvt_run(pos, vel, box, None, p, 1.0, dt, kT, tau, int(round(t_end / dt)),
                           series=True)
        H = _h_ext(r, 4, kT, tau)
        drift.append(np.abs(H - H[0]).max())
        assert abs(r["xi"]) > 1e-3          # the thermostat did act
    ratio = drift[0] / drift[1]
    assert 3.0 < ratio < 5.5, ratio         # second order: 4


def test_nvt_time_reversibility(oracle):
    w = wl.lj_fluid(108, 0.84, 1.2, seed=6)
    p = w.pairs.as_dict()
    fwd = oracle.nvt_run(w.pos, w.vel, w.box, None, p, 1.0, 0.005, 0.8, 0.3, 100)
    back = oracle.nvt_run(fwd["pos"], -fwd["vel"], w.box, None, p, 1.0, 0.005, 0.8, 0.3, 100,
                          xi=-fwd["xi"], image=fwd["image"])
    x0, _ = oracle.wrap(w.pos, w.box)
    d = back["pos"] - x0
    d -= w.box * np.rint(d / w.box)
    assert np.abs(d).max() < 1e-9
    assert np.allclose(back["vel"], -w.vel, rtol=0, atol=1e-9)
    assert abs(back["xi"]) < 1e-9 and abs(fwd["xi"]) > 1e-2


def test_nvt_drives_the_temperature_to_kT(oracle):
    w = wl.lj_fluid(256, 0.84, 1.0, seed=7)
    p = w.pairs.as_dict()
    n, g = w.n, 3 * w.n - 3
    r = oracle.nvt_run(w.pos, w.vel, w.box, None, p, 1.0, 0.005, 2.0, 0.5, 2000, series=True)
    T = 2.0 * r["ke"] / g
    assert abs(T[1000:].mean() - 2.0) < 0.2
    e = oracle.vv_run(w.pos, w.vel, w.box, None, p, 1.0, 0.005, 2000, series=True)
    assert 2.0 * e["ke"][1000:].mean() / g < 1.2          # NVE does not heat up

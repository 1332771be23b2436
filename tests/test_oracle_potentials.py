"""Pins for the oracle's other short-range pair potentials (Mie, WCA, Yukawa,
Gaussian; Section 3.1 lists them beside LJ, without formulas).

Each pin is a property the textbook potential has, not a retyped formula:

* Mie(n, m): with n = 12, m = 6 it is the 12-6 LJ potential; its minimum lies at
  r = sigma (n/m)^(1/(n-m)) with depth exactly -eps (what the prefactor is for),
  for integer and non-integer exponents;
* WCA: the 12-6 potential cut at its minimum, whatever the rcut table says;
  V(sigma) = eps, V >= 0 and repulsive inside the cut, nothing beyond it;
* Yukawa: kappa = 0 is the Coulomb pair; r V(r) solves the screened-Poisson
  radial equation (r V)'' = kappa^2 (r V);
* Gaussian: ln V is linear in r^2 with slope -1/(2 sigma^2), and V(0) = eps;
* for every potential on a two-type mixture: the energy vanishes continuously at
  r_cut (the shift), Newton's third law, F = -grad U by central differences, and
  the virial as the strain derivative of U.
"""
import math

import numpy as np
import pytest

from paper_1308_5587_gb300 import workloads as wl

TWO = (np.array([[1.0, 1.2], [1.2, 0.8]]), np.array([[1.0, 0.9], [0.9, 0.85]]))


def mixture(kind):
    """A two-type pair table for each potential (symmetric, per-pair parameters)."""
    eps, sig = TWO
    if kind == "lj":
        return {"eps": eps, "sigma": sig, "rcut": 2.5 * sig}
    if kind == "mie":
        return {"potential": "mie", "eps": eps, "sigma": sig, "rcut": 2.5 * sig,
                "mie_n": np.array([[12.0, 10.0], [10.0, 9.5]]),
                "mie_m": np.array([[6.0, 6.0], [6.0, 5.5]])}
    if kind == "wca":
        return {"potential": "wca", "eps": eps, "sigma": sig, "rcut": None}
    if kind == "yukawa":
        return {"potential": "yukawa", "eps": eps, "sigma": None,
                "rcut": np.array([[2.5, 2.2], [2.2, 2.0]]),
                "kappa": np.array([[1.0, 1.5], [1.5, 0.8]])}
    return {"potential": "gauss", "eps": eps, "sigma": sig, "rcut": 2.8 * sig}


KINDS = ["mie", "wca", "yukawa", "gauss"]


def single(kind, eps=1.0, sigma=1.0, rcut=2.5, **kw):
    p = {"potential": kind, "eps": np.array([[eps]]), "sigma": np.array([[sigma]]),
         "rcut": np.array([[rcut]])}
    for k, v in kw.items():
        p[k] = np.array([[v]])
    return p


def pair_energy_force(oracle, p, r, L=100.0):
    """(U, F_x on particle 0) for two particles r apart along x (d_01 = +r)."""
    pos = np.zeros((2, 3))
    pos[1, 0] = -r
    F, U, *_ = oracle.forces(pos, np.full(3, L), None, p)
    assert np.array_equal(F[0], -F[1])
    return U, F[0, 0]


# --- Mie ---------------------------------------------------------------------------

def test_mie_12_6_is_lennard_jones(oracle):
    w = wl.lj_fluid(500, 1.2, 1.0, seed=21, binary=True)
    lj = w.pairs.as_dict()
    mie = dict(lj, potential="mie", mie_n=np.full((2, 2), 12.0), mie_m=np.full((2, 2), 6.0))
    F0, U0, W0, *_ = oracle.forces(w.pos, w.box, w.types, lj)
    F1, U1, W1, *_ = oracle.forces(w.pos, w.box, w.types, mie)
    assert U1 == pytest.approx(U0, rel=1e-12)
    assert np.abs(F1 - F0).max() <= 1e-12 * np.abs(F0).max()
    assert np.abs(W1 - W0).max() <= 1e-12 * np.abs(W0).max()


@pytest.mark.parametrize("n,m", [(12.0, 6.0), (10.0, 6.0), (14.0, 7.0), (9.5, 5.5), (50.0, 49.0)])
@pytest.mark.parametrize("eps,sigma", [(1.0, 1.0), (0.7, 1.3)])
def test_mie_minimum_position_and_depth(oracle, n, m, eps, sigma):
    # a far cut (45 sigma) leaves a shift below 1e-8 eps
    p = single("mie", eps, sigma, 45.0 * sigma, mie_n=n, mie_m=m)
    r_min = sigma * (n / m) ** (1.0 / (n - m))
    U, F = pair_energy_force(oracle, p, r_min)
    assert U == pytest.approx(-eps, abs=1e-8 * eps)
    assert abs(F) <= 1e-9 * eps / sigma
    # repulsive inside the minimum, attractive outside it
    assert pair_energy_force(oracle, p, 0.98 * r_min)[1] > 0
    assert pair_energy_force(oracle, p, 1.02 * r_min)[1] < 0


# --- WCA ---------------------------------------------------------------------------

@pytest.mark.parametrize("eps,sigma", [(1.0, 1.0), (1.5, 0.8)])
def test_wca_closed_forms(oracle, eps, sigma):
    p = single("wca", eps, sigma, rcut=2.5 * sigma)   # the rcut table is not used
    rc = 2.0 ** (1.0 / 6.0) * sigma
    assert oracle.cutoffs(p)[0, 0] == pytest.approx(rc, rel=1e-15)
    U, F = pair_energy_force(oracle, p, sigma)
    assert U == pytest.approx(eps, rel=1e-13)              # 4 eps (1 - 1) + eps
    assert F == pytest.approx(24 * eps / sigma, rel=1e-13)
    for r in np.linspace(0.9 * sigma, rc * (1 - 1e-9), 25):
        U, F = pair_energy_force(oracle, p, r)
        assert U >= 0 and F > 0
    # continuous at the cut (value and force vanish there) and nothing beyond it
    U, F = pair_energy_force(oracle, p, rc * (1 - 1e-7))
    assert abs(U) < 1e-11 * eps and abs(F) < 1e-5 * eps / sigma
    assert pair_energy_force(oracle, p, rc * (1 + 1e-9)) == (0.0, 0.0)
    assert pair_energy_force(oracle, p, 2.0 * sigma) == (0.0, 0.0)


def test_wca_is_lj_cut_at_the_minimum(oracle):
    w = wl.lj_fluid(400, 1.2, 1.0, seed=22, binary=True)
    eps, sig = w.pairs.eps, w.pairs.sigma
    wca = {"potential": "wca", "eps": eps, "sigma": sig, "rcut": None}
    lj = {"eps": eps, "sigma": sig, "rcut": oracle.cutoffs(wca)}
    F0, U0, W0, *_ = oracle.forces(w.pos, w.box, w.types, lj)
    F1, U1, W1, *_ = oracle.forces(w.pos, w.box, w.types, wca)
    assert U1 == U0 and np.array_equal(F1, F0) and np.array_equal(W1, W0)


# --- Yukawa ------------------------------------------------------------------------

@pytest.mark.parametrize("eps", [1.0, 2.5])
def test_yukawa_without_screening_is_coulomb(oracle, eps):
    rc = 3.0
    p = single("yukawa", eps, 1.0, rc, kappa=0.0)
    for r in (0.5, 1.0, 1.7, 2.9):
        U, F = pair_energy_force(oracle, p, r)
        assert U == pytest.approx(eps / r - eps / rc, rel=1e-14)
        assert F == pytest.approx(eps / r ** 2, rel=1e-14)


@pytest.mark.parametrize("kappa", [0.5, 2.0])
def test_yukawa_solves_the_screened_poisson_equation(oracle, kappa):
    # far cut: the shift is below 1e-8 of the values tested
    p = single("yukawa", 1.3, 1.0, 30.0, kappa=kappa)
    h = 1e-3
    g = lambda r: r * pair_energy_force(oracle, p, r)[0]
    for r in (0.8, 1.3, 2.0):
        g2 = (g(r + h) - 2 * g(r) + g(r - h)) / h ** 2
        assert g2 == pytest.approx(kappa ** 2 * g(r), rel=1e-5)
    # and decays: the growing solution exp(+kappa r) is absent
    assert g(3.0) < g(2.0) < g(1.0)


# --- Gaussian ----------------------------------------------------------------------

@pytest.mark.parametrize("eps,sigma", [(1.0, 1.0), (0.4, 1.6)])
def test_gaussian_log_is_linear_in_r2(oracle, eps, sigma):
    p = single("gauss", eps, sigma, 12.0 * sigma)   # shift ~ exp(-72)
    rs = np.array([0.5, 1.0, 1.5, 2.2]) * sigma
    lnU = np.log([pair_energy_force(oracle, p, r)[0] for r in rs])
    slopes = np.diff(lnU) / np.diff(rs ** 2)
    assert np.allclose(slopes, -1.0 / (2 * sigma ** 2), rtol=1e-10, atol=0)
    U, F = pair_energy_force(oracle, p, 1e-5 * sigma)
    assert U == pytest.approx(eps, rel=1e-9)
    assert F == pytest.approx(1e-5 * eps / sigma, rel=1e-6)   # linear near r = 0


# --- every potential: shift, third law, gradient, virial -----------------------------

@pytest.mark.parametrize("kind", KINDS)
def test_energy_vanishes_at_the_cut(oracle, kind):
    p = mixture(kind)
    rc = oracle.cutoffs(p)
    for a, b in [(0, 0), (0, 1), (1, 1)]:
        pos = np.zeros((2, 3))
        pos[1, 1] = -rc[a, b] * (1 - 1e-10)
        F, U, *_ = oracle.forces(pos, np.full(3, 20.0), np.array([a, b], np.int32), p)
        assert abs(U) < 1e-8
        pos[1, 1] = -rc[a, b] * (1 + 1e-10)
        F, U, *_ = oracle.forces(pos, np.full(3, 20.0), np.array([a, b], np.int32), p)
        assert U == 0 and not F.any()


def _fluid_clear_of_cut(oracle, kind, n, rho, seed0, margin=1e-4):
    p = mixture(kind)
    rc = oracle.cutoffs(p)
    for seed in range(seed0, seed0 + 200):
        w = wl.lj_fluid(n, rho, 1.0, seed=seed, binary=True, jitter=0.2)
        d = w.pos[:, None, :] - w.pos[None, :, :]
        d -= w.box * np.rint(d / w.box)
        r = np.sqrt((d * d).sum(-1))
        np.fill_diagonal(r, 1e9)
        if np.abs(r - rc[w.types[:, None], w.types[None, :]]).min() > margin:
            return w, p
    raise AssertionError("no configuration clear of the cut")


@pytest.mark.parametrize("kind", KINDS)
def test_newton_third_law(oracle, kind):
    w, p = _fluid_clear_of_cut(oracle, kind, 400, 0.9, 500)
    F, *_ = oracle.forces(w.pos, w.box, w.types, p)
    assert np.abs(F).max() > 0
    assert np.linalg.norm(F.sum(0)) <= 1e-10 * np.linalg.norm(F, axis=1).sum()


@pytest.mark.parametrize("kind", KINDS)
def test_force_is_minus_energy_gradient(oracle, kind):
    w, p = _fluid_clear_of_cut(oracle, kind, 64, 0.6, 700)
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
    assert frms > 0
    assert np.abs(F + grad).max() <= 1e-6 * frms


@pytest.mark.parametrize("kind", KINDS)
def test_virial_is_strain_derivative(oracle, kind):
    w, p = _fluid_clear_of_cut(oracle, kind, 64, 0.6, 900)
    _, U, W, *_ = oracle.forces(w.pos, w.box, w.types, p)
    h = 1e-7
    for a, c in ((0, 0), (1, 3), (2, 5)):
        s = np.ones(3); s[a] += h
        up = oracle.forces(w.pos * s, w.box * s, w.types, p)[1]
        s[a] -= 2 * h
        dn = oracle.forces(w.pos * s, w.box * s, w.types, p)[1]
        assert -(up - dn) / (2 * h) == pytest.approx(W[c], rel=1e-6, abs=1e-6)
    # shear of an isolated cluster (no boundary pairs): the off-diagonal terms
    cl = wl.lj_fluid(27, 0.8, 1.0, seed=7, jitter=0.1, binary=True)
    big = np.full(3, 60.0)
    _, U, W, *_ = oracle.forces(cl.pos, big, cl.types, p)
    for (a, b), c in (((0, 1), 1), ((0, 2), 2), ((1, 2), 4)):
        def energy(gm):
            x = cl.pos.copy(); x[:, a] += gm * cl.pos[:, b]
            return oracle.forces(x, big, cl.types, p)[1]
        assert -(energy(h) - energy(-h)) / (2 * h) == pytest.approx(W[c], rel=1e-6, abs=1e-6)


@pytest.mark.parametrize("kind", KINDS)
def test_missing_tables_are_rejected(oracle, kind):
    p = mixture(kind)
    need = {"mie": "mie_n", "wca": "sigma", "yukawa": "kappa", "gauss": "sigma"}[kind]
    bad = dict(p, **{need: None})
    pos = np.zeros((2, 3)); pos[1, 0] = 1.0
    with pytest.raises(ValueError):
        oracle.forces(pos, np.full(3, 20.0), np.array([0, 1], np.int32), bad)

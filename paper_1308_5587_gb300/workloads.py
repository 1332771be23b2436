"""Seeded synthetic inputs shaped like the paper's LJ workloads.

This module holds no arithmetic of the MD method (no forces, no integration, no
neighbour search): it only draws initial conditions and parameter tables.  It is
the one module that both the CUDA path's callers and the CPU oracle's callers
use, so that both sides see bit-identical inputs.

Recipe (paper silent on all of it; the paper's own LJ benchmark is a
synthetic liquid, Section 5):
  * FCC lattice with n = ceil((N/4)^(1/3)) unit cells per side in a cubic box
    of side L = (N/rho)^(1/3); if 4 n^3 > N a seeded subset of N sites is kept
    (in lattice order); the lattice is offset by a/4 so no site sits on a face;
  * uniform jitter in [-jitter, +jitter) per component (default 0.05 sigma);
  * velocities N(0, sqrt(T/m)) per component, mean removed, then rescaled so
    that 2K/(3N-3) equals T exactly;
  * Kob-Andersen types: exactly round(0.8 N) type A (0) in a seeded random
    permutation, the rest type B (1);
  * numpy PCG64 streams spawned from one seed; base seed 20130826, replica or
    request k uses base + k.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 20130826


@dataclass
class PairTable:
    """Per type-pair eps, sigma, r_cut (ntypes x ntypes, symmetric), and the pair
    potential with its extra tables (Mie exponents, Yukawa screening)."""
    eps: np.ndarray
    sigma: np.ndarray
    rcut: np.ndarray
    potential: str = "lj"
    mie_n: np.ndarray | None = None
    mie_m: np.ndarray | None = None
    kappa: np.ndarray | None = None

    @property
    def ntypes(self) -> int:
        return int(self.eps.shape[0])

    def potential_kw(self):
        """The potential and its extra tables as keyword arguments."""
        return {"potential": self.potential, "mie_n": self.mie_n, "mie_m": self.mie_m,
                "kappa": self.kappa}

    def as_dict(self):
        return {"eps": self.eps, "sigma": self.sigma, "rcut": self.rcut, **self.potential_kw()}


def lj_single(eps=1.0, sigma=1.0, rcut=2.5) -> PairTable:
    one = np.ones((1, 1))
    return PairTable(eps * one, sigma * one, rcut * one)


def mie_single(n=10.0, m=6.0, eps=1.0, sigma=1.0, rcut=2.5) -> PairTable:
    one = np.ones((1, 1))
    return PairTable(eps * one, sigma * one, rcut * one, "mie", n * one, m * one)


def wca_single(eps=1.0, sigma=1.0) -> PairTable:
    """12-6 LJ cut at its minimum 2^(1/6) sigma (the rcut table is not read)."""
    one = np.ones((1, 1))
    return PairTable(eps * one, sigma * one, 2.0 ** (1.0 / 6.0) * sigma * one, "wca")


def yukawa_single(eps=1.0, kappa=1.0, rcut=2.5) -> PairTable:
    one = np.ones((1, 1))
    return PairTable(eps * one, one, rcut * one, "yukawa", kappa=kappa * one)


def gauss_single(eps=1.0, sigma=1.0, rcut=3.0) -> PairTable:
    one = np.ones((1, 1))
    return PairTable(eps * one, sigma * one, rcut * one, "gauss")


def kob_andersen(rcut_over_sigma=2.5) -> PairTable:
    """Kob-Andersen 80:20 binary mixture, r_cut = 2.5 sigma_ij."""
    eps = np.array([[1.0, 1.5], [1.5, 0.5]])
    sig = np.array([[1.0, 0.8], [0.8, 0.88]])
    return PairTable(eps, sig, rcut_over_sigma * sig)


@dataclass
class Workload:
    """One LJ system: initial state plus run parameters (tag order)."""
    pos: np.ndarray            # (N, 3) float64
    vel: np.ndarray            # (N, 3) float64
    types: np.ndarray          # (N,) int32
    box: np.ndarray            # (3,) float64
    pairs: PairTable
    r_buff: float = 0.4
    dt: float = 0.005
    mass: float = 1.0
    seed: int = BASE_SEED
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def _streams(seed: int, k: int):
    return [np.random.Generator(np.random.PCG64(s)) for s in np.random.SeedSequence(seed).spawn(k)]


def fcc_positions(n: int, rho: float, rng: np.random.Generator, jitter: float = 0.05):
    """FCC sites (subset if needed) + uniform jitter in a centred cubic box."""
    if n < 1:
        return np.zeros((0, 3)), np.full(3, 1.0)
    L = (n / rho) ** (1.0 / 3.0)
    m = int(math.ceil((n / 4.0) ** (1.0 / 3.0) - 1e-9))
    a = L / m
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    g = np.arange(m)
    cells = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    sites = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a
    if sites.shape[0] > n:
        keep = np.sort(rng.choice(sites.shape[0], size=n, replace=False))
        sites = sites[keep]
    pos = sites - 0.5 * L + 0.25 * a
    pos = pos + rng.uniform(-jitter, jitter, size=pos.shape)
    return pos, np.full(3, L)


def maxwell_boltzmann(n: int, T: float, mass: float, rng: np.random.Generator):
    """Gaussian velocities, zero net momentum, rescaled to 2K/(3N-3) = T."""
    v = rng.normal(0.0, math.sqrt(T / mass), size=(n, 3))
    if n < 2:
        return np.zeros((n, 3))
    v -= v.mean(axis=0)
    k = 0.5 * mass * float(np.sum(v * v))
    v *= math.sqrt(T * (3 * n - 3) / (2.0 * k))
    return v


def ka_types(n: int, rng: np.random.Generator, frac_a: float = 0.8):
    t = np.ones(n, np.int32)
    t[: int(round(frac_a * n))] = 0
    return rng.permutation(t).astype(np.int32)


def lj_fluid(n: int, rho: float, T: float, seed: int = BASE_SEED, pairs: PairTable | None = None,
             r_buff: float = 0.4, dt: float = 0.005, mass: float = 1.0, jitter: float = 0.05,
             binary: bool = False) -> Workload:
    rp, rv, rt = _streams(seed, 3)
    pos, box = fcc_positions(n, rho, rp, jitter)
    vel = maxwell_boltzmann(n, T, mass, rv)
    types = ka_types(n, rt) if binary else np.zeros(n, np.int32)
    pairs = pairs or (kob_andersen() if binary else lj_single())
    return Workload(pos, vel, types, box, pairs, r_buff, dt, mass, seed,
                    {"rho": rho, "T": T, "jitter": jitter})


# --- the five workload shapes -------------------------------------------------

def plain_fp64_4k(seed: int = BASE_SEED) -> Workload:
    """LJ fluid N=4,000, rho 0.84, T 1.2, r_cut 2.5 (shifted), r_buff 0.4, dt 0.005."""
    return lj_fluid(4000, 0.84, 1.2, seed)


def lj_64k(seed: int = BASE_SEED) -> Workload:
    """LJ fluid N=64,000, rho 0.84, T 1.2, r_cut 2.5, r_buff 0.4, dt 0.005."""
    return lj_fluid(64000, 0.84, 1.2, seed)


def ka_1m(seed: int = BASE_SEED, n: int = 1_000_000) -> Workload:
    """Kob-Andersen 80:20, N=10^6, rho 1.2, T 1.0, r_cut 2.5 sigma_ij, r_buff 0.3."""
    return lj_fluid(n, 1.2, 1.0, seed, binary=True, r_buff=0.3)


def paper_lj_64k(seed: int = BASE_SEED) -> Workload:
    """Section 5's LJ benchmark shape: N=64,000, rho 0.382, kT 1.2, r_cut 3.0 (shifted),
    dt 0.005, NVT with tau 1.0 (Listing 1's coupling time); r_buff 0.4 (not given)."""
    w = lj_fluid(64000, 0.382, 1.2, seed, pairs=lj_single(rcut=3.0))
    w.meta.update(integrator="nvt", kT=1.2, tau=1.0)
    return w


def potential_64k(kind: str, seed: int = BASE_SEED) -> Workload:
    """The LJ 64k geometry (N=64,000, rho 0.84, T 1.2, r_buff 0.4, dt 0.005) with one of
    the other pair potentials: Mie 10-6 (r_cut 2.5), WCA, Yukawa (eps 1, kappa 1,
    r_cut 2.5) or the Gaussian core (eps 1, sigma 1, r_cut 3.0)."""
    pairs = {"mie": (mie_single(10.0, 6.0), "n=10 m=6 rc=2.5"),
             "wca": (wca_single(), "rc=2^(1/6)"),
             "yukawa": (yukawa_single(1.0, 1.0, 2.5), "eps=1 kappa=1 rc=2.5"),
             "gauss": (gauss_single(1.0, 1.0, 3.0), "eps=1 sigma=1 rc=3.0")}[kind]
    w = lj_fluid(64000, 0.84, 1.2, seed, pairs=pairs[0])
    w.meta["pair"] = pairs[1]
    return w


def colloid_mixture(n_small: int, ratio: float = 5.0, phi_small: float = 0.2,
                    phi_large: float = 0.2, T: float = 1.0, seed: int = BASE_SEED,
                    r_buff: float = 0.4, dt: float = 0.002) -> Workload:
    """Size-disperse binary WCA mixture (the case the tree list is for, Section 5):
    small particles of diameter 1 (type 0) and large ones of diameter `ratio`
    (type 1) at volume fractions phi_small and phi_large; sigma_ij = (d_i + d_j)/2,
    eps = 1, r_cut,ij = 2^(1/6) sigma_ij, mass 1.

    Large particles sit on a simple cubic lattice (a seeded subset of its sites,
    jitter 0.05); small ones on a seeded subset of the FCC sites of spacing set by
    the small density that keep a distance >= 0.55 (1 + ratio) from every large one
    (jitter 0.05)."""
    rp, rv, rs = _streams(seed, 3)
    vs, vl = math.pi / 6.0, math.pi / 6.0 * ratio ** 3
    n_large = max(1, int(round(n_small * (phi_large / vl) / (phi_small / vs))))
    vol = n_small * vs / phi_small
    L = vol ** (1.0 / 3.0)
    box = np.full(3, L)
    m = int(math.ceil(n_large ** (1.0 / 3.0) - 1e-9))
    g = np.arange(m)
    big = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) * (L / m)
    big = big[np.sort(rs.choice(big.shape[0], n_large, replace=False))] - 0.5 * L
    big += rs.uniform(-0.05, 0.05, big.shape)
    # small-particle sites: every FCC site of m^3 cells (1.1 times as many sites as
    # small particles outside the excluded shells), minus those shells
    rmin = 0.55 * (1.0 + ratio)
    excl = min(0.9, n_large * 4.0 / 3.0 * math.pi * rmin ** 3 / vol)
    m = int(math.ceil((1.1 * n_small / (1.0 - excl) / 4.0) ** (1.0 / 3.0) - 1e-9))
    a = L / m
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    g = np.arange(m)
    cells = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    sites = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a - 0.5 * L + 0.25 * a
    from scipy.spatial import cKDTree   # periodic search of the excluded sites
    tree = cKDTree(np.mod(sites + 0.5 * L, L), boxsize=L)
    drop = tree.query_ball_point(np.mod(big + 0.5 * L, L), rmin)
    keep = np.ones(sites.shape[0], bool)
    for d in drop:
        keep[d] = False
    sites = sites[keep]
    if sites.shape[0] < n_small:
        raise ValueError("colloid_mixture: too few free sites for the small particles")
    small = sites[np.sort(rp.choice(sites.shape[0], n_small, replace=False))]
    small += rp.uniform(-0.05, 0.05, small.shape)
    pos = np.concatenate([small, big])
    pos -= L * np.floor((pos + 0.5 * L) / L)
    n = pos.shape[0]
    types = np.concatenate([np.zeros(n_small, np.int32), np.ones(n_large, np.int32)])
    vel = maxwell_boltzmann(n, T, 1.0, rv)
    d = np.array([1.0, ratio])
    sig = 0.5 * (d[:, None] + d[None, :])
    pairs = PairTable(np.ones((2, 2)), sig, 2.0 ** (1.0 / 6.0) * sig, "wca")
    return Workload(pos, vel, types, box, pairs, r_buff, dt, 1.0, seed,
                    {"ratio": ratio, "phi_small": phi_small, "phi_large": phi_large, "T": T,
                     "n_large": n_large})


def replica_params(count: int = 256, seed: int = BASE_SEED, n_lo: int = 500, n_hi: int = 20000):
    """(N_k, rho_k, T_k, seed_k) for the batched-ensemble shape."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = np.rint(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), count))).astype(int)
    rhos = rng.uniform(0.7, 0.9, count)
    ts = rng.uniform(0.8, 1.5, count)
    return [(int(ns[k]), float(rhos[k]), float(ts[k]), seed + 1 + k) for k in range(count)]


def replica(n: int, rho: float, T: float, seed: int) -> Workload:
    return lj_fluid(n, rho, T, seed, r_buff=0.4)


def request_trace(count: int = 1000, rate: float = 50.0, seed: int = BASE_SEED,
                  n_lo: int = 256, n_hi: int = 200000, steps_lo: int = 1000,
                  steps_hi: int = 50000):
    """Poisson arrival trace: list of dicts(arrival, n, rho, T, steps, seed)."""
    rng = np.random.Generator(np.random.PCG64(seed + 7))
    gaps = rng.exponential(1.0 / rate, count)
    t = np.cumsum(gaps)
    ns = np.rint(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), count))).astype(int)
    rhos = rng.uniform(0.7, 0.9, count)
    ts = rng.uniform(0.8, 1.5, count)
    steps = rng.integers(steps_lo, steps_hi + 1, count)
    return [dict(arrival=float(t[k]), n=int(ns[k]), rho=float(rhos[k]), T=float(ts[k]),
                 steps=int(steps[k]), seed=seed + 100000 + k) for k in range(count)]

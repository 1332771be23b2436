"""Plain FP64 CPU oracle for the Lennard-Jones MD hot path (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: the product library never imports, links or calls
anything here.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` / ``--impl reference`` leg use it.  It shares no code with the
CUDA path (``paper_1308_5587_gb300``) and imports nothing from it.

The arithmetic lives in ``lj_oracle.c``; its header states every definition
(minimum image, energy-shifted LJ and the other short-range pair potentials
Section 3.1 lists beside it -- Mie, WCA, Yukawa, Gaussian --, virial, velocity
Verlet, Nose-Hoover NVT, brute-force neighbour pairs) and which readings the
HOOMD-blue paper leaves open (Section 3.1 names the LJ pair force, the cell
neighbour list and the NVE integrator; Section 7.1 names force, energy and virial
as what is checked).

A pair-parameter dict holds ``eps``, ``sigma``, ``rcut`` (ntypes x ntypes or
scalars) and optionally ``potential`` ("lj" default, "mie", "wca", "yukawa",
"gauss"), ``mie_n`` / ``mie_m`` (Mie exponents) and ``kappa`` (Yukawa screening).

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(closed forms, finite differences, invariants, brute force against an
independent k-d tree, an independent ODE solver); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lj_oracle.c")
_LIB = os.path.join(_HERE, "liblj_oracle.so")
_lib = None


def build(force: bool = False, defines: tuple[str, ...] = (), out: str | None = None) -> str:
    """Compile lj_oracle.c with gcc (-O2, OpenMP, no fused multiply-add)."""
    out = out or _LIB
    if not force and not defines and os.path.exists(out) and \
            os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           *[f"-D{d}" for d in defines], _SRC, "-o", out + ".tmp", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


def _bind(lib):
    dp = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
    ip = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
    lp = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
    i64, i32 = C.c_int64, C.c_int32
    vp = C.c_void_p
    lib.oracle_set_threads.argtypes = [C.c_int]
    lib.oracle_get_threads.restype = C.c_int
    pt = [i32, i32, vp, vp, vp, vp, vp]   # ntypes, kind, eps, sigma, rcut, pa, pb
    lib.oracle_forces.argtypes = [i64, dp, dp, ip, *pt, dp, vp, vp, vp, vp]
    lib.oracle_forces_subset.argtypes = [i64, dp, dp, ip, *pt, i64, lp, dp, vp, vp]
    lib.oracle_cutoffs.argtypes = [*pt, dp]
    lib.oracle_neighbors.argtypes = [i64, dp, dp, ip, i32, dp, i64, vp, vp,
                                     C.POINTER(C.c_int64)]
    lib.oracle_wrap.argtypes = [i64, dp, dp, ip]
    lib.oracle_kinetic.argtypes = [i64, dp, C.c_double]
    lib.oracle_kinetic.restype = C.c_double
    lib.oracle_vv.argtypes = [i64, dp, dp, dp, ip, ip, *pt, C.c_double, C.c_double, i64, dp,
                              vp, vp]
    lib.oracle_thermo.argtypes = [i64, dp, C.c_double, dp, C.POINTER(C.c_double),
                                  C.POINTER(C.c_double)]
    lib.oracle_nvt.argtypes = [i64, dp, dp, dp, ip, ip, *pt, C.c_double,
                               C.c_double, C.c_double, C.c_double, i64, dp,
                               C.POINTER(C.c_double), C.POINTER(C.c_double), vp, vp, vp, vp]
    return lib


def load(path: str | None = None):
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if path is not None:
        return _bind(C.CDLL(path))
    if _lib is None:
        _lib = _bind(C.CDLL(build()))
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


POTENTIALS = {"lj": 0, "mie": 1, "wca": 2, "yukawa": 3, "gauss": 4}


class _Tables:
    """The pair model as the C functions take it: (ntypes, kind, eps, sigma, rcut,
    pa, pb); absent tables are passed as NULL."""

    def __init__(self, params, ntypes):
        def tab(key):
            if params.get(key) is None:
                return None
            a = np.broadcast_to(np.asarray(params[key], np.float64), (ntypes, ntypes))
            return np.ascontiguousarray(a).ravel().copy()
        self.kind = POTENTIALS[params.get("potential", "lj")]
        self.tables = [tab("eps"), tab("sigma"), tab("rcut")]
        if self.kind == POTENTIALS["mie"]:
            self.tables += [tab("mie_n"), tab("mie_m")]
        elif self.kind == POTENTIALS["yukawa"]:
            self.tables += [tab("kappa"), None]
        else:
            self.tables += [None, None]
        self.ntypes = ntypes

    def args(self):
        return [self.ntypes, self.kind, *[_ptr(t) for t in self.tables]]


def _pair_tables(params, ntypes):
    return _Tables(params, ntypes)


def cutoffs(params, lib=None):
    """The cut-off radius of every type pair (ntypes x ntypes): the rcut table,
    except for WCA, whose cut is the LJ minimum 2^(1/6) sigma."""
    lib = lib or load()
    nt = int(np.asarray(params["eps"]).shape[0]) if np.ndim(params["eps"]) == 2 else 1
    t = _Tables(params, nt)
    out = np.zeros(nt * nt)
    if lib.oracle_cutoffs(*t.args(), out):
        raise ValueError("oracle_cutoffs: a table the potential needs is missing")
    return out.reshape(nt, nt)


def _common(pos, box, types, params):
    pos = np.ascontiguousarray(pos, np.float64).reshape(-1, 3)
    box = np.ascontiguousarray(np.broadcast_to(box, (3,)), np.float64)
    n = pos.shape[0]
    types = np.zeros(n, np.int32) if types is None else np.ascontiguousarray(types, np.int32)
    ntypes = int(np.asarray(params["eps"]).shape[0]) if np.ndim(params["eps"]) == 2 else 1
    return pos, box, n, types, ntypes


def set_threads(n: int) -> None:
    load().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(load().oracle_get_threads())


def forces(pos, box, types, params, lib=None):
    """Returns (F[n,3], U, W[6], u_i[n], W_i[n,6]) for the whole system."""
    lib = lib or load()
    pos, box, n, types, nt = _common(pos, box, types, params)
    t = _pair_tables(params, nt)
    F = np.zeros((n, 3))
    U = np.zeros(1)
    W = np.zeros(6)
    ui = np.zeros(n)
    Wi = np.zeros((n, 6))
    rcode = lib.oracle_forces(n, box, pos, types, *t.args(), F, _ptr(U), _ptr(W), _ptr(ui),
                              _ptr(Wi))
    if rcode:
        raise ValueError(f"oracle_forces failed ({rcode})")
    return F, float(U[0]), W, ui, Wi


def forces_subset(pos, box, types, params, idx, lib=None):
    """Per-particle (F[m,3], u[m], W[m,6]) for the particles listed in idx."""
    lib = lib or load()
    pos, box, n, types, nt = _common(pos, box, types, params)
    t = _pair_tables(params, nt)
    idx = np.ascontiguousarray(idx, np.int64)
    m = idx.shape[0]
    F = np.zeros((m, 3))
    u = np.zeros(m)
    W = np.zeros((m, 6))
    rcode = lib.oracle_forces_subset(n, box, pos, types, *t.args(), m, idx, F, _ptr(u),
                                     _ptr(W))
    if rcode:
        raise ValueError(f"oracle_forces_subset failed ({rcode})")
    return F, u, W


def neighbors(pos, box, types, rlist, lib=None):
    """All pairs i<j with min-image r < rlist[ti, tj]: (pairs[M,2] int32, r[M])."""
    lib = lib or load()
    pos = np.ascontiguousarray(pos, np.float64).reshape(-1, 3)
    n = pos.shape[0]
    box = np.ascontiguousarray(np.broadcast_to(box, (3,)), np.float64)
    types = np.zeros(n, np.int32) if types is None else np.ascontiguousarray(types, np.int32)
    rl = np.atleast_2d(np.asarray(rlist, np.float64))
    nt = rl.shape[0]
    rl = np.ascontiguousarray(rl).ravel()
    cnt = C.c_int64(0)
    cap = 0
    while True:
        pairs = np.zeros((max(cap, 1), 2), np.int32)
        r = np.zeros(max(cap, 1))
        rcode = lib.oracle_neighbors(n, box, pos, types, nt, rl, cap, _ptr(pairs), _ptr(r),
                                     C.byref(cnt))
        if rcode:
            raise ValueError(f"oracle_neighbors failed ({rcode})")
        if cnt.value <= cap:
            return pairs[:cnt.value].copy(), r[:cnt.value].copy()
        cap = cnt.value


def wrap(pos, box, image=None, lib=None):
    lib = lib or load()
    pos = np.array(pos, np.float64).reshape(-1, 3)
    box = np.ascontiguousarray(np.broadcast_to(box, (3,)), np.float64)
    image = np.zeros(pos.shape, np.int32) if image is None else np.array(image, np.int32)
    lib.oracle_wrap(pos.shape[0], box, pos, image)
    return pos, image


def kinetic(vel, mass=1.0, lib=None):
    lib = lib or load()
    vel = np.ascontiguousarray(vel, np.float64).reshape(-1, 3)
    return float(lib.oracle_kinetic(vel.shape[0], vel, float(mass)))


def thermo(n, box, ke, virial, lib=None):
    """(T, P) from the kinetic energy and the virial tensor."""
    lib = lib or load()
    box = np.ascontiguousarray(np.broadcast_to(box, (3,)), np.float64)
    T = C.c_double(0)
    P = C.c_double(0)
    lib.oracle_thermo(int(n), box, float(ke), np.ascontiguousarray(virial, np.float64),
                      C.byref(T), C.byref(P))
    return T.value, P.value


def vv_run(pos, vel, box, types, params, mass, dt, nsteps, image=None, series=False, lib=None):
    """Velocity-Verlet NVE run.  Returns dict(pos, vel, image, force[, pe, ke])."""
    lib = lib or load()
    pos, box, n, types, nt = _common(pos, box, types, params)
    pos = pos.copy()
    vel = np.array(vel, np.float64).reshape(-1, 3)
    image = np.zeros((n, 3), np.int32) if image is None else np.array(image, np.int32)
    t = _pair_tables(params, nt)
    F = np.zeros((n, 3))
    pe = np.zeros(nsteps + 1) if series else None
    ke = np.zeros(nsteps + 1) if series else None
    rcode = lib.oracle_vv(n, box, pos, vel, image, types, *t.args(), float(mass), float(dt),
                          int(nsteps), F, _ptr(pe), _ptr(ke))
    if rcode:
        raise ValueError(f"oracle_vv failed ({rcode})")
    out = dict(pos=pos, vel=vel, image=image, force=F)
    if series:
        out["pe"], out["ke"] = pe, ke
    return out


def nvt_run(pos, vel, box, types, params, mass, dt, kT, tau, nsteps, xi=0.0, eta=0.0,
            image=None, series=False, lib=None):
    """Nose-Hoover (MTK) NVT run.  Returns dict(pos, vel, image, force, xi, eta
    [, pe, ke, xis, etas]); H = K + U + g kT (tau^2 xi^2 / 2 + eta), g = 3N - 3, is
    its conserved quantity."""
    lib = lib or load()
    pos, box, n, types, nt = _common(pos, box, types, params)
    pos = pos.copy()
    vel = np.array(vel, np.float64).reshape(-1, 3)
    image = np.zeros((n, 3), np.int32) if image is None else np.array(image, np.int32)
    t = _pair_tables(params, nt)
    F = np.zeros((n, 3))
    ser = [np.zeros(nsteps + 1) if series else None for _ in range(4)]
    x, e = C.c_double(xi), C.c_double(eta)
    rcode = lib.oracle_nvt(n, box, pos, vel, image, types, *t.args(), float(mass),
                           float(dt), float(kT), float(tau), int(nsteps), F, C.byref(x),
                           C.byref(e), *[_ptr(a) for a in ser])
    if rcode:
        raise ValueError(f"oracle_nvt failed ({rcode})")
    out = dict(pos=pos, vel=vel, image=image, force=F, xi=x.value, eta=e.value)
    if series:
        out["pe"], out["ke"], out["xis"], out["etas"] = ser
    return out

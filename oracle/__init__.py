"""Plain FP64 CPU oracle for the Lennard-Jones MD hot path (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: the product library never imports, links or calls
anything here.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` / ``--impl reference`` leg use it.  It shares no code with the
CUDA path (``paper_1308_5587_gb300``) and imports nothing from it.

The arithmetic lives in ``lj_oracle.c``; its header states every definition
(minimum image, energy-shifted LJ, virial, velocity Verlet, brute-force
neighbour pairs) and which readings the HOOMD-blue paper leaves open
(Section 3.1 names the LJ pair force, the cell neighbour list and the NVE
integrator; Section 7.1 names force, energy and virial as what is checked).

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
    lib.oracle_forces.argtypes = [i64, dp, dp, ip, i32, dp, dp, dp, dp, vp, vp, vp, vp]
    lib.oracle_forces_subset.argtypes = [i64, dp, dp, ip, i32, dp, dp, dp, i64, lp, dp, vp, vp]
    lib.oracle_neighbors.argtypes = [i64, dp, dp, ip, i32, dp, i64, vp, vp,
                                     C.POINTER(C.c_int64)]
    lib.oracle_wrap.argtypes = [i64, dp, dp, ip]
    lib.oracle_kinetic.argtypes = [i64, dp, C.c_double]
    lib.oracle_kinetic.restype = C.c_double
    lib.oracle_vv.argtypes = [i64, dp, dp, dp, ip, ip, i32, dp, dp, dp, C.c_double,
                              C.c_double, i64, dp, vp, vp]
    lib.oracle_thermo.argtypes = [i64, dp, C.c_double, dp, C.POINTER(C.c_double),
                                  C.POINTER(C.c_double)]
    lib.oracle_nvt.argtypes = [i64, dp, dp, dp, ip, ip, i32, dp, dp, dp, C.c_double,
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


def _pair_tables(params, ntypes):
    eps = np.ascontiguousarray(np.broadcast_to(params["eps"], (ntypes, ntypes)), np.float64)
    sig = np.ascontiguousarray(np.broadcast_to(params["sigma"], (ntypes, ntypes)), np.float64)
    rc = np.ascontiguousarray(np.broadcast_to(params["rcut"], (ntypes, ntypes)), np.float64)
    return eps.ravel().copy(), sig.ravel().copy(), rc.ravel().copy()


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
    eps, sig, rc = _pair_tables(params, nt)
    F = np.zeros((n, 3))
    U = np.zeros(1)
    W = np.zeros(6)
    ui = np.zeros(n)
    Wi = np.zeros((n, 6))
    rcode = lib.oracle_forces(n, box, pos, types, nt, eps, sig, rc, F, _ptr(U), _ptr(W),
                              _ptr(ui), _ptr(Wi))
    if rcode:
        raise ValueError(f"oracle_forces failed ({rcode})")
    return F, float(U[0]), W, ui, Wi


def forces_subset(pos, box, types, params, idx, lib=None):
    """Per-particle (F[m,3], u[m], W[m,6]) for the particles listed in idx."""
    lib = lib or load()
    pos, box, n, types, nt = _common(pos, box, types, params)
    eps, sig, rc = _pair_tables(params, nt)
    idx = np.ascontiguousarray(idx, np.int64)
    m = idx.shape[0]
    F = np.zeros((m, 3))
    u = np.zeros(m)
    W = np.zeros((m, 6))
    rcode = lib.oracle_forces_subset(n, box, pos, types, nt, eps, sig, rc, m, idx, F, _ptr(u),
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
    eps, sig, rc = _pair_tables(params, nt)
    F = np.zeros((n, 3))
    pe = np.zeros(nsteps + 1) if series else None
    ke = np.zeros(nsteps + 1) if series else None
    rcode = lib.oracle_vv(n, box, pos, vel, image, types, nt, eps, sig, rc, float(mass),
                          float(dt), int(nsteps), F, _ptr(pe), _ptr(ke))
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
    eps, sig, rc = _pair_tables(params, nt)
    F = np.zeros((n, 3))
    ser = [np.zeros(nsteps + 1) if series else None for _ in range(4)]
    x, e = C.c_double(xi), C.c_double(eta)
    rcode = lib.oracle_nvt(n, box, pos, vel, image, types, nt, eps, sig, rc, float(mass),
                           float(dt), float(kT), float(tau), int(nsteps), F, C.byref(x),
                           C.byref(e), *[_ptr(a) for a in ser])
    if rcode:
        raise ValueError(f"oracle_nvt failed ({rcode})")
    out = dict(pos=pos, vel=vel, image=image, force=F, xi=x.value, eta=e.value)
    if series:
        out["pe"], out["ke"], out["xis"], out["etas"] = ser
    return out

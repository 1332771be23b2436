"""Thin ctypes binding of libgbmd (include/gbmd.h).

Argument marshalling only: every step of the MD path runs in the library's CUDA
kernels.  The module-level functions carry the C names (gbmd_create, gbmd_step,
...); ``System`` and ``Batch`` wrap them for convenience.  PyTorch, when given,
only supplies CUDA stream handles and device pointers.

Loading fails loudly when libgbmd.so has not been built: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgbmd.so")

GBMD_OK = 0
GBMD_FP64 = 0
GBMD_MIXED = 1
STATUS = {0: "OK", -1: "BAD_ARG", -2: "BOX_TOO_SMALL", -3: "OOM", -4: "NLIST_OVERFLOW",
          -5: "NONFINITE", -6: "CUDA", -7: "TIMEOUT", -8: "STATE", -9: "NO_DEVICE"}
PRECISIONS = {"fp64": GBMD_FP64, "mixed": GBMD_MIXED}


class GbmdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
        self.status = STATUS.get(code, str(code))


class gbmd_desc(C.Structure):
    _fields_ = [("n", C.c_int64), ("box", C.c_double * 3), ("pos", C.c_void_p),
                ("vel", C.c_void_p), ("type", C.c_void_p), ("image", C.c_void_p),
                ("ntypes", C.c_int32), ("eps", C.c_void_p), ("sigma", C.c_void_p),
                ("rcut", C.c_void_p), ("r_buff", C.c_double), ("dt", C.c_double),
                ("mass", C.c_double), ("precision", C.c_int32), ("sort_period", C.c_int32),
                ("nlist_capacity", C.c_int32), ("threads_per_particle", C.c_int32),
                ("stream", C.c_void_p), ("device", C.c_int32), ("force_path", C.c_int32),
                ("integrator", C.c_int32), ("kT", C.c_double), ("tau", C.c_double),
                ("potential", C.c_int32), ("mie_n", C.c_void_p), ("mie_m", C.c_void_p),
                ("kappa", C.c_void_p), ("nlist", C.c_int32), ("n_ghost", C.c_int64)]


GBMD_PATH_GLOBAL, GBMD_PATH_STAGED = 0, 1
FORCE_PATHS = {"global": GBMD_PATH_GLOBAL, "staged": GBMD_PATH_STAGED}
GBMD_NVE, GBMD_NVT = 0, 1
INTEGRATORS = {"nve": GBMD_NVE, "nvt": GBMD_NVT}
GBMD_POT_LJ, GBMD_POT_MIE, GBMD_POT_WCA, GBMD_POT_YUKAWA, GBMD_POT_GAUSS = range(5)
POTENTIALS = {"lj": GBMD_POT_LJ, "mie": GBMD_POT_MIE, "wca": GBMD_POT_WCA,
              "yukawa": GBMD_POT_YUKAWA, "gauss": GBMD_POT_GAUSS}
GBMD_NLIST_CELL, GBMD_NLIST_TREE = 0, 1
NLISTS = {"cell": GBMD_NLIST_CELL, "tree": GBMD_NLIST_TREE}


class gbmd_thermo(C.Structure):
    _fields_ = [("step", C.c_int64), ("pe", C.c_double), ("ke", C.c_double),
                ("temperature", C.c_double), ("pressure", C.c_double),
                ("virial", C.c_double * 6), ("w", C.c_double), ("n_rebuilds", C.c_int64),
                ("xi", C.c_double), ("eta", C.c_double), ("h_ext", C.c_double)]

    def as_dict(self):
        return {"step": self.step, "pe": self.pe, "ke": self.ke, "temperature": self.temperature,
                "pressure": self.pressure, "virial": list(self.virial), "w": self.w,
                "n_rebuilds": self.n_rebuilds, "xi": self.xi, "eta": self.eta,
                "h_ext": self.h_ext}


class gbmd_info(C.Structure):
    _fields_ = [("n", C.c_int64), ("precision", C.c_int32), ("ntypes", C.c_int32),
                ("cells", C.c_int32 * 3), ("nlist_capacity", C.c_int32),
                ("threads_per_particle", C.c_int32), ("force_block", C.c_int32),
                ("step", C.c_int64), ("n_rebuilds", C.c_int64), ("n_sorts", C.c_int64),
                ("kernel_launches", C.c_int64), ("neighbors_total", C.c_int64),
                ("footprint_bytes", C.c_int64), ("force_path", C.c_int32),
                ("max_window", C.c_int32), ("cell_scale", C.c_double), ("nlist", C.c_int32),
                ("rebuild_pending", C.c_int32), ("n_ghost", C.c_int64)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["cells"] = list(self.cells)
        return d


_lib = None
_SIGS = {
    "gbmd_create": (C.c_int, [C.POINTER(gbmd_desc), C.POINTER(C.c_void_p)]),
    "gbmd_create_device": (C.c_int, [C.POINTER(gbmd_desc), C.POINTER(C.c_void_p)]),
    "gbmd_destroy": (C.c_int, [C.c_void_p]),
    "gbmd_step": (C.c_int, [C.c_void_p, C.c_int64]),
    "gbmd_sync": (C.c_int, [C.c_void_p]),
    "gbmd_get_forces": (C.c_int, [C.c_void_p, C.c_void_p]),
    "gbmd_get_thermo": (C.c_int, [C.c_void_p, C.POINTER(gbmd_thermo)]),
    "gbmd_get_thermo_noalloc": (C.c_int, [C.c_void_p, C.POINTER(gbmd_thermo)]),
    "gbmd_get_per_particle": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "gbmd_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.POINTER(C.c_int64)]),
    "gbmd_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]),
    "gbmd_get_neighbors": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]),
    "gbmd_get_info": (C.c_int, [C.c_void_p, C.POINTER(gbmd_info)]),
    "gbmd_footprint_bytes": (C.c_int64, [C.POINTER(gbmd_desc)]),
    "gbmd_set_step_limit": (C.c_int, [C.c_void_p, C.c_int64]),
    "gbmd_set_force_events": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "gbmd_autotune": (C.c_int, [C.c_void_p, C.c_char_p]),
    "gbmd_set_tuning": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    "gbmd_set_cell_scale": (C.c_int, [C.c_void_p, C.c_double]),
    "gbmd_set_thermostat": (C.c_int, [C.c_void_p, C.c_double, C.c_double]),
    "gbmd_batch_create": (C.c_int, [C.c_int32, C.c_void_p, C.c_int32, C.POINTER(C.c_void_p)]),
    "gbmd_batch_add": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_int32)]),
    "gbmd_batch_remove": (C.c_int, [C.c_void_p, C.c_int32]),
    "gbmd_batch_step": (C.c_int, [C.c_void_p, C.c_int64]),
    "gbmd_batch_sync": (C.c_int, [C.c_void_p]),
    "gbmd_batch_autotune": (C.c_int, [C.c_void_p, C.c_char_p]),
    "gbmd_batch_set_tuning": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    "gbmd_batch_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int64),
                                  C.POINTER(C.c_int64)]),
    "gbmd_batch_destroy": (C.c_int, [C.c_void_p]),
    "gbmd_last_error": (C.c_char_p, []),
    "gbmd_abi_version": (C.c_int, []),
    "gbmd_probe_arith": (C.c_int, [C.c_int32, C.c_int32, C.c_void_p, C.POINTER(C.c_double),
                                   C.POINTER(C.c_float)]),
    "gbmd_set_ghost_positions": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "gbmd_get_positions": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int32]),
}


def load(path: str | None = None):
    """Load libgbmd.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with __graft_entry__.build() "
                           "(there is no CPU fallback)")
    lib = C.CDLL(p)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _check(code: int):
    if code != GBMD_OK:
        raise GbmdError(code, load().gbmd_last_error().decode(errors="replace"))
    return code


def _arr(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream", stream))


def make_desc(n, box, pos, vel, types, eps, sigma, rcut, r_buff, dt, mass, precision,
              sort_period=0, nlist_capacity=0, threads_per_particle=0, stream=None,
              image=None, device=False, cuda_device=-1, force_path="global", integrator="nve",
              kT=0.0, tau=0.0, potential="lj", mie_n=None, mie_m=None, kappa=None, nlist="cell",
              n_ghost=0):
    """Build a gbmd_desc; returns (desc, keepalive) -- keep the second alive.  Pair
    tables are ntypes x ntypes arrays or scalars; a table the potential does not read
    may be None (sigma for Yukawa, rcut for WCA, mie_n / mie_m / kappa elsewhere)."""
    eps = np.atleast_2d(np.asarray(eps, np.float64))
    nt = eps.shape[0]
    eps = np.ascontiguousarray(np.broadcast_to(eps, (nt, nt)))

    def table(t):
        if t is None:
            return None
        return np.ascontiguousarray(np.broadcast_to(np.atleast_2d(np.asarray(t, np.float64)), (nt, nt)))
    sigma, rcut, mie_n, mie_m, kappa = (table(t) for t in (sigma, rcut, mie_n, mie_m, kappa))
    keep = [eps, sigma, rcut, mie_n, mie_m, kappa]
    d = gbmd_desc()
    d.n = int(n)
    box = np.broadcast_to(np.asarray(box, np.float64), (3,))
    for a in range(3):
        d.box[a] = float(box[a])
    if device:
        d.pos, d.vel = int(pos), int(vel)
        d.type = int(types) if types is not None else None
        d.image = int(image) if image is not None else None
    else:
        pos = _arr(pos, np.float64).reshape(-1, 3)
        vel = _arr(vel, np.float64).reshape(-1, 3)
        types = _arr(types, np.int32)
        image = _arr(image, np.int32)
        keep += [pos, vel, types, image]
        d.pos, d.vel, d.type, d.image = _ptr(pos), _ptr(vel), _ptr(types), _ptr(image)
    d.ntypes = nt
    d.eps, d.sigma, d.rcut = _ptr(eps), _ptr(sigma), _ptr(rcut)
    d.r_buff, d.dt, d.mass = float(r_buff), float(dt), float(mass)
    d.precision = PRECISIONS.get(precision, precision) if isinstance(precision, str) else int(precision)
    d.sort_period = int(sort_period)
    d.nlist_capacity = int(nlist_capacity)
    d.threads_per_particle = int(threads_per_particle)
    d.stream = _stream_handle(stream)
    d.device = int(cuda_device)
    d.force_path = FORCE_PATHS.get(force_path, force_path) if isinstance(force_path, str) else int(force_path)
    d.integrator = INTEGRATORS.get(integrator, integrator) if isinstance(integrator, str) else int(integrator)
    d.kT = float(kT)
    d.tau = float(tau)
    d.potential = POTENTIALS.get(potential, potential) if isinstance(potential, str) else int(potential)
    d.mie_n, d.mie_m, d.kappa = _ptr(mie_n), _ptr(mie_m), _ptr(kappa)
    d.nlist = NLISTS.get(nlist, nlist) if isinstance(nlist, str) else int(nlist)
    d.n_ghost = int(n_ghost)
    return d, keep


# ---- module-level functions with the C names -------------------------------------

def gbmd_create(desc: gbmd_desc) -> int:
    h = C.c_void_p()
    _check(load().gbmd_create(C.byref(desc), C.byref(h)))
    return h.value


def gbmd_create_device(desc: gbmd_desc) -> int:
    h = C.c_void_p()
    _check(load().gbmd_create_device(C.byref(desc), C.byref(h)))
    return h.value


def gbmd_destroy(h):
    return _check(load().gbmd_destroy(h))


def gbmd_step(h, nsteps: int):
    return _check(load().gbmd_step(h, int(nsteps)))


def gbmd_sync(h):
    return _check(load().gbmd_sync(h))


def gbmd_get_forces(h, n: int, out=None):
    out = np.empty((n, 3)) if out is None else out
    _check(load().gbmd_get_forces(h, _ptr(out)))
    return out


def gbmd_get_thermo(h) -> dict:
    t = gbmd_thermo()
    _check(load().gbmd_get_thermo(h, C.byref(t)))
    return t.as_dict()


def gbmd_get_thermo_noalloc(h) -> dict:
    """gbmd_get_thermo without any GPU allocation (static scratch; see gbmd.h)."""
    t = gbmd_thermo()
    _check(load().gbmd_get_thermo_noalloc(h, C.byref(t)))
    return t.as_dict()


def gbmd_get_per_particle(h, n: int):
    u = np.empty(n)
    w = np.empty((n, 6))
    _check(load().gbmd_get_per_particle(h, _ptr(u), _ptr(w)))
    return u, w


def gbmd_get_state(h, n: int, pos=None, vel=None, image=None):
    pos = np.empty((n, 3)) if pos is None else pos
    vel = np.empty((n, 3)) if vel is None else vel
    image = np.empty((n, 3), np.int32) if image is None else image
    step = C.c_int64(0)
    _check(load().gbmd_get_state(h, _ptr(pos), _ptr(vel), _ptr(image), C.byref(step)))
    return pos, vel, image, step.value


def gbmd_set_state(h, pos, vel, image=None, step: int = 0):
    pos = _arr(pos, np.float64)
    vel = _arr(vel, np.float64)
    image = _arr(image, np.int32)
    return _check(load().gbmd_set_state(h, _ptr(pos), _ptr(vel), _ptr(image), int(step)))


def gbmd_get_neighbors(h, n: int, cap: int):
    counts = np.empty(n, np.int32)
    idx = np.empty((n, cap), np.int32)
    _check(load().gbmd_get_neighbors(h, _ptr(counts), _ptr(idx), int(cap)))
    return counts, idx


def gbmd_get_info(h) -> dict:
    i = gbmd_info()
    _check(load().gbmd_get_info(h, C.byref(i)))
    return i.as_dict()


def gbmd_set_ghost_positions(h, pos, device: bool = False):
    """Ghost positions (n_ghost x 3, ghost tag order): a host array, or a device
    pointer (int) with device=True."""
    if device:
        _check(load().gbmd_set_ghost_positions(h, int(pos), 1))
        return
    p = np.ascontiguousarray(pos, np.float64)
    _check(load().gbmd_set_ghost_positions(h, _ptr(p), 0))


def gbmd_get_positions(h, tags, out=None):
    """Wrapped positions (m x 3) of the particles with the given tags (host arrays)."""
    t = np.ascontiguousarray(tags, np.int32).ravel()
    out = np.empty((t.size, 3), np.float64) if out is None else out
    _check(load().gbmd_get_positions(h, _ptr(t), t.size, _ptr(out), 0))
    return out


def gbmd_get_positions_device(h, tags_ptr: int, m: int, out_ptr: int):
    """As gbmd_get_positions with device pointers (int32 tags, m x 3 FP64 out)."""
    _check(load().gbmd_get_positions(h, int(tags_ptr), int(m), int(out_ptr), 1))


def gbmd_footprint_bytes(desc: gbmd_desc) -> int:
    r = load().gbmd_footprint_bytes(C.byref(desc))
    if r < 0:
        _check(int(r))
    return int(r)


def gbmd_set_step_limit(h, step: int):
    return _check(load().gbmd_set_step_limit(h, int(step)))


def gbmd_set_force_events(h, ev_begin, ev_end):
    """ev_begin / ev_end: cudaEvent_t handles (int) or torch.cuda.Event, or None."""
    def handle(e):
        return None if e is None else int(getattr(e, "cuda_event", e))
    return _check(load().gbmd_set_force_events(h, handle(ev_begin), handle(ev_end)))


def gbmd_autotune(h, cache_path: str | None = None):
    return _check(load().gbmd_autotune(h, cache_path.encode() if cache_path else None))


def gbmd_set_tuning(h, tpp: int, block: int):
    return _check(load().gbmd_set_tuning(h, int(tpp), int(block)))


def gbmd_set_cell_scale(h, scale: float):
    return _check(load().gbmd_set_cell_scale(h, float(scale)))


def gbmd_set_thermostat(h, xi: float, eta: float):
    return _check(load().gbmd_set_thermostat(h, float(xi), float(eta)))


def gbmd_batch_create(precision, stream=None, cuda_device=-1) -> int:
    h = C.c_void_p()
    p = PRECISIONS.get(precision, precision) if isinstance(precision, str) else int(precision)
    _check(load().gbmd_batch_create(p, _stream_handle(stream), int(cuda_device), C.byref(h)))
    return h.value


def gbmd_batch_add(b, s) -> int:
    slot = C.c_int32(-1)
    _check(load().gbmd_batch_add(b, s, C.byref(slot)))
    return slot.value


def gbmd_batch_remove(b, slot: int):
    return _check(load().gbmd_batch_remove(b, int(slot)))


def gbmd_batch_step(b, nsteps: int):
    return _check(load().gbmd_batch_step(b, int(nsteps)))


def gbmd_batch_sync(b):
    return _check(load().gbmd_batch_sync(b))


def gbmd_batch_autotune(b, cache_path: str | None = None):
    return _check(load().gbmd_batch_autotune(b, cache_path.encode() if cache_path else None))


def gbmd_batch_set_tuning(b, tpp: int, block: int):
    return _check(load().gbmd_batch_set_tuning(b, int(tpp), int(block)))


def gbmd_batch_info(b) -> dict:
    m = C.c_int32(0)
    n = C.c_int64(0)
    L = C.c_int64(0)
    _check(load().gbmd_batch_info(b, C.byref(m), C.byref(n), C.byref(L)))
    return {"members": m.value, "particles": n.value, "kernel_launches": L.value}


def gbmd_batch_destroy(b):
    return _check(load().gbmd_batch_destroy(b))


def gbmd_last_error() -> str:
    return load().gbmd_last_error().decode(errors="replace")


def gbmd_abi_version() -> int:
    return int(load().gbmd_abi_version())


PROBE_KINDS = {"dfma": 0, "ffma": 1, "drcp": 2}


def gbmd_probe_arith(kind: str, iters: int, stream=None):
    """(operations, milliseconds) of one timed probe launch on the current device."""
    ops = C.c_double(0)
    ms = C.c_float(0)
    _check(load().gbmd_probe_arith(PROBE_KINDS.get(kind, kind) if isinstance(kind, str)
                                   else int(kind), int(iters), _stream_handle(stream),
                                   C.byref(ops), C.byref(ms)))
    return ops.value, ms.value


# ---- convenience wrappers ----------------------------------------------------------

class System:
    """One LJ system resident on the GPU (owns a gbmd_system handle)."""

    def __init__(self, pos, vel, box, types=None, eps=1.0, sigma=1.0, rcut=2.5, r_buff=0.4,
                 dt=0.005, mass=1.0, precision="mixed", sort_period=0, nlist_capacity=0,
                 threads_per_particle=0, stream=None, image=None, device=False, n=None,
                 cuda_device=-1, force_path="global", integrator="nve", kT=0.0, tau=0.0,
                 potential="lj", mie_n=None, mie_m=None, kappa=None, nlist="cell", n_ghost=0):
        n = int(n if n is not None else np.asarray(pos).reshape(-1, 3).shape[0])
        desc, keep = make_desc(n, box, pos, vel, types, eps, sigma, rcut, r_buff, dt, mass,
                               precision, sort_period, nlist_capacity, threads_per_particle,
                               stream, image, device, cuda_device, force_path, integrator, kT, tau,
                               potential, mie_n, mie_m, kappa, nlist, n_ghost)
        self.n = n
        self.box = np.broadcast_to(np.asarray(box, np.float64), (3,)).copy()
        self.precision = precision
        self.handle = gbmd_create_device(desc) if device else gbmd_create(desc)
        del keep

    @classmethod
    def from_workload(cls, w, precision="mixed", **kw):
        p = w.pairs
        for k, v in p.potential_kw().items():
            kw.setdefault(k, v)
        return cls(w.pos, w.vel, w.box, w.types, p.eps, p.sigma, p.rcut, w.r_buff, w.dt, w.mass,
                   precision, **kw)

    def step(self, n: int):
        gbmd_step(self.handle, n)

    def sync(self):
        gbmd_sync(self.handle)

    def forces(self, out=None):
        return gbmd_get_forces(self.handle, self.n, out)

    def thermo(self) -> dict:
        return gbmd_get_thermo(self.handle)

    def per_particle(self):
        return gbmd_get_per_particle(self.handle, self.n)

    def state(self):
        return gbmd_get_state(self.handle, self.n)

    def set_state(self, pos, vel, image=None, step=0):
        gbmd_set_state(self.handle, pos, vel, image, step)

    def neighbors(self, cap: int = 256):
        return gbmd_get_neighbors(self.handle, self.n, cap)

    def info(self) -> dict:
        return gbmd_get_info(self.handle)

    def set_step_limit(self, step: int):
        gbmd_set_step_limit(self.handle, step)

    def autotune(self, cache_path=None):
        gbmd_autotune(self.handle, cache_path)

    def set_tuning(self, tpp: int, block: int):
        gbmd_set_tuning(self.handle, tpp, block)

    def set_cell_scale(self, scale: float):
        gbmd_set_cell_scale(self.handle, scale)

    def set_ghost_positions(self, pos):
        gbmd_set_ghost_positions(self.handle, pos)

    def positions(self, tags, out=None):
        return gbmd_get_positions(self.handle, tags, out)

    def set_thermostat(self, xi: float, eta: float):
        gbmd_set_thermostat(self.handle, xi, eta)

    def set_force_events(self, ev_begin, ev_end):
        gbmd_set_force_events(self.handle, ev_begin, ev_end)

    def close(self):
        if getattr(self, "handle", None):
            gbmd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many systems stepped with shared launches (owns a gbmd_batch handle)."""

    def __init__(self, precision="mixed", stream=None, cuda_device=-1):
        self.handle = gbmd_batch_create(precision, stream, cuda_device)
        self.members = {}

    def add(self, system: System) -> int:
        slot = gbmd_batch_add(self.handle, system.handle)
        self.members[slot] = system
        return slot

    def remove(self, slot: int) -> System:
        gbmd_batch_remove(self.handle, slot)
        return self.members.pop(slot)

    def step(self, n: int):
        gbmd_batch_step(self.handle, n)

    def sync(self):
        gbmd_batch_sync(self.handle)

    def autotune(self, cache_path=None):
        gbmd_batch_autotune(self.handle, cache_path)

    def set_tuning(self, tpp: int, block: int):
        gbmd_batch_set_tuning(self.handle, tpp, block)

    def info(self) -> dict:
        return gbmd_batch_info(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            gbmd_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""One system split into spatial domains over several ranks, one GPU each.

Sections 2 and 5 of the paper: HOOMD-blue runs one system on several GPUs by
spatial domain decomposition over MPI, each GPU integrating the particles of its
domain and exchanging the positions of the particles near the domain boundaries
every step.  This module is that decomposition over ``torch.distributed`` (NCCL
between GPUs, gloo on the host), on top of the library's ghost particles
(``gbmd_desc.n_ghost``, ``gbmd_set_ghost_positions``, ``gbmd_get_positions``).

Domains are slabs along one box axis: rank r of P owns the particles whose
coordinate along that axis lies in [-L/2 + r W, -L/2 + (r + 1) W), W = L / P.  Its
local system holds its own particles (in global-id order) followed by ghosts: the
particles of the other ranks within r_ghost = r_cut,max + r_buff of its slab (the
periodic distance along the axis), chosen at the last rebuild.  Every step:

1. each rank sends the current positions of its particles that are ghosts
   elsewhere (send lists fixed at the rebuild) and receives its ghosts' positions
   (one all-to-all);
2. it steps its local system: forces on every local particle, integration of its
   own ones only (ghosts keep the positions they were given);
3. the ranks agree (one all-reduce) whether any particle moved more than r_buff / 2
   since the rebuild.  If so, every rank rebuilds: particles that left a slab go to
   their new owner with their velocity and image counts, ghosts are chosen again,
   and each local system is created afresh (its own neighbour list built from the
   new owned + ghost set).

This keeps the Verlet-list guarantee across domains: a pair inside r_cut now was
inside r_cut + r_buff at the rebuild, when the partner lay within r_ghost of the
slab and so became a ghost.  Forces on a rank's own particles are therefore those of
the whole system.

The exchange goes through host memory on gloo and through device memory on NCCL;
ownership changes only at rebuilds.  Engines are pluggable: ``GpuEngine`` (the
library) is the product path; any object with the same methods can stand in.
"""
from __future__ import annotations

import numpy as np

# columns of a migrating particle's record: id, position (3), velocity (3), image
# counts (3), type
_REC = 11
# columns of a ghost record: id, position (3), type
_GHOST = 5


class Slabs:
    """The slab geometry: owners and halo membership along one axis."""

    def __init__(self, box, nranks: int, r_ghost: float, axis: int | None = None):
        self.box = np.broadcast_to(np.asarray(box, np.float64), (3,)).copy()
        self.P = int(nranks)
        self.axis = int(np.argmax(self.box)) if axis is None else int(axis)
        self.L = float(self.box[self.axis])
        self.W = self.L / self.P
        self.r_ghost = float(r_ghost)

    def owner(self, pos) -> np.ndarray:
        """Owning rank of each (wrapped or not) position."""
        x = np.asarray(pos, np.float64)[:, self.axis]
        x = x - self.L * np.floor((x + 0.5 * self.L) / self.L)   # [-L/2, L/2)
        r = np.floor((x + 0.5 * self.L) / self.W).astype(np.int64)
        return np.clip(r, 0, self.P - 1)

    def slab_gap(self, pos, rank: int) -> np.ndarray:
        """Periodic distance along the axis from each position to slab `rank`
        (0 inside it)."""
        x = np.asarray(pos, np.float64)[:, self.axis]
        lo = -0.5 * self.L + rank * self.W
        c = lo + 0.5 * self.W                         # slab centre
        d = x - c
        d = d - self.L * np.rint(d / self.L)          # periodic offset from the centre
        return np.maximum(np.abs(d) - 0.5 * self.W, 0.0)

    def halo(self, pos, rank: int) -> list[np.ndarray]:
        """For each rank k != `rank`: indices of the given positions (owned by
        `rank`) that are ghosts on k (within r_ghost of slab k); [] for k = rank."""
        out = []
        for k in range(self.P):
            if k == rank:
                out.append(np.zeros(0, np.int64))
            else:
                out.append(np.flatnonzero(self.slab_gap(pos, k) < self.r_ghost))
        return out


class GpuEngine:
    """A domain's local system on the GPU (the library's ghost particles)."""

    def __init__(self, pos, vel, types, image, n_ghost, w, precision, **kw):
        from . import gbmd
        self.n_own = len(pos) - n_ghost
        self.s = gbmd.System(pos, vel, w.box, types, w.pairs.eps, w.pairs.sigma, w.pairs.rcut,
                             w.r_buff, w.dt, w.mass, precision, image=image, n_ghost=n_ghost,
                             **kw)

    def set_ghosts(self, pos):
        self.s.set_ghost_positions(pos)

    def step(self):
        self.s.step(1)

    def rebuild_pending(self) -> bool:
        return bool(self.s.info()["rebuild_pending"])

    def owned_state(self):
        pos, vel, img, _ = self.s.state()
        k = self.n_own
        return pos[:k].copy(), vel[:k].copy(), img[:k].copy()

    def positions(self, idx):
        return self.s.positions(np.asarray(idx, np.int32))

    def forces(self):
        return self.s.forces()[:self.n_own].copy()

    def close(self):
        self.s.close()


class DomainRun:
    """One rank's part of a system decomposed into slabs.

    ``ids``, ``pos``, ``vel``, ``image``, ``types`` are the rank's initial particles
    (global ids; any subset, e.g. the whole system on every rank: each rank keeps
    what it owns).  ``w`` carries box, pair table, r_buff, dt and mass.  ``comm`` is
    torch.distributed (initialised), or None for one rank.  ``engine`` builds a local
    system from (pos, vel, types, image, n_ghost); the default is ``GpuEngine``.
    """

    def __init__(self, w, ids, pos, vel, types, image=None, comm=None, precision="fp64",
                 engine=None, axis=None, **engine_kw):
        self.w = w
        self.comm = comm
        self.rank = comm.get_rank() if comm is not None else 0
        self.P = comm.get_world_size() if comm is not None else 1
        rc = float(np.max(np.asarray(w.pairs.rcut, np.float64)))
        self.slabs = Slabs(w.box, self.P, rc + w.r_buff, axis)
        self.precision = precision
        self.engine_kw = engine_kw
        self.make_engine = engine or (lambda p, v, t, im, ng: GpuEngine(p, v, t, im, ng, w,
                                                                         precision, **engine_kw))
        self.eng = None
        self.n_rebuilds = 0
        self.n_migrated = 0
        self.step_count = 0
        ids = np.asarray(ids, np.int64)
        pos = np.asarray(pos, np.float64).reshape(-1, 3)
        vel = np.asarray(vel, np.float64).reshape(-1, 3)
        img = np.zeros((len(ids), 3), np.int64) if image is None else np.asarray(image, np.int64)
        types = np.zeros(len(ids), np.int64) if types is None else np.asarray(types, np.int64)
        mine = self.slabs.owner(pos) == self.rank
        self._build(ids[mine], pos[mine], vel[mine], img[mine], types[mine])

    # ---- communication ------------------------------------------------------------

    def _alltoall_rows(self, parts: list[np.ndarray], width: int) -> list[np.ndarray]:
        """Send parts[k] (rows of `width` float64) to rank k; returns the rows from
        each rank, in rank order."""
        if self.comm is None:
            return [parts[0].reshape(-1, width)]
        import torch
        dist = self.comm
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        counts = torch.tensor([len(p) for p in parts], dtype=torch.int64, device=dev)
        rcounts = torch.empty_like(counts)
        dist.all_to_all_single(rcounts, counts)
        rc = [int(c) for c in rcounts.tolist()]
        send = torch.from_numpy(np.concatenate([p.reshape(-1, width) for p in parts])
                                .astype(np.float64).ravel()).to(dev)
        recv = torch.empty(sum(rc) * width, dtype=torch.float64, device=dev)
        dist.all_to_all_single(recv, send, [c * width for c in rc],
                               [len(p) * width for p in parts])
        flat = recv.cpu().numpy().reshape(-1, width)
        out, o = [], 0
        for c in rc:
            out.append(flat[o:o + c])
            o += c
        return out

    def _any(self, flag: bool) -> bool:
        if self.comm is None:
            return bool(flag)
        import torch
        dev = "cuda" if self.comm.get_backend() == "nccl" else "cpu"
        t = torch.tensor([1 if flag else 0], dtype=torch.int32, device=dev)
        self.comm.all_reduce(t, op=self.comm.ReduceOp.MAX)
        return bool(t.item())

    # ---- rebuild ----------------------------------------------------------------

    def _build(self, ids, pos, vel, img, types):
        """Owned particles (any order) -> the local system with fresh ghosts."""
        order = np.argsort(ids, kind="stable")
        self.ids = ids[order]
        pos, vel, img, types = pos[order], vel[order], img[order], types[order]
        if len(self.ids) == 0:
            raise RuntimeError(f"rank {self.rank} owns no particle: too many domains for "
                               "this system")
        self.types = types
        # ghosts: every rank sends its owned particles within r_ghost of each other slab
        self.send_idx = self.slabs.halo(pos, self.rank)
        parts = [np.column_stack([self.ids[ix], pos[ix], types[ix]]) if len(ix)
                 else np.zeros((0, _GHOST)) for ix in self.send_idx]
        recv = self._alltoall_rows(parts, _GHOST)
        self.recv_counts = [len(r) for r in recv]
        ghosts = np.concatenate(recv) if recv else np.zeros((0, _GHOST))
        self.ghost_ids = ghosts[:, 0].astype(np.int64)
        n_ghost = len(ghosts)
        allpos = np.concatenate([pos, ghosts[:, 1:4]])
        allvel = np.concatenate([vel, np.zeros((n_ghost, 3))])
        allimg = np.concatenate([img, np.zeros((n_ghost, 3), np.int64)]).astype(np.int32)
        alltypes = np.concatenate([types, ghosts[:, 4].astype(np.int64)]).astype(np.int32)
        if self.eng is not None:
            self.eng.close()
        self.eng = self.make_engine(allpos, allvel, alltypes, allimg, n_ghost)

    def _rebuild(self):
        """Migrate the particles that left their slab, then choose ghosts again."""
        self._exchange()   # current ghosts: the full-step velocities need F(x) now
        pos, vel, img = self.eng.owned_state()
        dest = self.slabs.owner(pos)
        parts = []
        for k in range(self.P):
            m = dest == k
            parts.append(np.column_stack([self.ids[m], pos[m], vel[m], img[m], self.types[m]])
                         if m.any() else np.zeros((0, _REC)))
        self.n_migrated += int((dest != self.rank).sum())
        got = np.concatenate(self._alltoall_rows(parts, _REC))
        self._build(got[:, 0].astype(np.int64), got[:, 1:4], got[:, 4:7],
                    got[:, 7:10].astype(np.int64), got[:, 10].astype(np.int64))
        self.n_rebuilds += 1

    # ---- stepping ---------------------------------------------------------------

    def _exchange(self):
        """Send the current positions of this rank's ghosts-elsewhere; receive its own
        ghosts' positions (in the order fixed at the rebuild)."""
        if self.P == 1:   # one domain: no ghosts
            return
        allix = np.concatenate(self.send_idx) if self.send_idx else np.zeros(0, np.int64)
        cur = self.eng.positions(allix) if len(allix) else np.zeros((0, 3))
        parts, o = [], 0
        for ix in self.send_idx:
            parts.append(cur[o:o + len(ix)])
            o += len(ix)
        recv = self._alltoall_rows(parts, 3)
        got = np.concatenate(recv) if recv else np.zeros((0, 3))
        if len(got):
            self.eng.set_ghosts(got)

    def step(self, n: int = 1):
        for _ in range(int(n)):
            self._exchange()
            self.eng.step()
            self.step_count += 1
            if self._any(self.eng.rebuild_pending()):
                self._rebuild()

    # ---- readouts ----------------------------------------------------------------

    def owned(self):
        """(ids, wrapped positions, full-step velocities, image counts) of this rank's
        particles (collective: the ghosts are brought up to date first)."""
        self._exchange()
        pos, vel, img = self.eng.owned_state()
        return self.ids.copy(), pos, vel, img

    def forces(self):
        """(ids, forces) on this rank's particles at the current positions (collective:
        the ghosts are brought up to date first)."""
        self._exchange()
        return self.ids.copy(), self.eng.forces()

    def close(self):
        if self.eng is not None:
            self.eng.close()
            self.eng = None

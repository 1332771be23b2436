"""Domain decomposition (Sections 2 and 5: one system split into spatial domains,
one GPU each) -- the host side, on CPU.

* The slab geometry: every particle has exactly one owner, and every pair closer
  than r_ghost across two slabs finds its partner among the ghosts (brute force;
  with 5 and 8 slabs narrower than r_ghost, ghosts also come from slabs that are
  not adjacent).
* The whole decomposition of a 2,000-particle LJ fluid on 2 and 3 gloo ranks, each
  running its domain with an engine that computes forces with the FP64 oracle
  (``oracle.forces_subset`` on its owned particles against owned + ghosts): after
  100 velocity-Verlet steps, with rebuilds and particles migrating between slabs,
  the gathered positions, velocities and image counts equal the oracle's
  single-system run (``vv_run``) to 1e-9.  A ghost reach 0.6 sigma short of
  r_cut + r_buff fails this on both (checked with a mutated copy, kept out of the
  tree).
The same driver runs the library's engine on the GPU in ``test_gpu_domain.py``.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1308_5587_gb300 import workloads as wl
from paper_1308_5587_gb300.domain import DomainRun, Slabs


def mi(d, box):
    return d - box * np.rint(d / box)


def test_slabs_own_every_particle_once_and_halo_is_complete():
    rng = np.random.default_rng(5)
    box = np.array([20.0, 14.0, 12.0])
    pos = (rng.random((3000, 3)) - 0.5) * box * 3          # any periodic image
    for P in (1, 2, 3, 5, 8):
        sl = Slabs(box, P, 2.9)
        assert sl.axis == 0
        own = sl.owner(pos)
        assert own.min() >= 0 and own.max() < P
        xw = pos[:, 0] - box[0] * np.floor((pos[:, 0] + box[0] / 2) / box[0])
        assert np.array_equal(own, np.clip(np.floor((xw + box[0] / 2) / (box[0] / P)), 0, P - 1))
        for k in range(P):
            mine = own == k
            assert np.all(sl.slab_gap(pos[mine], k) == 0)
            ghosts = np.zeros(len(pos), bool)
            for r in range(P):
                if r == k:
                    continue
                idx = np.flatnonzero(own == r)
                ghosts[idx[sl.halo(pos[idx], r)[k]]] = True
            # brute force: every particle of another slab within r_ghost of one of k's
            d = mi(pos[mine][:, None, :] - pos[~mine][None, :, :], box)
            near = (np.sqrt((d ** 2).sum(-1)) < 2.9).any(0)
            assert np.all(ghosts[np.flatnonzero(~mine)[near]])
            assert not ghosts[mine].any()


class OracleEngine:
    """A domain's local system computed with the FP64 oracle (test only): the
    library's step in its leapfrog form -- kick by the force at the current
    positions (half a kick right after creation), drift, wrap; ghosts stay put; a
    rebuild is pending once an owned particle moved more than r_buff / 2."""

    def __init__(self, pos, vel, types, image, n_ghost, w):
        import oracle
        self.o = oracle
        self.w = w
        self.n = len(pos)
        self.n_own = self.n - n_ghost
        self.own = np.arange(self.n_own)
        p, k = oracle.wrap(np.asarray(pos, np.float64), w.box)
        self.pos = p
        self.img = np.asarray(image, np.int64) + k
        self.vel = np.asarray(vel, np.float64).copy()
        self.types = np.asarray(types, np.int32)
        self.build = self.pos[:self.n_own].copy()
        self.vfull = True
        self.h = 0.5 * w.dt / w.mass

    def _force(self):
        F, _, _ = self.o.forces_subset(self.pos, self.w.box, self.types, self.w.pairs.as_dict(),
                                       self.own)
        return F

    def set_ghosts(self, pos):
        p, _ = self.o.wrap(np.asarray(pos, np.float64), self.w.box)
        self.pos[self.n_own:] = p

    def step(self):
        F = self._force()
        kick = self.h if self.vfull else 2 * self.h
        v = self.vel[:self.n_own] + kick * F
        x = self.pos[:self.n_own] + self.w.dt * v
        xw, k = self.o.wrap(x, self.w.box)
        self.vel[:self.n_own] = v
        self.pos[:self.n_own] = xw
        self.img[:self.n_own] += k
        self.vfull = False

    def rebuild_pending(self):
        d = mi(self.pos[:self.n_own] - self.build, self.w.box)
        return bool(((d ** 2).sum(1) > (0.5 * self.w.r_buff) ** 2).any())

    def owned_state(self):
        v = self.vel[:self.n_own].copy()
        if not self.vfull:
            v += self.h * self._force()
        return self.pos[:self.n_own].copy(), v, self.img[:self.n_own].copy()

    def positions(self, idx):
        return self.pos[np.asarray(idx, np.int64)]

    def forces(self):
        return self._force()

    def close(self):
        pass


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, nsteps, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import oracle
    oracle.build()
    oracle.set_threads(1)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = wl.lj_fluid(2000, 0.84, 1.2, seed=900)
    run = DomainRun(w, np.arange(w.n), w.pos, w.vel, w.types, comm=dist,
                    engine=lambda p, v, t, im, ng: OracleEngine(p, v, t, im, ng, w))
    run.step(nsteps)
    ids, pos, vel, img = run.owned()
    q.put((rank, ids, pos, vel, img, run.n_rebuilds, run.n_migrated,
           int(sum(run.recv_counts))))
    run.close()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_decomposed_run_equals_the_single_system(oracle, world):
    nsteps = 100
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(k, world, port, nsteps, q)) for k in range(world)]
    for p in ps:
        p.start()
    res = [q.get(timeout=600) for _ in ps]
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    w = wl.lj_fluid(2000, 0.84, 1.2, seed=900)
    ref = oracle.vv_run(w.pos, w.vel, w.box, w.types, w.pairs.as_dict(), w.mass, w.dt, nsteps)
    ids = np.concatenate([r[1] for r in res])
    assert np.array_equal(np.sort(ids), np.arange(w.n))           # each particle once
    pos = np.empty((w.n, 3)); vel = np.empty((w.n, 3)); img = np.empty((w.n, 3), np.int64)
    for r in res:
        pos[r[1]], vel[r[1]], img[r[1]] = r[2], r[3], r[4]
    assert np.abs(mi(pos - ref["pos"], w.box)).max() < 1e-9
    assert np.abs(vel - ref["vel"]).max() < 1e-9
    assert np.array_equal(img, ref["image"])
    assert min(r[5] for r in res) >= 1             # rebuilt at least once
    assert sum(r[6] for r in res) > 0              # and particles changed slab
    assert all(r[7] > 0 for r in res)              # every domain had ghosts

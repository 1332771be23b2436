"""Domain decomposition on the GPU: the library's ghost particles under the slab
driver (``domain.DomainRun`` with ``GpuEngine``).

Two ranks run as two processes on one GPU with a gloo process group: the exchange
goes through host memory and neither rank's kernels wait on the other's, so the
two domains need not run at the same time.  A 4,000-particle LJ fluid is split into
two slabs; after 100 steps with rebuilds and migrations the gathered state equals:
* FP64: the oracle's single-system velocity Verlet to 1e-9 (the parity tolerance of
  the single-system trajectory);
* mixed: the FP64 oracle and the library's own single-system mixed run to 1e-4
  sigma (the bound the mixed trajectory tests use: only the order of the FP32 force
  sums differs from the single system, and 100 chaotic steps amplify that to ~1e-5),
  and the forces at the final positions equal the oracle's there to 1e-5 (relative
  L2), the mixed force tolerance.
The single-system library calls with ghosts are checked in the same file: ghosts
keep the positions they are given, and a rebuild is left to the caller.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_1308_5587_gb300 import gbmd, workloads as wl
from paper_1308_5587_gb300.domain import DomainRun

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    from paper_1308_5587_gb300 import _build
    _build.build()
    oracle.build()
    oracle.set_threads(os.cpu_count() or 1)


def mi(d, box):
    return d - box * np.rint(d / box)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, prec, nsteps, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = wl.lj_fluid(4000, 0.84, 1.2, seed=910)
    run = DomainRun(w, np.arange(w.n), w.pos, w.vel, w.types, comm=dist, precision=prec)
    n_ghost = int(sum(run.recv_counts))
    run.step(nsteps)
    ids, pos, vel, img = run.owned()
    fid, F = run.forces()
    q.put((rank, ids, pos, vel, img, F, run.n_rebuilds, run.n_migrated, n_ghost))
    run.close()
    dist.destroy_process_group()


def _decomposed(prec, nsteps, world=2):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(k, world, port, prec, nsteps, q)) for k in range(world)]
    for p in ps:
        p.start()
    res = [q.get(timeout=900) for _ in ps]
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    n = sum(len(r[1]) for r in res)
    pos = np.empty((n, 3)); vel = np.empty((n, 3)); img = np.empty((n, 3), np.int64)
    F = np.empty((n, 3))
    ids = np.concatenate([r[1] for r in res])
    assert np.array_equal(np.sort(ids), np.arange(n))
    for r in res:
        pos[r[1]], vel[r[1]], img[r[1]], F[r[1]] = r[2], r[3], r[4], r[5]
    assert min(r[6] for r in res) >= 1          # rebuilt
    assert sum(r[7] for r in res) > 0           # particles changed slab
    assert all(r[8] > 0 for r in res)           # both domains had ghosts
    return pos, vel, img, F


def test_decomposed_fp64_equals_the_oracle():
    nsteps = 100
    pos, vel, img, F = _decomposed("fp64", nsteps)
    w = wl.lj_fluid(4000, 0.84, 1.2, seed=910)
    ref = oracle.vv_run(w.pos, w.vel, w.box, w.types, w.pairs.as_dict(), w.mass, w.dt, nsteps)
    assert np.abs(mi(pos - ref["pos"], w.box)).max() < 1e-9
    assert np.abs(vel - ref["vel"]).max() < 1e-9
    assert np.array_equal(img, ref["image"])
    Fo, *_ = oracle.forces(pos, w.box, w.types, w.pairs.as_dict())
    assert np.linalg.norm(F - Fo) / np.linalg.norm(Fo) < 1e-12


def test_decomposed_mixed_equals_the_single_system():
    nsteps = 100
    pos, vel, img, F = _decomposed("mixed", nsteps)
    w = wl.lj_fluid(4000, 0.84, 1.2, seed=910)
    s = gbmd.System.from_workload(w, precision="mixed")
    s.step(nsteps)
    p1, v1, i1, _ = s.state()
    s.close()
    assert np.abs(mi(pos - p1, w.box)).max() < 1e-4
    ref = oracle.vv_run(w.pos, w.vel, w.box, w.types, w.pairs.as_dict(), w.mass, w.dt, nsteps)
    assert np.abs(mi(pos - ref["pos"], w.box)).max() < 1e-4
    Fo, *_ = oracle.forces(pos, w.box, w.types, w.pairs.as_dict())
    assert np.linalg.norm(F - Fo) / np.linalg.norm(Fo) < 1e-5


@pytest.mark.parametrize("prec,nlist", [("fp64", "cell"), ("mixed", "cell"), ("mixed", "tree")])
def test_ghosts_keep_their_positions_and_leave_rebuilds_to_the_caller(prec, nlist):
    w = wl.lj_fluid(3000, 0.84, 1.2, seed=911)
    ng = 500
    s = gbmd.System.from_workload(w, precision=prec, n_ghost=ng, nlist=nlist)
    assert s.info()["n_ghost"] == ng
    tags = np.arange(w.n - ng, w.n)
    g0 = s.positions(tags)
    rng = np.random.default_rng(3)
    moved = g0 + rng.normal(scale=0.01, size=g0.shape)
    s.set_ghost_positions(moved)
    s.step(1)
    got = s.positions(tags)
    assert np.abs(mi(got - moved, w.box)).max() < 1e-12       # set, and not integrated
    own = s.positions(np.arange(w.n - ng))
    assert np.abs(mi(own - mi(w.pos[:w.n - ng], w.box), w.box)).max() > 1e-4   # owned moved
    # no device rebuild: after enough steps the request is pending, the list unbuilt
    n0 = s.info()["n_rebuilds"]
    for _ in range(400):
        s.set_ghost_positions(s.positions(tags))
        s.step(1)
        if s.info()["rebuild_pending"]:
            break
    info = s.info()
    assert info["rebuild_pending"] == 1 and info["n_rebuilds"] == n0
    s.close()


def test_ghost_calls_with_device_buffers():
    import torch
    w = wl.lj_fluid(2000, 0.84, 1.2, seed=912)
    ng = 300
    s = gbmd.System.from_workload(w, precision="fp64", n_ghost=ng)
    tags = torch.arange(w.n - ng, w.n, dtype=torch.int32, device="cuda")
    out = torch.empty((ng, 3), dtype=torch.float64, device="cuda")
    gbmd.gbmd_get_positions_device(s.handle, tags.data_ptr(), ng, out.data_ptr())
    torch.cuda.synchronize()
    host = s.positions(np.arange(w.n - ng, w.n))
    assert np.array_equal(out.cpu().numpy(), host)
    moved = out + 0.01
    gbmd.gbmd_set_ghost_positions(s.handle, moved.data_ptr(), device=True)
    s.sync()
    assert np.abs(mi(s.positions(np.arange(w.n - ng, w.n)) - moved.cpu().numpy(), w.box)).max() < 1e-12
    s.close()

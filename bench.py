#!/usr/bin/env python
"""Benchmark of the LJ MD hot path on GB300 (one JSON line on stdout, rank 0).

Workload (default): the Kob-Andersen 80:20 binary Lennard-Jones mixture,
N = 10^6, rho 1.2, T 1.0, r_cut 2.5 sigma_ij (energy-shifted), r_buff 0.3, dt 0.005,
Morton re-sort every 100 steps, mixed precision (FP32 pair forces, FP64
positions/integration/reductions), seeded synthetic FCC+jitter input.  A "step" is
one velocity-Verlet time step of the whole path: the step kernel (pair force, then
kick, drift, wrap, shadow and the rebuild check) and the conditional
cell-list/neighbour-list rebuild that follows it.

Timing: W untimed warm-up steps, then exactly K steps between CUDA events on the
system's stream.  At 10^6 particles the inputs (the neighbour list alone is ~370 MB)
exceed the 129 MB L2, and the K steps are one gbmd_step(K) call (run as 16-step CUDA
graphs) between one pair of events; smaller workloads write 256 MB between steps so
that every step starts with a cold L2, and each step is then bracketed by its own
pair of events.  A second, shorter pass brackets the
force kernel of every step with its own pair of events (event nodes inside the
step graph) for the roofline figure; those nodes add a few microseconds to a step,
so the headline pass runs without them.  Clocks are sampled with nvidia-smi during
the timed region.  An end-to-end loop through the public API with host buffers
(upload state, run a chunk of steps, read energy and forces back) gives "e2e".

Beside the headline (skipped with --no-sub): the arithmetic peaks measured by the
library's probe, the LJ 64k fluid in mixed precision and on the plain FP64 path
with the FP64 pipe roofline ("vs FP64 plain path"), the 256-replica batched
ensemble against that plain FP64 single-system loop, and a short served stream
(p50/p99 latency).

--impl reference times the CPU oracle (FP64, O(N^2)) on this host's cores on a
bounded sample of the same workload.  Under torchrun each rank runs its own
replica (the path has no collective); value = all ranks' particle-steps / the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-timesteps/sec and TPS (1 GB300) vs FP64 plain path; p50/p99 served latency"
UNIT = "particle-steps/s"
FALLBACK_HBM_GBS = 6800.0
L2_FLUSH_BYTES = 256 << 20


# ---------------------------------------------------------------------------
# multi-rank plumbing (replicas only)
# ---------------------------------------------------------------------------

def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), \
        int(os.environ.get("LOCAL_RANK", 0))


def dist_init(world):
    if world <= 1:
        return None
    import torch
    import torch.distributed as dist
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    dist.init_process_group(backend)
    return dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def reduce_scalar(dist, x: float, op: str) -> float:
    """max or sum of a float over ranks (identity without a process group)."""
    if dist is None:
        return float(x)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.25)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), float(f[3]), f[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[3][k].lower() == "active"})
        loaded = [r for r in rows if r[2] > 200.0] or rows
        return {"sm_mhz": statistics.median(r[0] for r in loaded),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(r[2] for r in rows)}


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def make_workload(name: str, rank: int):
    from paper_1308_5587_gb300 import workloads as wl
    seed = wl.BASE_SEED + rank
    if name == "lj64k":
        return wl.lj_64k(seed), "mixed", 100, \
            "lj_fluid N=64000 rho=0.84 T=1.2 rc=2.5 shifted rbuff=0.4 dt=0.005"
    if name == "lj64k_fp64":   # the same fluid on the plain FP64 path
        return wl.lj_64k(seed), "fp64", 100, \
            "lj_fluid N=64000 rho=0.84 T=1.2 rc=2.5 shifted rbuff=0.4 dt=0.005 fp64"
    if name == "ka1m":
        return wl.ka_1m(seed), "mixed", 100, \
            "kob_andersen_80_20 N=1000000 rho=1.2 T=1.0 rc=2.5sigma_ij rbuff=0.3 dt=0.005 sort=100"
    if name == "plain4k":
        return wl.plain_fp64_4k(seed), "fp64", 0, \
            "lj_fluid N=4000 rho=0.84 T=1.2 rc=2.5 shifted rbuff=0.4 dt=0.005 fp64"
    if name in COLLOID_WORKLOADS:   # size-disperse: the tree list's case
        ratio = 10.0 if "_r10" in name else 5.0
        w = wl.colloid_mixture(250000, ratio=ratio, seed=seed)
        nl = "cell" if name.endswith("_cell") else "tree"
        w.meta["nlist"] = nl
        return w, "mixed", 100, \
            (f"wca_colloid_mixture N={w.n} (250000 d=1 + {w.meta['n_large']} d={ratio:g}) "
             f"phi=0.2+0.2 T=1.0 rc=2^(1/6)sigma_ij rbuff=0.4 dt=0.002 nlist={nl}")
    if name in POTENTIAL_WORKLOADS:   # the other pair potentials on the LJ 64k geometry
        w = wl.potential_64k(name[:-3], seed)
        return w, "mixed", 100, f"{name[:-3]}_fluid N=64000 rho=0.84 T=1.2 {w.meta['pair']} " \
                                "rbuff=0.4 dt=0.005"
    if name in ("paper64k", "paper64k_mixed"):   # Section 5's LJ benchmark, NVT
        prec = "fp64" if name == "paper64k" else "mixed"
        return wl.paper_lj_64k(seed), prec, 100, \
            f"lj_fluid N=64000 rho=0.382 kT=1.2 rc=3.0 shifted rbuff=0.4 dt=0.005 NVT tau=1.0 {prec}"
    raise SystemExit(f"unknown workload {name}")


POTENTIAL_WORKLOADS = ("mie64k", "wca64k", "yukawa64k", "gauss64k")
COLLOID_WORKLOADS = ("colloid250k", "colloid250k_cell", "colloid250k_r10", "colloid250k_r10_cell")


def system_kw(w):
    """system arguments a workload asks for in its meta: the integrator (NVE unless
    NVT) and the neighbour-list builder (cell list unless the tree)"""
    m = w.meta or {}
    kw = {}
    if m.get("integrator") == "nvt":
        kw.update(integrator="nvt", kT=m["kT"], tau=m["tau"])
    if m.get("nlist"):
        kw["nlist"] = m["nlist"]
    return kw


# Section 5: HOOMD-blue v2.6 on one V100, full FP64, this LJ workload (context only)
PAPER_V100_FP64 = 2.75e8


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("k_force.cuh", "k_force.cu", "step_core.cuh", "gbmd_internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1308_5587_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(workload: str, precision: str):
    """dram bytes per force launch from a committed ncu summary, if the kernel is unchanged."""
    p = os.path.join(ROOT, "profiles", "force_traffic.json")
    try:
        d = json.load(open(p))
    except (OSError, ValueError):
        return None
    e = d.get(f"{workload}:{precision}")
    if not e or e.get("kernel_sha") != kernel_source_hash():
        return None
    return float(e["dram_bytes_per_launch"])


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def timed_steps(torch, s, K: int, W: int, flush, stream, dist, force_events: bool = False,
                region: bool = False, counts: dict = None):
    """W warm-up steps, then K steps each bracketed by events on the stream; returns
    per-step milliseconds, per-force-kernel milliseconds (force_events: event nodes
    around the force kernel inside the step graph, which add a few microseconds to
    the step, so the headline pass runs without them) and the number of library
    kernels executed.  region (inputs larger than L2, nothing between steps): the K
    steps are one call, run as the library runs them (16-step CUDA graphs), between
    one pair of events; every step is then given the mean."""
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    for e4 in ev:                    # torch creates the CUDA events at the first record
        for e in e4:
            e.record(stream)
    torch.cuda.synchronize()
    if force_events:
        s.set_force_events(ev[0][1], ev[0][2])   # step graph built with the event nodes
    for _ in range(W):
        if flush is not None:
            flush.zero_()
        s.step(1)
    s.sync()
    barrier(dist)
    torch.cuda.synchronize()
    i0 = s.info()
    l0 = i0["kernel_launches"]
    whole = region and flush is None and not force_events
    if whole:
        ev[0][0].record(stream)
        s.step(K)
        ev[0][3].record(stream)
    else:
        for k in range(K):
            if flush is not None:
                flush.zero_()
            if force_events:
                s.set_force_events(ev[k][1], ev[k][2])
            ev[k][0].record(stream)
            s.step(1)
            ev[k][3].record(stream)
    torch.cuda.synchronize()
    barrier(dist)
    s.sync()
    i1 = s.info()
    l1 = i1["kernel_launches"]
    if counts is not None and "n_rebuilds" in i1:
        counts["rebuilds"] = int(i1["n_rebuilds"] - i0["n_rebuilds"])
    if whole:
        step_ms = np.full(K, ev[0][0].elapsed_time(ev[0][3]) / K)
    else:
        step_ms = np.array([e[0].elapsed_time(e[3]) for e in ev])
    force_ms = None
    if force_events:
        s.set_force_events(None, None)
        force_ms = np.array([e[1].elapsed_time(e[2]) for e in ev])
    return step_ms, force_ms, l1 - l0


def e2e_loop(torch, w, precision, sort_period, stream, dev, chunk: int, iters: int):
    """Public-API loop with host buffers: upload (pinned) state -> `chunk` steps ->
    read energy and forces back; wall-clock per particle-step."""
    from paper_1308_5587_gb300 import gbmd
    n = w.n
    s = gbmd.System.from_workload(w, precision=precision, sort_period=sort_period,
                                  stream=stream, cuda_device=dev, **system_kw(w))
    pos = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
    vel = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
    img = torch.empty((n, 3), dtype=torch.int32, pin_memory=True).numpy()
    frc = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
    pos[:] = w.pos
    vel[:] = w.vel
    img[:] = 0
    for _ in range(2):   # warm-up
        s.set_state(pos, vel, img, 0)
        s.step(chunk)
        s.thermo()
        s.forces(out=frc)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(iters):
        s.set_state(pos, vel, img, 0)
        s.step(chunk)
        th = s.thermo()
        s.forces(out=frc)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    s.close()
    assert math.isfinite(th["pe"])
    return n * chunk * iters / dt, (pos.nbytes + vel.nbytes + img.nbytes) / chunk, \
        (frc.nbytes + 8 * 11) / chunk


def cpu_baseline(w, world_rank):
    """The oracle as it stands: one full O(N^2) force evaluation (the per-step cost
    of its velocity Verlet; the integration itself is O(N)), on all host cores."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    p = w.pairs.as_dict()
    n = w.n
    if n <= 100_000:
        t0 = time.perf_counter()
        oracle.forces(w.pos, w.box, w.types, p)
        dt = time.perf_counter() - t0
        return {"value": n / dt, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
                "sample": f"one full O(N^2) force evaluation of all {n} particles "
                          f"({dt:.2f} s); integration is O(N) and not counted"}
    # about 10 s on 16 cores at N = 10^6 (each sampled particle against all N)
    m = min(n, 49152)
    idx = np.random.default_rng(0).choice(n, m, replace=False)
    t0 = time.perf_counter()
    oracle.forces_subset(w.pos, w.box, w.types, p, idx)
    dt = time.perf_counter() - t0
    return {"value": m / dt, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
            "extrapolated": True,
            "sample": f"forces on {m} sampled particles against all {n} ({dt:.2f} s), "
                      "extrapolated to particle-steps/s (the cost per particle does not "
                      "depend on which particles are sampled)"}


def cpu_single_thread(w):
    """The same oracle on one core: forces of a sample of particles against all N."""
    import oracle
    oracle.build()
    p = w.pairs.as_dict()
    m = min(w.n, 3072)   # about 10 s on one core at N = 10^6
    idx = np.random.default_rng(0).choice(w.n, m, replace=False)
    old = oracle.get_threads()
    oracle.set_threads(1)
    try:
        t0 = time.perf_counter()
        oracle.forces_subset(w.pos, w.box, w.types, p, idx)
        dt = time.perf_counter() - t0
    finally:
        oracle.set_threads(old)
    return {"value": m / dt, "unit": UNIT, "cores": 1, "extrapolated": True,
            "sample": f"forces on {m} sampled particles against all {w.n} ({dt:.2f} s), "
                      "extrapolated to particle-steps/s"}


def run_system(torch, w, precision, sort_period, stream, dist, local, flush, steps, warmup,
               force_path="global", autotune=False, tune_cache=None, sample_clocks=True):
    """Create a system, time `steps` steps (headline pass, no event nodes) and a
    second pass with the force kernel between event nodes; returns the numbers the
    lines below are built from."""
    from paper_1308_5587_gb300 import gbmd
    s = gbmd.System.from_workload(w, precision=precision, sort_period=sort_period,
                                  stream=stream.cuda_stream, cuda_device=local,
                                  force_path=force_path, **system_kw(w))
    if autotune:
        s.autotune(tune_cache)
    clocks = ClockSampler(local) if sample_clocks else None
    if clocks:
        clocks.start()
    step_ms, _, launches = timed_steps(torch, s, steps, warmup, flush, stream, dist,
                                       region=True)
    clk = clocks.stop() if clocks else None
    cnt = {}
    step1_ms, force_ms, _ = timed_steps(torch, s, min(steps, 1000), 3, flush, stream, dist,
                                        force_events=True, counts=cnt)
    info = s.info()
    th = s.thermo()
    s.close()
    assert math.isfinite(th["pe"]), "non-finite energy"
    t_local = float(step_ms.sum()) / 1e3
    t_max = reduce_scalar(dist, t_local, "max")
    units = reduce_scalar(dist, w.n * steps, "sum")
    # the steps that rebuilt the lists (as many as the device counted in the second
    # pass, single-step graphs with the force-kernel event nodes) are its slowest
    med = float(np.median(step1_ms))
    k_reb = min(cnt.get("rebuilds", 0), step1_ms.size)
    reb = np.sort(step1_ms)[step1_ms.size - k_reb:] if k_reb else step1_ms[:0]
    split = {"median_step_ms": round(med, 5),
             "rebuild_steps": int(reb.size), "of_steps": int(step1_ms.size),
             "rebuild_step_ms_mean": round(float(reb.mean()), 5) if reb.size else None,
             "pass": "single-step graphs with event nodes around the force kernel"}
    return {"value": units / t_max, "t_max": t_max, "ms_per_step": 1e3 * t_max / steps,
            "step_ms_mean": float(step_ms.mean()), "force_ms_mean": float(force_ms.mean()),
            "launches": int(launches), "info": info, "clocks": clk, "split": split}


def hbm_roofline(n, nbar, precision, force_ms, step_ms, info, workload):
    """Roofline of the step kernel (pair force + integration) in algorithmic bytes
    per launch: the pair force's own shadow, count and indices (16 + 4 + 4 <n>;
    neighbour positions come from L1/L2) plus the integration's x, v read and
    written (96), build shadow read (16) and next shadow written (16), i.e.
    148 + 4 <n> per particle; FP64 gathers a 32 B own position and also writes its
    next one.  The pair force alone, as a separate kernel writing its force
    (36 + 4 <n>), is given beside it on the same kernel time."""
    peak, peak_kind = measured_peaks()
    if precision == "mixed":
        fused = n * (16 + 4 + 4 * nbar + 96 + 16 + 16)
        k5 = n * (16 + 4 + 4 * nbar + 16)
    else:
        fused = n * (32 + 4 + 4 * nbar + 96 + 16 + 16 + 32)
        k5 = n * (32 + 4 + 4 * nbar + 32)
    achieved = fused / (force_ms * 1e-3) / 1e9
    k5_ach = k5 / (force_ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": recorded_traffic(workload, precision),
            "count": "fused step kernel: N (148 + 4 <n>) B per launch",
            "kernel": (f"k_force_staged<{precision}>" if info["force_path"] == 1 else
                       f"k_force<{precision}> (step mode) tpp={info['threads_per_particle']} "
                       f"block={info['force_block']}"),
            "alg_bytes_per_launch": int(fused), "mean_neighbors": round(nbar, 2),
            "force_ms_mean": round(force_ms, 5), "peak_kind": f"of {peak_kind}",
            "force_share_of_step": round(force_ms / step_ms, 3),
            "k5_only": {"count": "pair force alone: N (36 + 4 <n>) B per launch",
                        "alg_bytes_per_launch": int(k5), "achieved": round(k5_ach, 1),
                        "frac": round(k5_ach / peak, 4)}}


def probe_peaks(torch, local):
    """Arithmetic peaks measured here by the library's probe: FP64 FMA, FP32 FMA and
    the FP64 reciprocal, per second and per SM per clock at the sampled SM clock."""
    from paper_1308_5587_gb300 import gbmd
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    clocks = ClockSampler(local)
    clocks.start()
    out = {}
    for kind, iters in (("dfma", 2048), ("ffma", 65536), ("drcp", 512)):
        best = None
        for _ in range(3):
            ops, ms = gbmd.gbmd_probe_arith(kind, iters)
            rate = ops / (ms * 1e-3)
            best = rate if best is None else max(best, rate)
        out[kind] = {"ops_per_s": best}
    clk = clocks.stop()
    mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz")
    for v in out.values():
        v["per_sm_per_clock"] = round(v["ops_per_s"] / (sms * mhz * 1e6), 3) if mhz else None
    out["sms"] = sms
    out["clocks"] = clk
    out["drcp_in_dfma_slots"] = round(out["dfma"]["ops_per_s"] / out["drcp"]["ops_per_s"], 2)
    return out


def fp64_roofline(n, nbar, force_ms, peaks, r_cut, r_list):
    """Roofline of the FP64 step kernel against the measured FP64 FMA rate.  FP64
    operations (each add, multiply or fused multiply-add counts one) from the
    kernel's arithmetic: a listed pair beyond r_cut is rejected by an FP32 test on
    the fixed-point shadow and takes none; a pair inside r_cut takes the
    displacement (3), r^2 (3), one reciprocal (counted as the DFMA slots it takes,
    measured by the probe), r^-6 (2), the force factor (3) and the three
    accumulations (3); per particle the integration's kicks, drifts, rounding and
    FP64 shadow (13).  The share of listed pairs inside r_cut is the uniform-fluid
    estimate (r_cut / r_list)^3."""
    rcp = peaks["drcp_in_dfma_slots"]
    f_cut = (r_cut / r_list) ** 3
    per_pair = f_cut * (14 + rcp)
    ops = n * (nbar * per_pair + 13)
    achieved = ops / (force_ms * 1e-3)
    peak = peaks["dfma"]["ops_per_s"]
    return {"bound": "fp64", "achieved": round(achieved / 1e12, 4), "peak": round(peak / 1e12, 4),
            "unit": "T FP64 ops/s", "frac": round(achieved / peak, 4), "traffic": None,
            "kernel": "k_force<fp64> (step mode)", "ops_per_launch": int(ops),
            "ops_per_listed_pair": round(per_pair, 2), "share_inside_rcut": round(f_cut, 3),
            "peak_kind": "of measured (gbmd_probe_arith DFMA, this run)"}


def gpu_arm(args):
    import torch
    from paper_1308_5587_gb300 import _build
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = dist_init(world)
    _build.build()
    stream = torch.cuda.current_stream()
    w, precision, sort_period, wdesc = make_workload(args.workload, rank)
    n = w.n
    flush = None
    if n * 500 < 256e6:     # working set < L2: write 256 MB between steps
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    r = run_system(torch, w, precision, sort_period, stream, dist, local, flush, args.steps,
                   args.warmup, args.force_path, args.autotune, args.tune_cache)
    info = r["info"]
    value = r["value"]
    nbar = info["neighbors_total"] / n
    roofline = hbm_roofline(n, nbar, precision, r["force_ms_mean"], r["step_ms_mean"], info,
                            args.workload)
    # second line: the whole step -- the step kernel plus the amortised rebuild, which
    # writes the list (4 <n>) and ~60 B of cell-list and count traffic per particle
    peak, peak_kind = measured_peaks()
    reb = info["n_rebuilds"] / max(info["step"], 1)
    step_bytes = roofline["alg_bytes_per_launch"] + n * reb * (60 + 4 * nbar)
    step_achieved = step_bytes / (r["step_ms_mean"] * 1e-3) / 1e9
    roofline_step = {"bound": "hbm", "achieved": round(step_achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(step_achieved / peak, 4),
                     "alg_bytes_per_step": int(step_bytes), "peak_kind": f"of {peak_kind}"}

    if precision == "fp64":   # the FP64 path is bound by the FP64 pipe, not by memory
        r_cut = float(np.max(w.pairs.rcut))
        roofline = dict(fp64_roofline(n, nbar, r["force_ms_mean"], probe_peaks(torch, local),
                                      r_cut, r_cut + w.r_buff), hbm=roofline)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
           "scaling": "weak",
           "vs_baseline": (value / PAPER_V100_FP64 if args.workload == "paper64k" else None),
           "dtype": "f32 pair forces + f64 integration" if precision == "mixed" else "f64",
           "data": "synthetic (seeded FCC + jitter, Maxwell-Boltzmann; no dataset)",
           "config": {"workload": wdesc, "n": n, "precision": precision,
                      "parallelism": f"replicas x{world}" if world > 1 else "single system",
                      "l2": "flushed between steps (256 MB write)" if flush is not None
                      else "inputs larger than L2 (nlist > 129 MB)",
                      "timed_iteration": ("one MD step per event pair (direct kernel launches)"
                                          if args.no_graphs else
                                          "one MD step per event pair (single-step CUDA graph)"
                                          if flush is not None else
                                          "all K steps between one event pair, as one "
                                          "gbmd_step(K) call (16-step CUDA graphs)"),
                      "threads_per_particle": info["threads_per_particle"],
                      "force_block": info["force_block"], "nlist_capacity": info["nlist_capacity"],
                      "force_path": "staged" if info["force_path"] == 1 else "global",
                      "sort_period": sort_period},
           "tps": args.steps / r["t_max"], "roofline": roofline, "roofline_step": roofline_step,
           "step_split": r["split"],
           "clocks": r["clocks"], "gpu_launches": r["launches"],
           "rebuilds_per_step": round(reb, 4)}

    # end to end through the public API with host buffers
    chunk = 100
    iters = max(3, min(30, args.steps // chunk))
    e2e_v, h2d, d2h = e2e_loop(torch, w, precision, sort_period, stream.cuda_stream, local, chunk,
                               iters)
    e2e_v = reduce_scalar(dist, e2e_v, "sum")
    out["e2e"] = {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                  "d2h_bytes_per_step": int(d2h),
                  "loop": f"{iters} x (set_state from pinned host -> {chunk} steps -> "
                          "thermo + forces to pinned host)"}

    if not args.no_sub and world == 1:
        sub_records(torch, args, out, stream, dist, local)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(w, rank)
        out["cpu_baseline"]["single_thread"] = cpu_single_thread(w)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def sub_records(torch, args, out, stream, dist, local):
    """Beside the headline: the arithmetic peaks, the LJ 64k fluid in mixed precision
    and on the plain FP64 path (with the FP64 roofline), and the batched ensemble
    against that plain FP64 single-system loop."""
    from paper_1308_5587_gb300 import workloads as wl
    peaks = probe_peaks(torch, local)
    out["peaks_probe"] = peaks
    w64 = wl.lj_64k(wl.BASE_SEED)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    k = max(20, min(args.steps, 200))
    mixed = run_system(torch, w64, "mixed", 100, stream, dist, local, flush, k, 5,
                       sample_clocks=False)
    fp64 = run_system(torch, w64, "fp64", 100, stream, dist, local, flush, k, 5,
                      sample_clocks=False)
    nbar64 = fp64["info"]["neighbors_total"] / w64.n
    out["lj64k"] = {
        "workload": "lj_fluid N=64000 rho=0.84 T=1.2 rc=2.5 shifted rbuff=0.4 dt=0.005",
        "steps": k, "l2": "flushed between steps (256 MB write)",
        "mixed": {"value": mixed["value"], "unit": UNIT, "ms_per_step": mixed["ms_per_step"],
                  "roofline": hbm_roofline(w64.n, mixed["info"]["neighbors_total"] / w64.n,
                                           "mixed", mixed["force_ms_mean"],
                                           mixed["step_ms_mean"], mixed["info"], "lj64k")},
        "fp64_plain": {"value": fp64["value"], "unit": UNIT, "ms_per_step": fp64["ms_per_step"],
                       "force_ms_mean": round(fp64["force_ms_mean"], 5),
                       "roofline": fp64_roofline(w64.n, nbar64, fp64["force_ms_mean"], peaks,
                                                 2.5, 2.5 + w64.r_buff)},
        "mixed_over_fp64": round(mixed["value"] / fp64["value"], 2)}
    torch.cuda.synchronize()
    del flush
    b = run_batch(torch, args.replicas, 50, 5, stream, dist, local, autotune=False)
    b["fp64_single_system_loop"] = {"value": fp64["value"], "unit": UNIT,
                                    "what": "plain FP64 path, LJ 64k single system (above)"}
    b["batched_over_fp64_loop"] = round(b["value"] / fp64["value"], 2)
    out["batched"] = b
    out["served"] = served_short(torch, stream, local, fp64["value"])


def served_short(torch, stream, local, fp64_value):
    """A short served stream beside the headline: the served trace's shape (Poisson
    arrivals at 50/s, N log-uniform in [256, 200000], rho, T as the batch) with 48
    requests and their step counts scaled by 1/20 (U{50..2500}), under the 150 GB
    budget.  The full trace (1,000 requests, U{1000..50000} steps) runs for minutes:
    `--workload serve --requests 1000`."""
    from paper_1308_5587_gb300 import serve, workloads as wl
    be = serve.GpuBackend("mixed", stream=stream.cuda_stream, cuda_device=local)
    serve.Scheduler(be, 1 << 40).run([serve.Request(-1, 0.0, 50, 4000,
                                                    dict(n=4000, rho=0.8, T=1.0, seed=1))])
    trace = wl.request_trace(48, 50.0, seed=wl.BASE_SEED + 2000, steps_lo=50, steps_hi=2500)
    summ = serve.Scheduler(be, int(150e9), max_quantum=2000).run(serve.requests_from_trace(trace))
    be.close()
    done = [r for r in summ.records if r.finished is not None]
    value = summ.particle_steps / summ.makespan
    return {"value": value, "unit": UNIT,
            "workload": "served stream: 48 requests, Poisson 50/s, N log-uniform [256, 200000], "
                        "rho U(0.7, 0.9), T U(0.8, 1.5), steps U{50..2500} (the served "
                        "trace's steps / 20), budget 150 GB, mixed",
            "latency_s": {"p50": summ.p50, "p99": summ.p99, "mean": summ.mean,
                          "completed": len(done),
                          "rejected": sum(r.rejected for r in summ.records)},
            "makespan_s": summ.makespan, "quanta": summ.quanta,
            "peak_resident_bytes": summ.peak_resident_bytes,
            "over_fp64_single_system_loop": round(value / fp64_value, 2)}


# ---------------------------------------------------------------------------
# batched ensemble: 256 replicas stepped together (one launch per kernel per step)
# ---------------------------------------------------------------------------

class _BatchStepper:
    """The batch seen through the calls timed_steps makes on a system."""

    def __init__(self, batch, systems):
        self.b, self.systems = batch, systems

    def step(self, k):
        self.b.step(k)

    def sync(self):
        self.b.sync()

    def info(self):
        return {"kernel_launches": self.b.info()["kernel_launches"]}

    def set_force_events(self, a, b):
        self.systems[0].set_force_events(a, b)   # events live in the batch's step graph


def run_batch(torch, replicas, steps, warmup, stream, dist, local, autotune=True):
    """The batched ensemble (replicas of uneven size in one batch), timed like a
    single system; returns a record for the JSON line."""
    from paper_1308_5587_gb300 import gbmd, workloads as wl
    rank, _, _ = dist_env()
    params = wl.replica_params(replicas, seed=wl.BASE_SEED + 1000 * rank)
    ws = [wl.replica(*p) for p in params]
    b = gbmd.Batch("mixed", stream=stream.cuda_stream, cuda_device=local)
    systems = [gbmd.System.from_workload(w, precision="mixed", sort_period=100,
                                         stream=stream.cuda_stream, cuda_device=local)
               for w in ws]
    for x in systems:
        b.add(x)
    if autotune:
        b.autotune(None)
    n = sum(w.n for w in ws)
    clocks = ClockSampler(local)
    clocks.start()
    stepper = _BatchStepper(b, systems)
    step_ms, _, launches = timed_steps(torch, stepper, steps, warmup, None, stream, dist,
                                       region=True)
    clk = clocks.stop()
    step1_ms, force_ms, _ = timed_steps(torch, stepper, min(steps, 500), 3, None, stream, dist,
                                        force_events=True)
    med = float(np.median(step1_ms))
    reb = step1_ms[step1_ms > 1.8 * med]
    infos = [x.info() for x in systems]
    tune = (infos[0]["threads_per_particle"], infos[0]["force_block"])
    th = [x.thermo() for x in systems[:4]]
    assert all(math.isfinite(t["pe"]) for t in th)
    t_max = reduce_scalar(dist, float(step_ms.sum()) / 1e3, "max")
    value = reduce_scalar(dist, n * steps, "sum") / t_max
    alg_bytes = sum(i["n"] * (16 + 4 + 96 + 16 + 16) + 4 * i["neighbors_total"] for i in infos)
    peak, peak_kind = measured_peaks()
    f_mean = float(force_ms.mean())
    achieved = alg_bytes / (f_mean * 1e-3) / 1e9
    for slot in list(b.members):
        b.remove(slot).close()
    b.close()
    return {"value": value, "unit": UNIT, "steps": steps, "warmup": warmup,
            "ms_per_step": 1e3 * t_max / steps, "tps": steps / t_max,
            "workload": f"batched ensemble: {len(ws)} LJ replicas, N_k log-uniform "
                        "[500, 20000], rho U(0.7, 0.9), T U(0.8, 1.5), rc 2.5, "
                        "rbuff 0.4, dt 0.005, mixed",
            "n": n, "replicas": len(ws), "threads_per_particle": tune[0],
            "force_block": tune[1], "autotuned": bool(autotune),
            "l2": "inputs larger than L2",
            "step_split": {"median_step_ms": round(med, 5), "rebuild_steps": int(reb.size),
                           "of_steps": int(step1_ms.size),
                           "rebuild_step_ms_mean": round(float(reb.mean()), 5) if reb.size
                           else None},
            "timed_iteration": "all K steps of every replica between one event pair, as one "
                               "gbmd_batch_step(K) call (16-step CUDA graphs)",
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                         "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None,
                         "kernel": "k_force<mixed> (step mode) over all replicas",
                         "alg_bytes_per_launch": int(alg_bytes),
                         "force_ms_mean": round(f_mean, 5), "peak_kind": f"of {peak_kind}"},
            "clocks": clk, "gpu_launches": int(launches)}


def batch_arm(args):
    import torch
    from paper_1308_5587_gb300 import _build
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = dist_init(world)
    _build.build()
    stream = torch.cuda.current_stream()
    r = run_batch(torch, args.replicas, args.steps, args.warmup, stream, dist, local,
                  autotune=not args.no_autotune)
    out = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32 pair forces + f64 integration",
           "data": "synthetic (seeded FCC + jitter, Maxwell-Boltzmann; no dataset)",
           "config": {"workload": r["workload"], "n": r["n"], "replicas": r["replicas"],
                      "precision": "mixed",
                      "parallelism": f"replicas x{world}" if world > 1 else "one batch",
                      "l2": r["l2"], "timed_iteration": r["timed_iteration"],
                      "threads_per_particle": r["threads_per_particle"],
                      "force_block": r["force_block"]},
           "tps": r["tps"], "roofline": r["roofline"], "step_split": r["step_split"],
           "clocks": r["clocks"], "gpu_launches": r["gpu_launches"], "e2e": None}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# served stream: Poisson arrivals, continuous batching under an HBM budget
# ---------------------------------------------------------------------------

def serve_arm(args):
    import torch
    from paper_1308_5587_gb300 import _build, serve, workloads as wl
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = dist_init(world)
    _build.build()
    stream = torch.cuda.current_stream()
    be = serve.GpuBackend("mixed", stream=stream.cuda_stream, cuda_device=local)
    # warm-up request (module load, first graph capture): not part of the trace
    serve.Scheduler(be, 1 << 40).run([serve.Request(-1, 0.0, 50, 4000,
                                                    dict(n=4000, rho=0.8, T=1.0, seed=1))])
    trace = wl.request_trace(args.requests, args.rate, seed=wl.BASE_SEED + 1000 * rank)
    reqs = serve.requests_from_trace(trace)
    budget = int(args.budget_gb * 1e9)
    sch = serve.Scheduler(be, budget, max_quantum=args.quantum)
    launches0 = be.batch.info()["kernel_launches"]
    clocks = ClockSampler(local)
    clocks.start()
    summ = sch.run(reqs)
    clk = clocks.stop()
    launches = be.batch.info()["kernel_launches"] - launches0
    be.close()
    done = [r for r in summ.records if r.finished is not None]
    t_max = reduce_scalar(dist, summ.makespan, "max")
    value = reduce_scalar(dist, summ.particle_steps, "sum") / t_max
    steps = sum(r.steps for r in done)
    up = sum(r.n * (24 + 24 + 4) for r in done)     # positions, velocities, types
    down = sum(8 * 11 for r in done)                # thermodynamic record per request
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": steps, "warmup": 1, "ms_per_step": None, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32 pair forces + f64 integration",
           "data": "synthetic (seeded Poisson request trace; seeded LJ fluids)",
           "config": {"workload": f"served stream: {len(reqs)} requests, Poisson "
                                  f"{args.rate}/s, N log-uniform [256, 200000], rho U(0.7, 0.9), "
                                  "T U(0.8, 1.5), steps U{1000..50000}, rc 2.5, rbuff 0.4, "
                                  "dt 0.005, mixed",
                      "budget_bytes": budget, "max_quantum": args.quantum,
                      "parallelism": f"replicas x{world}" if world > 1 else "one batch"},
           "latency_s": {"p50": summ.p50, "p99": summ.p99, "mean": summ.mean,
                         "completed": len(done),
                         "rejected": sum(r.rejected for r in summ.records)},
           "makespan_s": summ.makespan, "quanta": summ.quanta,
           "peak_resident_bytes": summ.peak_resident_bytes,
           "clocks": clk, "gpu_launches": int(launches),
           "e2e": {"value": value, "unit": UNIT,
                   "h2d_bytes_per_step": int(up / max(steps, 1)),
                   "d2h_bytes_per_step": int(down / max(steps, 1)),
                   "loop": "whole trace: host inputs generated and uploaded at admission, "
                           "results read back at retirement"}}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle
# ---------------------------------------------------------------------------

def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    if args.workload in ("batch", "serve"):
        raise SystemExit("--impl reference times the single-system workloads "
                         "(lj64k, ka1m, plain4k)")
    w, precision, sort_period, wdesc = make_workload(args.workload, 0)
    p = w.pairs.as_dict()
    n = w.n
    rng = np.random.default_rng(1)
    # size each step's sample so that the whole run takes about two minutes
    probe = rng.choice(n, 32, replace=False)
    t0 = time.perf_counter()
    oracle.forces_subset(w.pos, w.box, w.types, p, probe)
    per_particle = (time.perf_counter() - t0) / 32
    budget = 100.0 / max(args.steps + args.warmup, 1)
    m = int(min(n, max(8, budget / max(per_particle, 1e-9))))
    pos = w.pos.copy()
    vel = w.vel.copy()
    h = 0.5 * w.dt / w.mass

    def one_step(k):
        idx = rng.choice(n, m, replace=False)
        F, _, _ = oracle.forces_subset(pos, w.box, w.types, p, idx)
        vel[idx] += h * F            # the sampled particles' kick; drift below
        pos[idx] += w.dt * vel[idx]

    for k in range(args.warmup):
        one_step(k)
    t0 = time.perf_counter()
    for k in range(args.steps):
        one_step(k)
    dt = time.perf_counter() - t0
    value = m * args.steps / dt
    sample = (f"per step: forces on {m} random particles against all {n} "
              f"(O(m N) of the O(N^2) step) + their kick/drift")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * dt / args.steps * (n / m), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded FCC + jitter, Maxwell-Boltzmann; no dataset)",
           "config": {"workload": wdesc, "n": n, "precision": "fp64 (CPU oracle)",
                      "parallelism": "host cores"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.get_threads(),
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def peaks_arm(args):
    import torch
    from paper_1308_5587_gb300 import _build
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    _build.build()
    p = probe_peaks(torch, local)
    if rank == 0:
        print(json.dumps({"peaks_probe": p, "device": torch.cuda.get_device_name(local)}),
              flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", choices=["gbmd", "reference"], default="gbmd")
    ap.add_argument("--workload", choices=["lj64k", "lj64k_fp64", "ka1m", "plain4k", "paper64k",
                                           "paper64k_mixed",
                                           *POTENTIAL_WORKLOADS, *COLLOID_WORKLOADS,
                                           "batch", "serve"],
                    default="ka1m")
    ap.add_argument("--replicas", type=int, default=256, help="batch workload: replicas")
    ap.add_argument("--no-autotune", action="store_true", help="batch workload: fixed tuning")
    ap.add_argument("--requests", type=int, default=200, help="serve workload: trace length")
    ap.add_argument("--rate", type=float, default=50.0, help="serve workload: arrivals per s")
    ap.add_argument("--budget-gb", type=float, default=150.0, help="serve workload: HBM budget")
    ap.add_argument("--quantum", type=int, default=2000, help="serve workload: max steps per quantum")
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--tune-cache", default=None,
                    help="with --autotune: text file to read / append the tuning choices")
    ap.add_argument("--force-path", choices=["global", "staged"], default="global",
                    help="neighbour gather through L1/L2 by 32-bit index (default) or "
                         "from a shared-memory window by 16-bit index")
    ap.add_argument("--no-sub", "--no-fp64", dest="no_sub", action="store_true",
                    help="skip the sub-records beside the headline (arithmetic peaks, LJ 64k "
                         "mixed and plain FP64, batched ensemble)")
    ap.add_argument("--peaks", action="store_true",
                    help="only run the arithmetic probe (FP64 / FP32 FMA, FP64 reciprocal) and "
                         "print its rates")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graphs", action="store_true",
                    help="launch the same kernels directly instead of through CUDA graphs "
                         "(ncu cannot profile kernels inside graphs with conditional nodes)")
    args = ap.parse_args(argv)
    if args.no_graphs:
        os.environ["GBMD_NO_GRAPHS"] = "1"
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        reference_arm(args)
    elif args.peaks:
        peaks_arm(args)
    elif args.workload == "batch":
        batch_arm(args)
    elif args.workload == "serve":
        serve_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()

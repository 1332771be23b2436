"""The served stream on the GPU: each request's result in the shared batch is
bitwise the result of the same request run alone, every request stops at exactly
its own step count, and admission keeps the resident footprint within the budget."""
import numpy as np
import pytest

from paper_1308_5587_gb300 import gbmd, serve, workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1308_5587_gb300 import _build
    _build.build()


def _requests(count, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    t = 0.0
    for k in range(count):
        t += rng.exponential(0.002)
        n = int(np.exp(rng.uniform(np.log(256), np.log(3000))))
        w = wl.lj_fluid(n, float(rng.uniform(0.7, 0.9)), float(rng.uniform(0.8, 1.5)),
                        seed=9000 + k, r_buff=0.4)
        reqs.append(serve.Request(k, t, int(rng.integers(30, 250)), n, w))
    return reqs


def test_served_results_equal_each_request_alone():
    reqs = _requests(10, seed=31)
    be = serve.GpuBackend("mixed", keep_state=True)
    summ = serve.Scheduler(be, budget_bytes=1 << 40, max_quantum=64).run(reqs)
    be.close()
    assert summ.quanta > 1
    for rec, r in zip(summ.records, sorted(reqs, key=lambda x: x.arrival)):
        assert rec.finished is not None
        pos, vel, img, step = rec.result["state"]
        assert step == r.steps
        s = gbmd.System.from_workload(r.payload, precision="mixed")
        s.step(r.steps)
        p2, v2, i2, st2 = s.state()
        assert st2 == r.steps
        assert np.array_equal(pos, p2) and np.array_equal(vel, v2) and np.array_equal(img, i2)
        assert rec.result["pe"] == s.thermo()["pe"]
        s.close()


def test_admission_respects_a_small_budget():
    reqs = _requests(12, seed=32)
    be = serve.GpuBackend("mixed")
    fps = sorted(be.footprint(r) for r in reqs)
    budget = fps[-1] + fps[-2]          # only a few systems fit at once
    summ = serve.Scheduler(be, budget_bytes=budget, max_quantum=64).run(reqs)
    be.close()
    assert fps[-1] < summ.peak_resident_bytes <= budget
    assert all(r.finished is not None and r.result["step"] == r.steps for r in summ.records)
    # a request's footprint is what the library reports for its description
    w = reqs[0].payload
    d, keep = gbmd.make_desc(w.n, w.box, w.pos, w.vel, w.types, w.pairs.eps, w.pairs.sigma,
                             w.pairs.rcut, w.r_buff, w.dt, w.mass, "mixed")
    rec0 = next(r for r in summ.records if r.rid == 0)
    assert rec0.footprint == gbmd.gbmd_footprint_bytes(d)

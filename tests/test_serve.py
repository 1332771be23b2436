"""Host logic of the served stream (paper_1308_5587_gb300.serve) on a simulated
device: FIFO admission under the byte budget, exact per-request step counts,
quantum bounds, rejection, and latency accounting."""
import math

import pytest

from paper_1308_5587_gb300 import serve, workloads as wl


def _run(reqs, budget, rate=1e9, **kw):
    be = serve.SimBackend(rate=rate)
    sch = serve.Scheduler(be, budget, clock=be.clock, wait=be.wait, **kw)
    quanta = []
    adv = be.advance
    be.advance = lambda k: (quanta.append(k), adv(k))
    return sch.run(reqs), be, quanta


def _trace(count, rate, seed=11):
    tr = wl.request_trace(count, rate, seed=seed, n_lo=256, n_hi=20000, steps_lo=100,
                          steps_hi=3000)
    return serve.requests_from_trace(tr)


def test_every_request_runs_exactly_its_steps_within_the_budget():
    reqs = _trace(60, rate=200.0)
    budget = 700 * 40000
    summ, be, quanta = _run(reqs, budget)
    assert all(r.finished is not None and not r.rejected for r in summ.records)
    for r, q in zip(summ.records, sorted(reqs, key=lambda x: x.arrival)):
        assert r.result["step"] == q.steps
    assert max(b for _, _, _, b in be.log) <= budget
    assert summ.peak_resident_bytes <= budget
    assert all(16 <= k <= 2000 for k in quanta)
    assert summ.particle_steps == sum(q.n * q.steps for q in reqs)


def test_admission_is_first_in_first_out():
    reqs = _trace(40, rate=500.0, seed=12)
    summ, be, _ = _run(reqs, budget=700 * 25000)
    starts = [rid for ev, rid, _, _ in be.log if ev == "start"]
    order = [r.rid for r in sorted(reqs, key=lambda x: (x.arrival, x.rid))]
    assert starts == order
    adm = [r.admitted for r in summ.records]
    assert adm == sorted(adm)


def test_request_larger_than_the_budget_is_rejected():
    reqs = [serve.Request(0, 0.0, 100, 1000), serve.Request(1, 0.0, 100, 10**6),
            serve.Request(2, 0.1, 100, 2000)]
    summ, _, _ = _run(reqs, budget=700 * 5000)
    rec = {r.rid: r for r in summ.records}
    assert rec[1].rejected and rec[1].finished is None
    assert rec[0].finished is not None and rec[2].finished is not None


def test_latency_of_a_lone_request_is_its_service_time():
    # one request: the quantum ends when it finishes, so latency = steps * n / rate
    n, steps, rate = 5000, 1234, 2e8
    summ, _, quanta = _run([serve.Request(0, 0.5, steps, n)], budget=10**9, rate=rate,
                           max_quantum=500)
    assert sum(quanta) == steps and max(quanta) == 500
    assert summ.records[0].latency == pytest.approx(steps * n / rate)
    assert summ.p50 == summ.p99 == pytest.approx(steps * n / rate)


def test_light_load_has_no_queueing():
    # arrivals far apart: every request runs alone
    reqs = [serve.Request(k, 10.0 * k, 200 + 10 * k, 1000 + 100 * k) for k in range(8)]
    summ, _, _ = _run(reqs, budget=10**9, rate=1e8)
    for r in summ.records:
        assert r.admitted == pytest.approx(r.arrival)
        assert r.latency == pytest.approx(r.n * r.steps / 1e8)


def test_percentile_nearest_rank():
    xs = list(range(1, 101))
    assert serve.percentile(xs, 50) == 50
    assert serve.percentile(xs, 99) == 99
    assert serve.percentile(xs, 100) == 100
    assert serve.percentile([3.0], 99) == 3.0


def test_bad_scheduler_arguments():
    be = serve.SimBackend()
    with pytest.raises(ValueError):
        serve.Scheduler(be, 0)
    with pytest.raises(ValueError):
        serve.Scheduler(be, 10, max_quantum=8, min_quantum=16)

"""Continuous batching: cases that share the device give the same result as
when run alone, admission respects the memory budget, and a failing case is
evicted without affecting the others."""
import numpy as np
import pytest

from paper_2507_03366_gb300 import eulbfs, serving
from paper_2507_03366_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FIELDS = ("H", "T", "C", "p", "u", "v")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2507_03366_gb300 import build
    build.build()


def trace(n=6, seed=11):
    rng = np.random.default_rng(seed)
    reqs = []
    for k in range(n):
        side = int(rng.choice([32, 48, 64]))
        case = wl.droplet(side, theta_deg=float(rng.uniform(70, 130)), St=float(rng.uniform(0.1, 0.4)), Tw=-0.5,
                          impact_speed=0.03, name=f"req{k}")
        reqs.append(wl.Request(k, 0.002 * k, case, int(rng.integers(15, 60))))
    return reqs


def alone(case, steps, precision):
    s = eulbfs.Solver([case], precision=precision)
    s.step(steps)
    return s.fields()


@pytest.mark.parametrize("precision", [eulbfs.FP32C, eulbfs.FP64])
def test_served_results_equal_alone(precision):
    reqs = trace()
    rep = serving.serve(reqs, precision=precision, chunk=7, keep_fields=True, realtime=False)
    assert all(o.error is None for o in rep.outcomes)
    assert rep.max_resident >= 2          # the cases overlapped on the device
    for o, r in zip(rep.outcomes, reqs):
        assert o.steps == r.steps
        ref = alone(r.case, r.steps, precision)
        for k in FIELDS:
            assert np.array_equal(o.fields[k], ref[k]), (r.rid, k)


def test_budget_defers_admission_and_all_complete():
    reqs = trace(5, seed=12)
    biggest = max(eulbfs.lib().eulbfs_domain_bytes(r.case.nx, r.case.ny, eulbfs.FP32C) for r in reqs)
    rep = serving.serve(reqs, budget_bytes=biggest + 1024, chunk=5, realtime=False)
    s = rep.summary()
    assert s["completed"] == 5 and s["failed"] == 0
    assert rep.rejected_busy > 0          # some case waited for memory
    assert s["p99_s"] >= s["p50_s"] > 0.0


def test_failing_case_is_evicted_without_affecting_others():
    reqs = trace(4, seed=13)
    bad = wl.droplet(32, theta_deg=90.0, impact_speed=0.03, name="unstable")
    bad.dt = 40.0                          # far beyond the explicit stability bound
    reqs.insert(2, wl.Request(99, 0.001, bad, 60))
    rep = serving.serve(reqs, chunk=6, keep_fields=True, realtime=False)
    by_id = {o.rid: o for o in rep.outcomes}
    assert by_id[99].error is not None and "ENONFINITE" in by_id[99].error
    for r in reqs:
        if r.rid == 99:
            continue
        o = by_id[r.rid]
        assert o.error is None
        ref = alone(r.case, r.steps, eulbfs.FP32C)
        for k in FIELDS:
            assert np.array_equal(o.fields[k], ref[k]), (r.rid, k)


def test_diverged_case_is_evicted_within_one_chunk():
    """A diverging case with a long step limit leaves after the chunk in which
    it diverged instead of holding its slot until its last step."""
    reqs = trace(3, seed=15)
    bad = wl.droplet(32, theta_deg=90.0, impact_speed=0.03, name="unstable_long")
    bad.dt = 40.0
    chunk = 6
    reqs.insert(1, wl.Request(77, 0.001, bad, 100000))
    rep = serving.serve(reqs, chunk=chunk, keep_fields=True, realtime=False)
    by_id = {o.rid: o for o in rep.outcomes}
    assert by_id[77].error is not None and "ENONFINITE" in by_id[77].error
    assert by_id[77].steps <= 2 * chunk, by_id[77].steps
    for r in reqs:
        if r.rid != 77:
            o = by_id[r.rid]
            assert o.error is None and o.steps == r.steps
            ref = alone(r.case, r.steps, eulbfs.FP32C)
            for k in FIELDS:
                assert np.array_equal(o.fields[k], ref[k]), (r.rid, k)


def test_realtime_trace_reports_latency():
    reqs = trace(4, seed=14)
    rep = serving.serve(reqs, chunk=8, realtime=True)
    s = rep.summary()
    assert s["completed"] == 4
    for o in rep.outcomes:
        assert o.finished_s >= o.admitted_s >= o.arrival_s - 1e-9
    assert s["gcups"] > 0

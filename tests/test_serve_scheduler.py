"""Continuous-batching scheduler (serve.Server) with a fake executor: slots, HBM admission, arrival order,
overlap of jobs in flight, failure isolation.  No GPU."""
import threading
import time

import pytest

from paper_2107_10423_gb300 import serve


class FakeExec:
    def __init__(self, service_s=0.05, fail_ids=()):
        self.service_s = service_s
        self.fail_ids = set(fail_ids)
        self.lock = threading.Lock()
        self.active = 0
        self.max_active = 0

    def __call__(self, job):
        with self.lock:
            self.active += 1
            self.max_active = max(self.max_active, self.active)
        time.sleep(self.service_s)
        with self.lock:
            self.active -= 1
        if job.job_id in self.fail_ids:
            raise RuntimeError("injected failure")
        return {"ok": job.job_id}


def _jobs(arrivals, fp=1):
    return [serve.Job(i, a, None, footprint=fp) for i, a in enumerate(arrivals)]


def test_slots_limit_concurrency_and_jobs_overlap():
    ex = FakeExec(0.05)
    srv = serve.Server(max_slots=3, hbm_budget=100, executor=ex)
    jobs = srv.run(_jobs([0.0] * 8))
    assert ex.max_active == 3
    assert all(j.result == {"ok": j.job_id} for j in jobs)
    # 8 jobs of 50 ms on 3 slots: about 3 waves, far less than 8 serial services
    span = max(j.finish for j in jobs)
    assert span < 8 * 0.05 * 0.8


def test_admission_by_memory_budget():
    ex = FakeExec(0.03)
    jobs = _jobs([0.0, 0.0, 0.0, 0.0], fp=60)
    srv = serve.Server(max_slots=4, hbm_budget=100, executor=ex)
    srv.run(jobs)
    assert ex.max_active == 1            # two 60-byte jobs never fit together in 100


def test_arrival_order_and_latency():
    ex = FakeExec(0.02)
    arr = [0.0, 0.05, 0.1, 0.15]
    srv = serve.Server(max_slots=1, hbm_budget=10, executor=ex)
    jobs = srv.run(_jobs(arr))
    starts = [j.start for j in jobs]
    assert starts == sorted(starts)
    for j in jobs:
        assert j.start >= j.arrival - 1e-3 and j.latency >= 0.02 - 1e-3
    s = serve.summarize(jobs)
    assert s["completed"] == 4 and s["p99_latency_s"] >= s["p50_latency_s"] > 0


def test_late_arrival_admitted_while_others_run():
    ex = FakeExec(0.2)
    srv = serve.Server(max_slots=4, hbm_budget=100, executor=ex)
    jobs = srv.run(_jobs([0.0, 0.05]))
    a, b = jobs
    assert b.start < a.finish            # continuous batching: admitted while job 0 is in flight


def test_failed_job_is_isolated():
    ex = FakeExec(0.01, fail_ids=[1])
    srv = serve.Server(max_slots=2, hbm_budget=100, executor=ex)
    jobs = srv.run(_jobs([0.0, 0.0, 0.0]))
    assert "error" in jobs[1].result and jobs[0].result == {"ok": 0} and jobs[2].result == {"ok": 2}
    assert serve.summarize(jobs)["completed"] == 2


def test_oversize_job_rejected():
    srv = serve.Server(max_slots=2, hbm_budget=10, executor=FakeExec())
    with pytest.raises(ValueError):
        srv.run(_jobs([0.0], fp=11))


def test_footprint_grows_with_size():
    from paper_2107_10423_gb300 import synth
    a = serve.footprint_bytes(synth.water_cluster(2, 1, targets="homo_lumo"))
    b = serve.footprint_bytes(synth.water_cluster(8, 1, targets="homo_lumo"))
    assert 0 < a < b


def test_library_footprint_bound_properties():
    """gw_plan_footprint (host only): grows with the system, borrowing B saves exactly its FP64 bytes, the work-space
    cap bounds the work space, and the largest job of the serving stream fits the default HBM budget."""
    from paper_2107_10423_gb300 import gw, synth
    s = synth.water_cluster(8, 1, targets="homo_lumo")
    own = gw.footprint(s.n_occ, s.n_virt, s.n_aux, 2, precision=gw.GW_PREC_MIXED)
    bor = gw.footprint(s.n_occ, s.n_virt, s.n_aux, 2, borrow=True, precision=gw.GW_PREC_MIXED)
    assert own - bor == 8 * (s.n_aux * s.n_ov + 2 * s.n_bas * s.n_aux)
    small = gw.footprint(s.n_occ, s.n_virt, s.n_aux, 2, precision=gw.GW_PREC_MIXED, workspace_mb=64)
    assert small < own
    big = synth.water_cluster(64, 1, targets="homo_lumo")
    fp = serve.footprint_bytes(big, True, serve.workspace_for(big))
    assert fp < serve.Server().hbm_budget

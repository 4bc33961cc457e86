"""Continuous-batching G0W0 job server on one GPU.

Jobs (a synth.System plus host inputs) arrive over time.  The dispatcher admits an arrived job as soon as a slot is
free and its device footprint (B tensors, their mixed-precision copies and work space) fits the HBM budget; each
admitted job runs on its own plan and CUDA stream in a worker thread, so the work of jobs in flight overlaps on the
device while new arrivals keep being admitted.  A job that fails in mixed precision is re-run in FP64.  Latency is
finish time minus arrival time; the summary reports jobs/s, p50 and p99.

The executor is injectable: `run_job` by default (libgw through the ctypes binding), or any callable taking a Job and
returning a dict, which is how the scheduling logic is tested without a GPU.
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Job:
    job_id: int
    arrival: float                 # seconds after the stream starts
    system: object                 # synth.System
    B_ia: np.ndarray = None
    B_nm: np.ndarray = None
    footprint: int = 0             # device bytes reserved while in flight
    result: dict = field(default_factory=dict)
    start: float = 0.0
    finish: float = 0.0

    @property
    def latency(self) -> float:
        return self.finish - self.arrival


def footprint_bytes(system, mixed: bool = True, workspace_mb: int = 0) -> int:
    """Device bytes a job may hold: the library's own bound for a plan of this size (gw_plan_footprint, computed from
    the same caps the plan allocates by), with B_ia and B_nm copied in from the host."""
    from . import gw
    return gw.footprint(system.n_occ, system.n_virt, system.n_aux, len(system.targets), borrow=False,
                        precision=gw.GW_PREC_MIXED if mixed else gw.GW_PREC_FP64, workspace_mb=workspace_mb)


def workspace_for(system) -> int:
    """Work-space cap (MiB) that scales with the job: small jobs keep their buffers small."""
    per_freq = system.n_aux * system.n_aux * 36
    return int(min(8192, max(256, (per_freq * 130) >> 20)))


def run_job(job: Job, precision: str = "mixed", qp: str = "linearised") -> dict:
    """Default executor: one plan (own CUDA stream) for the job, screening + QP solve; FP64 re-run on failure."""
    from . import gw
    s = job.system
    B_ia = job.B_ia if job.B_ia is not None else s.b_ia()     # inputs are generated when the job is admitted
    B_nm = job.B_nm if job.B_nm is not None else s.b_nm()
    mode = gw.GW_QP_LINEARISED if qp == "linearised" else gw.GW_QP_STEPTREE
    tries = [gw.GW_PREC_MIXED, gw.GW_PREC_FP64] if precision == "mixed" else [gw.GW_PREC_FP64]
    last = None
    for prec in tries:
        try:
            with gw.Plan(s.eps, s.n_occ, B_ia, B_nm, s.targets, precision=prec,
                         workspace_mb=workspace_for(s)) as p:
                p.screening()
                e, z, st = p.qp_solve(mode)
            return {"e_qp": e, "z": z, "status": st, "precision": "mixed" if prec == gw.GW_PREC_MIXED else "fp64"}
        except gw.GWError as err:          # mixed failed: fall back to FP64 for this job
            last = err
    return {"error": str(last)}


class Server:
    """Arrival-driven continuous batching with admission by slots and HBM footprint (default budget 250 GiB of the
    GB300's 284 GB, which admits the largest job of the stream, (H2O)_64 in mixed precision, alone)."""

    def __init__(self, max_slots: int = 4, hbm_budget: int = 250 << 30, executor=None, poll_s: float = 0.001):
        self.max_slots = max_slots
        self.hbm_budget = hbm_budget
        self.executor = executor or run_job
        self.poll_s = poll_s
        self.log = []                      # (time, event, job_id) for tests and traces

    def run(self, jobs, time_scale: float = 1.0):
        """Serve `jobs` (arrival times in seconds, scaled by time_scale).  Returns the jobs with timings/results."""
        pending = sorted(jobs, key=lambda j: (j.arrival, j.job_id))
        for j in pending:
            if j.footprint > self.hbm_budget:
                raise ValueError(f"job {j.job_id} needs {j.footprint} bytes, more than the HBM budget")
        inflight = {}
        used = 0
        lock = threading.Lock()
        done_cv = threading.Condition(lock)
        finished = []
        t0 = time.perf_counter()

        def now():
            return (time.perf_counter() - t0) / time_scale

        def worker(job):
            try:
                job.result = self.executor(job)
            except Exception as e:   # a failed job is reported, the server keeps going
                job.result = {"error": repr(e)}
            with lock:
                job.finish = now()
                finished.append(job)
                done_cv.notify_all()

        queue = []
        while pending or queue or inflight:
            t = now()
            while pending and pending[0].arrival <= t:
                queue.append(pending.pop(0))
            with lock:
                for j in finished:
                    inflight.pop(j.job_id, None)
                    used -= j.footprint
                    self.log.append((j.finish, "finish", j.job_id))
                finished.clear()
                # admit in arrival order while a slot is free and the footprint fits (no overtaking)
                while queue and len(inflight) < self.max_slots and used + queue[0].footprint <= self.hbm_budget:
                    j = queue.pop(0)
                    j.start = now()
                    used += j.footprint
                    inflight[j.job_id] = threading.Thread(target=worker, args=(j,), daemon=True)
                    self.log.append((j.start, "start", j.job_id))
                    inflight[j.job_id].start()
                if not pending and not queue and not inflight:
                    break
                wait = self.poll_s
                if pending and not queue:
                    wait = max(0.0, min(wait * 50, (pending[0].arrival - now()) * time_scale))
                done_cv.wait(timeout=max(wait, 1e-4))
        return sorted(jobs, key=lambda j: j.job_id)


def summarize(jobs, makespan: float = None) -> dict:
    lat = np.array([j.latency for j in jobs])
    ok = [j for j in jobs if "error" not in j.result]
    span = makespan if makespan is not None else (max(j.finish for j in jobs) - min(j.arrival for j in jobs))
    return {"jobs": len(jobs), "completed": len(ok), "jobs_per_s": len(ok) / span if span > 0 else None,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_wait_s": float(np.mean([j.start - j.arrival for j in jobs])),
            "fp64_fallbacks": sum(1 for j in ok if j.result.get("precision") == "fp64")}


def make_jobs(stream, n_max: int = None, limit: int = None, mixed: bool = True, inputs: bool = False):
    """Jobs from synth.serving_stream(): (arrival, System) pairs.  The queue keeps the System (sizes, seed, targets)
    and the footprint; the executor generates the host inputs when it runs the job (``inputs=True`` generates them
    here instead)."""
    jobs = []
    for k, (arr, s) in enumerate(stream):
        if n_max is not None and s.meta.get("n_water", 0) > n_max:
            continue
        j = Job(k, arr, s, s.b_ia() if inputs else None, s.b_nm() if inputs else None)
        j.footprint = footprint_bytes(s, mixed, workspace_for(s))
        jobs.append(j)
        if limit is not None and len(jobs) >= limit:
            break
    return jobs

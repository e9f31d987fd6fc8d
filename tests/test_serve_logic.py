"""Admission and scheduling of the serving loop with a fake job runner (CPU, no GPU)."""
import threading
import time

import numpy as np

from paper_2509_15948_gb300 import Song
from paper_2509_15948_gb300.serve import Job, Server, latency_summary


def make_jobs(n, arrivals, sizes):
    return [Job(i, Song(4, 1, [0, 0, -1, -1], 44100), None, None, None, arrival=a, train_steps=10, n_iter=1,
                finetune_steps=5) for i, a in zip(range(n), arrivals)], dict(enumerate(sizes))


class Recorder:
    def __init__(self, duration):
        self.duration = duration
        self.lock = threading.Lock()
        self.running = 0
        self.max_running = 0
        self.events = []

    def __call__(self, job):
        with self.lock:
            self.running += 1
            self.max_running = max(self.max_running, self.running)
            self.events.append(("start", job.job_id, time.perf_counter()))
        time.sleep(self.duration[job.job_id])
        with self.lock:
            self.running -= 1
            self.events.append(("end", job.job_id, time.perf_counter()))
        return {"la_final": float(job.job_id)}


def test_budget_is_never_exceeded_and_admission_is_in_arrival_order():
    jobs, size = make_jobs(6, [0.0, 0.0, 0.0, 0.01, 0.02, 0.03], [40, 30, 50, 20, 60, 10])
    rec = Recorder({i: 0.05 for i in range(6)})
    srv = Server(100, runner=rec, footprint=lambda j: size[j.job_id])
    res = srv.run(jobs)
    assert srv.peak_in_use <= 100 and srv.in_use == 0
    starts = [e[1] for e in rec.events if e[0] == "start"]
    assert starts == sorted(starts)                     # FIFO: no job overtakes an earlier arrival
    assert all(r.error is None and r.la_final == r.job_id for r in res)
    assert all(r.admitted >= r.arrival and r.finished > r.admitted for r in res)


def test_jobs_arriving_later_overlap_with_running_jobs():
    jobs, size = make_jobs(3, [0.0, 0.05, 0.10], [10, 10, 10])
    rec = Recorder({0: 0.4, 1: 0.3, 2: 0.2})
    srv = Server(100, runner=rec, footprint=lambda j: size[j.job_id])
    res = srv.run(jobs)
    assert rec.max_running == 3                          # admitted while the first job still runs
    assert res[2].admitted < res[0].finished
    s = latency_summary(res)
    assert s["jobs"] == 3 and s["failed"] == 0 and s["p50_s"] <= s["p99_s"]


def test_a_failing_job_returns_its_memory():
    jobs, size = make_jobs(3, [0.0, 0.0, 0.0], [60, 60, 60])

    def runner(job):
        if job.job_id == 0:
            raise RuntimeError("boom")
        time.sleep(0.01)
        return {}

    srv = Server(100, runner=runner, footprint=lambda j: size[j.job_id])
    res = srv.run(jobs)
    assert res[0].error.startswith("RuntimeError") and res[1].error is None and res[2].error is None
    assert srv.in_use == 0 and srv.peak_active == 1


def test_oversized_job_is_refused():
    jobs, size = make_jobs(1, [0.0], [200])
    srv = Server(100, runner=lambda j: {}, footprint=lambda j: size[j.job_id])
    try:
        srv.run(jobs)
    except ValueError as e:
        assert "more than the budget" in str(e)
    else:
        raise AssertionError("expected ValueError")

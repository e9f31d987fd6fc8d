"""Serving loop for whole-song search jobs on one GPU, with continuous batching.

A job is one song's mixing-graph search (Alg. 3: console training, then prune / fine-tune rounds).  Jobs
arrive over time.  An admitted job gets its own console (parameters, Adam state, audio, targets and scratch
stay resident on the device until the job ends), its own CUDA stream and its own host worker thread, so the
steps of all admitted jobs are in flight on the GPU together and fill it where one song alone would not.
Admission is by device-memory footprint: the footprint of a job is what mg_plan reports for its console, and
a job is admitted as soon as it fits in the budget left by the running jobs.  Waiting jobs are admitted in
arrival order (a job that does not fit holds back the ones behind it, so large jobs are not starved), and
every finishing job frees its memory and wakes the admission loop.

A job's computation does not depend on the other jobs (its own console, stream and random generators), so
its result is the same alone and in the mix.
"""
from __future__ import annotations

import dataclasses
import threading
import time
from typing import Callable, List, Optional, Sequence

import numpy as np


@dataclasses.dataclass
class Job:
    """One search request: a single song with its dry tracks and target mix."""
    job_id: int
    song: object                      # paper_2509_15948_gb300.Song
    sources: object                   # float32 [K][L]
    target: object                    # float32 [2][L]
    reverb_noise: Optional[object]    # float32 [n_reverbs][2][2 fs] or None
    init_params: Optional[np.ndarray] = None
    train_steps: int = 1000
    n_iter: int = 3
    finetune_steps: int = 500
    lr: float = 1e-2
    tau: float = 0.01
    seed: int = 0
    arrival: float = 0.0              # seconds after the start of the run


@dataclasses.dataclass
class JobResult:
    job_id: int
    arrival: float
    admitted: float
    finished: float
    footprint: int
    track_seconds: float              # K * L / fs of the song
    steps: int                        # console training steps (initial + fine-tuning)
    params: Optional[np.ndarray] = None
    present: Optional[np.ndarray] = None
    la_final: Optional[float] = None
    pruning_ratio: Optional[float] = None
    error: Optional[str] = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class Server:
    """Admission control plus one worker thread per admitted job.

    runner(job) runs the job and returns a dict of result fields; footprint(job) returns its device bytes.
    Both default to the CUDA console (run_search_job / job_footprint); tests pass their own."""

    def __init__(self, budget_bytes: int, runner: Optional[Callable] = None, footprint: Optional[Callable] = None,
                 max_active: int = 64, cfg=None, device: int = 0):
        self.budget = int(budget_bytes)
        self.cfg = cfg
        self.device = device
        self.runner = runner or (lambda job: run_search_job(job, cfg, device))
        self.footprint = footprint or (lambda job: job_footprint(job, cfg))
        self.max_active = max_active
        self._cv = threading.Condition()
        self.in_use = 0
        self.peak_in_use = 0
        self.peak_active = 0

    def run(self, jobs: Sequence[Job]) -> List[JobResult]:
        """Serves `jobs` (arrival times relative to now) to completion; returns results in job order."""
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        future = sorted(jobs, key=lambda j: (j.arrival, j.job_id))
        sizes = {j.job_id: int(self.footprint(j)) for j in jobs}
        for j in jobs:
            if sizes[j.job_id] > self.budget:
                raise ValueError(f"job {j.job_id} needs {sizes[j.job_id]} bytes, more than the budget {self.budget}")
        waiting: List[Job] = []
        results = {}
        active = {}

        def work(job: Job, admitted: float):
            fs = self.cfg.sample_rate if self.cfg is not None else 44100.0
            res = JobResult(job.job_id, job.arrival, admitted, 0.0, sizes[job.job_id],
                            job.song.num_tracks * job.song.num_samples / fs,
                            job.train_steps + job.n_iter * job.finetune_steps)
            try:
                for k, v in (self.runner(job) or {}).items():
                    setattr(res, k, v)
            except Exception as e:  # the job fails alone; its memory is returned
                res.error = f"{type(e).__name__}: {e}"
            res.finished = now()
            with self._cv:
                self.in_use -= sizes[job.job_id]
                del active[job.job_id]
                results[job.job_id] = res
                self._cv.notify_all()

        with self._cv:
            while future or waiting or active:
                t = now()
                while future and future[0].arrival <= t:
                    waiting.append(future.pop(0))
                while waiting and len(active) < self.max_active and \
                        self.in_use + sizes[waiting[0].job_id] <= self.budget:
                    job = waiting.pop(0)
                    self.in_use += sizes[job.job_id]
                    self.peak_in_use = max(self.peak_in_use, self.in_use)
                    th = threading.Thread(target=work, args=(job, now()), daemon=True)
                    active[job.job_id] = th
                    self.peak_active = max(self.peak_active, len(active))
                    th.start()
                if not (future or waiting or active):
                    break
                timeout = max(0.0, future[0].arrival - now()) if future else None
                self._cv.wait(timeout=timeout)
        return [results[j.job_id] for j in jobs]


def job_footprint(job: Job, cfg=None) -> int:
    """Device bytes of the job's console (mg_plan, host only)."""
    from . import ConsoleConfig, plan
    cfg = cfg or ConsoleConfig(retain_spectra=-1)
    return int(plan([job.song], cfg)["device_bytes"]) + (64 << 20)   # + streams, events, graph, torch tensors


def run_search_job(job: Job, cfg=None, device: int = 0) -> dict:
    """Runs one job on its own console and stream; frees the console before returning."""
    import torch
    from . import Console, ConsoleConfig
    from .search import search
    cfg = cfg or ConsoleConfig(retain_spectra=-1)
    torch.cuda.set_device(device)
    con = Console([job.song], [job.sources], [job.target], job.reverb_noise, cfg)
    try:
        with torch.cuda.stream(con.stream):
            if job.init_params is not None:
                con.set_params(job.init_params)
            res = search(con, job.n_iter, job.train_steps, job.finetune_steps, lr=job.lr, tau=job.tau,
                         seed=job.seed)
            params = con.get_params().cpu().numpy()
        return {"params": params, "present": res.present, "la_final": res.la_final[0],
                "pruning_ratio": res.pruning_ratio[0]}
    finally:
        con.close()


def latency_summary(results: Sequence[JobResult]) -> dict:
    """p50 / p99 job latency (arrival to completion) and aggregate training throughput."""
    lat = np.array([r.latency for r in results if r.error is None])
    span = max(r.finished for r in results) - min(r.arrival for r in results)
    ts = sum(r.track_seconds * r.steps for r in results if r.error is None)
    errors = sorted({r.error for r in results if r.error is not None})
    return {"jobs": len(results), "failed": sum(r.error is not None for r in results), "errors": errors[:3],
            "p50_s": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_s": float(np.percentile(lat, 99)) if lat.size else None,
            "span_s": float(span), "track_s_per_s": float(ts / span) if span > 0 else None}

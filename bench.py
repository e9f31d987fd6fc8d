#!/usr/bin/env python
"""Throughput benchmark of the mixing-console hot path: forward + loss + backward + Adam per song, in
track-seconds of audio per second.

One step = one CUDA-graph replay of forward_loss + backward + adam_step over every song of the batch (all
processor types, dry/wet, subgroup and master sums, multi-resolution STFT loss, regularisers).  Default
workload: 64 songs with 4-32 tracks, 1-8 subgroups and 5-30 s at 44.1 kHz (uneven batch in one persistent
launch per processor type).  Inputs are resident in HBM and far larger than L2 (no flush needed).

Multi-GPU: songs are independent, so N ranks run N independent replicas (weak scaling, no collective).
--impl reference times the FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

FS = W.FS
STREAM_BYTES_PER_SAMPLE = 8  # one stereo FP32 sample


# ------------------------------------------------------------------------------------------------
# workloads
# ------------------------------------------------------------------------------------------------
def workload_layouts(name: str, rank: int = 0, songs: int = 64):
    if name == "uneven":
        return (W.layout_uneven_batch(songs, seed=2 + 1000 * rank),
                f"uneven batch: {songs} songs, K~U{{4..32}}, S~U{{1..8}}, 5-30 s")
    if name == "search":
        return [W.layout_single_search()], "single search song: 16 tracks x 10 s, 4 subgroups"
    if name == "plain":
        return [W.layout_plain()], "plain console: 4 tracks x 2 s, one subgroup of 2"
    raise ValueError(name)


def source_bank(n: int = 24, seconds: float = 30.0, key: int = 0):
    return [W.source_track((0xBA, key, i), int(seconds * FS)) for i in range(n)]


def song_sources_from_bank(bank, layout, song: int):
    """Crops of the seeded bank (pink-noise bursts + decaying notes, peak -6 dBFS), one per track."""
    out = np.empty((layout.num_tracks, layout.num_samples), np.float32)
    for k in range(layout.num_tracks):
        b = bank[(7 * song + 3 * k) % len(bank)]
        off = (song * 9973 + k * 7919) % max(1, b.shape[0] - layout.num_samples + 1)
        x = b[off: off + layout.num_samples]
        if x.shape[0] < layout.num_samples:
            x = np.pad(x, (0, layout.num_samples - x.shape[0]))
        out[k] = x
    return out


def model_bytes(layouts, types="ecnsgdr"):
    """Algorithmic bytes of one fwd+bwd step: 5 stereo streams per processor node (forward reads u, writes y;
    backward reads dy and u, writes du), 2 per input plus 2 per output of each mix sum, 2 for the loss."""
    nt = len([t for t in "ecnsgdr" if t in types])
    tot = 0
    per_type = {t: 0 for t in "ecnsgdr"}
    for l in layouts:
        chains = l.num_tracks + l.num_subgroups
        ungrouped = sum(1 for g in l.track_group if g < 0)
        streams = 5 * nt * chains + 2 * (l.num_tracks - ungrouped) + 2 * l.num_subgroups + 2 * (l.num_subgroups + ungrouped) + 2 + 2
        tot += streams * l.num_samples * STREAM_BYTES_PER_SAMPLE
        for t in "ecnsgdr":
            if t in types:
                per_type[t] += 5 * chains * l.num_samples * STREAM_BYTES_PER_SAMPLE
    return tot, per_type


# FP32 peak of the GB300 from its unit counts: 152 SMs x 128 FP32 lanes x 2 flops per FMA x the SM clock
N_SM, FP32_LANES = 152, 128


def fp32_peak_tflops(sm_mhz: float) -> float:
    return N_SM * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12


def rfft_flops(n) -> float:
    """2.5 n log2 n flops per real FFT of size n."""
    n = float(n)
    return 2.5 * n * math.log2(n) if n > 1 else 0.0


def model_flops(layouts, types="ecnsgdr", fs=FS, n_fft=(512, 2048, 8192), hop_div=4, warmup=0):
    """Algorithmic FP32 flops of one fwd+bwd step, counting FFTs only (2.5 n log2 n per real FFT of size n):
    * reverb r and delay d: one FFT convolution per node at the linear-convolution length n = L + Nh - 1
      (Nh = 2 fs taps for r; 20 slots of round(0.1 fs) plus 38 for d), 12 real FFTs per node and step
      (forward: u, h and the inverse, per channel; backward: dy, and the inverses to du and dL/dh, per
      channel); r adds its FIR synthesis, a 384-point inverse STFT of mid and side (Eqs. 9-10) and its adjoint;
    * equalizer e (2047 taps): overlap-save with 8192-point blocks of 6146 outputs, 8 real FFTs per block
      (forward: u and the inverse per channel; backward: dy and the inverse to du per channel) plus 4 per node
      (filter spectrum, inverse of the tap correlation);
    * loss: per resolution n and frame, the two channels' forward STFTs and their two adjoint inverses
      (4 real FFTs of n; the target spectra are computed once, M and S follow from L and R by linearity)."""
    nh_r = int(round(2 * fs))
    D = int(round(0.1 * fs))
    nh_d = 20 * D + 38
    rev_frames = (nh_r - 384) // 192 + 1
    out = {"e": 0.0, "r": 0.0, "d": 0.0, "loss": 0.0}
    for l in layouts:
        chains = l.num_tracks + l.num_subgroups
        L = l.num_samples
        if "r" in types:
            out["r"] += chains * (12 * rfft_flops(L + nh_r - 1) + 4 * rev_frames * rfft_flops(384))
        if "d" in types:
            out["d"] += chains * 12 * rfft_flops(L + nh_d - 1)
        if "e" in types:
            blocks = -(-L // 6146)
            out["e"] += chains * (8 * blocks + 4) * rfft_flops(8192)
        for n in n_fft:
            hop = n // hop_div
            frames = (L - n) // hop + 1 if L >= n else 0
            frames -= min(frames, -(-warmup // hop))
            out["loss"] += 4 * frames * rfft_flops(n)
    return out


# ------------------------------------------------------------------------------------------------
# clocks sampling during the timed region
# ------------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, device_index: int = 0):
        self.idx = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# Algorithmic bytes per complex point of a node's four-step FFT grid (N = f 2^k points) moved by one launch of
# the row kernels of the reverb/delay convolution with retained spectra (reads and writes of the N-point
# arrays T1, T2, Hz): k_row_bwd2 reads the dL/dy_bar spectrum, Hz and the input spectrum and writes dU and dH;
# k_row_conv reads the input spectrum and Hz and writes the kept spectrum and the product; k_row_fwd_hz
# transforms Hz in place.
KERNEL_BYTES_PER_POINT = {"row_bwd2": 40, "row_conv": 32, "row_hz": 16}
# ncu DRAM bytes (read + write) per grid point of k_row_bwd2, from the one-song capture summarised in
# profiles/, valid while the kernel's sources hash to KERNEL_SRC_SHA1 (otherwise the traffic is reported null)
ROW_BWD2_DRAM_BYTES_PER_POINT = 32.46
KERNEL_SRC_SHA1 = "394c99fdfa5d785c1b617b5e76eb85ba5c8fde5a"
KERNEL_SRCS = ("k_conv_rowbwd.cu", "k_conv_common.cuh", "mg_fftp.cuh", "mg_fft.cuh", "mg_internal.cuh")


def kernel_src_sha1():
    import hashlib
    h = hashlib.sha1()
    for name in KERNEL_SRCS:
        with open(os.path.join(ROOT, "paper_2509_15948_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def aggregate_over_ranks(elapsed_ms: float, units: float, world: int):
    """Whole-job timing of a weak-scaling run (each rank its own batch): the maximum of the ranks' elapsed times
    and the sum of the units they processed, over the default process group (NCCL on GPUs, gloo on CPUs).  One
    rank returns its own values."""
    if world <= 1:
        return elapsed_ms, units
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([elapsed_ms], dtype=torch.float64, device=dev)
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------------------------------------
# oracle timing (CPU baseline / reference arm)
# ------------------------------------------------------------------------------------------------
def oracle_sample_step(layout, seed=0):
    """One FP64 oracle fwd+bwd on a bounded sample song; returns (seconds, track-seconds)."""
    import torch
    from oracle import console as OC
    songs = [OC.SongSpec(layout.num_tracks, layout.num_subgroups, layout.track_group, layout.num_samples)]
    bank = [W.source_track((0xBA, 0, i), layout.num_samples) for i in range(layout.num_tracks)]
    src = [np.stack(bank)]
    types = W.processor_types([layout])
    noise = W.reverb_noise((seed,), sum(t == "r" for t in types))
    gt, keep = W.ground_truth(types, (seed, 77))
    tgt = OC.Console(songs, src, None, noise).render_targets(gt, keep)
    con = OC.Console(songs, src, tgt, noise)
    params = W.init_params(types, (seed, 5))
    t0 = time.perf_counter()
    con.loss_and_grad(params, alpha_p=1e-4)
    dt = time.perf_counter() - t0
    return dt, layout.num_tracks * layout.num_samples / FS, torch.get_num_threads()


def cpu_sample_layout():
    # a bounded sample shaped like the workload's songs: 4 tracks x 2 s, one subgroup of 2 tracks
    return W.layout_plain(2 * FS), "4 tracks x 2 s (1 subgroup) of the workload, one fwd+bwd per step"


def run_reference(args, metric, config):
    import torch
    torch.set_num_threads(os.cpu_count() or 1)
    lay, desc = cpu_sample_layout()
    for _ in range(max(0, args.warmup)):
        oracle_sample_step(lay)
    tot_t, tot_ts = 0.0, 0.0
    for _ in range(args.steps):
        dt, ts, cores = oracle_sample_step(lay)
        tot_t += dt
        tot_ts += ts
    value = tot_ts / tot_t
    line = {"impl": "reference", "metric": metric, "value": value, "unit": "track-s/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config,
            "cpu_baseline": {"value": value, "unit": "track-s/s", "cores": torch.get_num_threads(), "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": "track-s/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------------
def build_console(layouts, rank, per_song_seed=0):
    import torch
    import paper_2509_15948_gb300 as M
    from paper_2509_15948_gb300 import build as B
    B.build()
    bank = source_bank(key=rank)
    sources = [song_sources_from_bank(bank, l, s) for s, l in enumerate(layouts)]
    songs = [M.Song(l.num_tracks, l.num_subgroups, l.track_group, l.num_samples) for l in layouts]
    types = W.processor_types(layouts)
    noise = W.reverb_noise((rank, 9), sum(t == "r" for t in types))
    zeros = [np.zeros((2, l.num_samples), np.float32) for l in layouts]
    t0 = time.perf_counter()
    con = M.Console(songs, sources, zeros, noise, M.ConsoleConfig(autotune=1))
    create_s = time.perf_counter() - t0
    # ground-truth targets rendered by the console itself (seeded graph keeping ~1/3 of the processors)
    gt, keep = W.ground_truth(types, (rank, 77))
    gtp = gt.copy()
    gtp[con.n_proc_params:] = 30.0          # w = sigmoid(30) * keep = keep in FP32
    con.set_params(gtp)
    _, mixes = con.forward_loss(mask=keep, with_mix=True)
    mixes = [m.cpu().numpy() for m in mixes]
    for s in range(len(layouts)):
        con.update_audio(s, torch.as_tensor(sources[s]), torch.as_tensor(mixes[s]))
    con.set_params(W.init_params(types, (rank, 5)))
    con.set_alpha_p(1e-4)
    torch.cuda.synchronize()
    con.create_seconds = create_s
    return con, sources, mixes


def prepare_serving_jobs(args, rank):
    """Songs of the serving run (drawn like the uneven batch), their sources, reverb noises and targets (each
    job's ground-truth graph rendered by a console, outside any timed region)."""
    import torch
    import paper_2509_15948_gb300 as M
    layouts = W.layout_uneven_batch(args.serve_jobs, seed=40 + rank)
    bank = source_bank(key=100 + rank)
    sources = [song_sources_from_bank(bank, l, s) for s, l in enumerate(layouts)]
    songs = [M.Song(l.num_tracks, l.num_subgroups, l.track_group, l.num_samples) for l in layouts]
    types = [W.processor_types([l]) for l in layouts]
    noises = [W.reverb_noise((rank, 11, j), sum(t == "r" for t in types[j])) for j in range(len(layouts))]
    targets = []
    for j, l in enumerate(layouts):
        zeros = [np.zeros((2, l.num_samples), np.float32)]
        con = M.Console([songs[j]], [sources[j]], zeros, noises[j], M.ConsoleConfig(retain_spectra=-1))
        gt, keep = W.ground_truth(types[j], (rank, 78, j))
        gt[con.n_proc_params:] = 30.0
        con.set_params(gt)
        _, mixes = con.forward_loss(mask=keep, with_mix=True)
        targets.append(mixes[0].cpu().numpy())
        con.close()
    torch.cuda.synchronize()
    return songs, sources, types, noises, targets


def serving_run(args, rank, rate, prepared):
    """Serving under a Poisson stream of search jobs at `rate` jobs/s (0: all at once), with continuous
    batching and admission by footprint."""
    import paper_2509_15948_gb300 as M
    from paper_2509_15948_gb300.serve import Job, Server, latency_summary
    songs, sources, types, noises, targets = prepared
    rng = np.random.default_rng(0x5E + rank)
    n = len(songs)
    t_arr = np.cumsum(rng.exponential(1.0 / rate, n)) if rate > 0 else np.zeros(n)
    t_arr -= t_arr[0]
    jobs = [Job(j, songs[j], sources[j], targets[j], noises[j], init_params=W.init_params(types[j], (rank, 6, j)),
                train_steps=args.serve_train_steps, n_iter=args.serve_rounds, finetune_steps=args.serve_finetune_steps,
                seed=j, arrival=float(t_arr[j])) for j in range(n)]
    budget = int(args.serve_budget_gb * (1 << 30))
    srv = Server(budget, cfg=M.ConsoleConfig(retain_spectra=-1))
    res = srv.run(jobs)
    out = latency_summary(res)
    out.update({"arrival_rate_jobs_per_s": rate if rate > 0 else "burst",
                "budget_gb": args.serve_budget_gb, "peak_gb_admitted": srv.peak_in_use / (1 << 30),
                "peak_concurrent_jobs": srv.peak_active,
                "schedule": f"{args.serve_train_steps} Adam steps + {args.serve_rounds} x (dry/wet round, "
                            f"{args.serve_finetune_steps} steps)",
                "jobs_desc": "K~U{4..32}, S~U{1..8}, 5-30 s at 44.1 kHz, one song per job",
                "mean_pruning_ratio": float(np.mean([r.pruning_ratio for r in res if r.error is None]))})
    return out


def _round_record(trials):
    return [(t.song, t.type, tuple(int(i) for i in t.candidates), t.la, t.accepted) for t in trials]


def search_run(args, rank):
    """The single-song search: 16 tracks x 10 s in 4 subgroups, the target rendered from a seeded ground-truth
    graph keeping about a third of the processors; Adam (lr 1e-2) for search_train steps, then search_rounds x
    {dry/wet round (Alg. 3), prune, search_finetune steps}.  Before the search, from the trained state, one
    brute-force round and one dry/wet round are timed with one full masked render per trial (one mask per
    call) and with speculative windows over the batched scorer, and their trial sequences compared."""
    import torch
    import paper_2509_15948_gb300 as M
    from paper_2509_15948_gb300 import search as GS
    lay = W.layout_single_search()
    bank = source_bank(key=300 + rank, seconds=10.0)
    src = song_sources_from_bank(bank, lay, 0)
    types = W.processor_types([lay])
    noise = W.reverb_noise((rank, 17), sum(t == "r" for t in types))
    song = M.Song(lay.num_tracks, lay.num_subgroups, lay.track_group, lay.num_samples)
    con = M.Console([song], [src], [np.zeros((2, lay.num_samples), np.float32)], noise, M.ConsoleConfig(autotune=1))
    gt, keep = W.ground_truth(types, (rank, 80))
    gt[con.n_proc_params:] = 30.0
    con.set_params(gt)
    _, mixes = con.forward_loss(mask=keep, with_mix=True)
    con.update_audio(0, torch.as_tensor(src), mixes[0].clone())
    con.set_params(W.init_params(types, (rank, 8)))
    sync = lambda: con.stream.synchronize()
    out = {"workload": "16 tracks x 10 s, 4 subgroups; Adam lr 1e-2 x %d, then %d x {dry/wet round, prune, %d steps}"
                       % (args.search_train, args.search_rounds, args.search_finetune)}
    # training of the search (the first phase), timed
    t0 = time.perf_counter()
    res = GS.search(con, 0, args.search_train, 0, lr=1e-2, tau=0.01, seed=rank)
    sync()
    out["train_s"] = time.perf_counter() - t0
    # rounds from the trained state: one trial per call with full renders, then speculative windows
    l_min = res.l_min
    rounds = {}
    for name, fn in (("brute_force", GS.brute_force_round), ("dry_wet", GS.dry_wet_round)):
        rec = {}
        for mode, (full, window) in (("per_trial_full_render", (True, 1)), ("batched_windows", (False, 16))):
            con.set_score_mode(full)
            fn(con, l_min, 0.01, [GS.SplitMix64(GS.song_seed(rank, 0))], window=window)   # warm-up
            sync()
            calls = [0]
            orig = con.prune_scores

            def counted(masks, _o=orig):
                calls[0] += 1
                return _o(masks)
            con.prune_scores = counted
            t1 = time.perf_counter()
            _, _, trials = fn(con, l_min, 0.01, [GS.SplitMix64(GS.song_seed(rank, 0))], window=window)
            sync()
            dt = time.perf_counter() - t1
            con.prune_scores = orig
            rec[mode] = {"wall_s": dt, "trials": len(trials), "trials_per_s": len(trials) / dt,
                         "calls": calls[0], "accepted": sum(t.accepted for t in trials), "_seq": _round_record(trials)}
        con.set_score_mode(False)
        a, b = rec["per_trial_full_render"], rec["batched_windows"]
        rec["same_trials"] = a.pop("_seq") == b.pop("_seq")
        rec["speedup"] = a["wall_s"] / b["wall_s"]
        rounds[name] = rec
    out["rounds_from_trained_state"] = rounds
    # the rest of the search: rounds, pruning and fine-tuning
    t0 = time.perf_counter()
    res2 = GS.search(con, args.search_rounds, 0, args.search_finetune, lr=1e-2, tau=0.01, seed=rank,
                     ramp_steps=(2 * args.search_rounds * args.search_finetune) // 3)
    sync()
    out["rounds_and_finetune_s"] = time.perf_counter() - t0
    out["wall_s"] = out["train_s"] + out["rounds_and_finetune_s"]
    out["seconds"] = {"train": out["train_s"], "rounds": res2.seconds["rounds"], "finetune": res2.seconds["finetune"]}
    out["la_after_training"] = float(res.la_final[0])
    out["la_final"] = float(res2.la_final[0])
    out["pruning_ratio"] = float(res2.pruning_ratio[0])
    out["trials_per_round"] = [len(t) for t in res2.trials]
    out["accepted_per_round"] = [sum(x.accepted for x in t) for t in res2.trials]
    out["processors"] = int(con.n_processors)
    out["ground_truth_kept"] = int(np.sum(keep))
    con.close()
    return out


def long_song_run(args, rank):
    """64 tracks x 60 s in 8 subgroups, FFT-domain recomputation (retain_spectra = -1): fwd+bwd+Adam
    throughput and the console's device footprint against the 40 GB activation budget."""
    import torch
    import paper_2509_15948_gb300 as M
    lay = W.layout_long()
    bank = source_bank(key=200 + rank, seconds=60.0)
    src = song_sources_from_bank(bank, lay, 0)
    types = W.processor_types([lay])
    noise = W.reverb_noise((rank, 13), sum(t == "r" for t in types))
    song = M.Song(lay.num_tracks, lay.num_subgroups, lay.track_group, lay.num_samples)
    con = M.Console([song], [src], [np.zeros((2, lay.num_samples), np.float32)], noise,
                    M.ConsoleConfig(retain_spectra=-1))
    gt, keep = W.ground_truth(types, (rank, 79))
    gt[con.n_proc_params:] = 30.0
    con.set_params(gt)
    _, mixes = con.forward_loss(mask=keep, with_mix=True)
    con.update_audio(0, torch.as_tensor(src), mixes[0].clone())
    con.set_params(W.init_params(types, (rank, 7)))
    con.set_alpha_p(1e-4)
    for _ in range(2):
        con.train_step(lr=1e-2)
    con.stream.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(con.stream)
    for _ in range(args.long_steps):
        losses = con.train_step(lr=1e-2)
    b.record(con.stream)
    con.stream.synchronize()
    ms = a.elapsed_time(b) / args.long_steps
    info = con.get_info()
    out = {"workload": "64 tracks x 60 s, 8 subgroups, FFT-domain recomputation", "ms_per_step": ms,
           "track_s_per_s": info["track_seconds"] / (ms / 1e3), "device_gb": info["device_bytes"] / (1 << 30),
           "budget_gb": 40, "losses_finite": bool(torch.isfinite(losses).all().item()), "steps": args.long_steps}
    con.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="uneven", choices=["uneven", "search", "plain"])
    ap.add_argument("--songs", type=int, default=64, help="songs of the uneven batch (smaller: profiling cases)")
    ap.add_argument("--profiler-range", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    ap.add_argument("--prof-steps", type=int, default=3, help="instrumented steps of the stage split")
    ap.add_argument("--per-node-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-baseline-steps", type=int, default=3)
    ap.add_argument("--long-steps", type=int, default=3, help="steps of the 64 x 60 s song (0: skip)")
    ap.add_argument("--serve-jobs", type=int, default=16, help="search jobs of the serving run (0: skip)")
    ap.add_argument("--serve-rate", type=float, default=2.0, help="Poisson arrival rate, jobs/s (0: burst)")
    ap.add_argument("--serve-budget-gb", type=float, default=24.0)
    ap.add_argument("--serve-sweep", default="", help="comma-separated arrival rates (jobs/s, 0 = all at once); "
                                                       "one serving run per rate over the same jobs")
    ap.add_argument("--serve-train-steps", type=int, default=60)
    ap.add_argument("--serve-rounds", type=int, default=3)
    ap.add_argument("--serve-finetune-steps", type=int, default=20)
    ap.add_argument("--search-train", type=int, default=2000, help="single-song search: Adam steps (0: skip)")
    ap.add_argument("--search-rounds", type=int, default=5)
    ap.add_argument("--search-finetune", type=int, default=500)
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    metric = "console fwd+bwd track-s/s batched vs per-node GPU; search-job p50/p99 latency"
    layouts, wdesc = workload_layouts(args.workload, rank, args.songs)
    config = {"workload": wdesc, "songs": len(layouts), "tracks": sum(l.num_tracks for l in layouts),
              "subgroups": sum(l.num_subgroups for l in layouts),
              "seconds": round(sum(l.num_samples for l in layouts) / FS, 2), "sample_rate": FS,
              "types": "ecnsgdr", "loss": "MRSTFT 512/2048/8192 hop 1/4, 96 Mel, A-weighted; L_g, L_p; Adam lr 1e-2",
              "parallelism": f"replicas x{world}", "l2": "inputs far larger than L2 (no flush needed)"}

    if args.impl == "reference":
        if rank == 0:
            run_reference(args, metric, config)
        return

    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dev = torch.cuda.current_device()
    con, sources, mixes = build_console(layouts, rank)
    info = con.get_info()
    track_seconds = info["track_seconds"]
    create_s = round(con.create_seconds, 2)
    # autotuned four-step splits: "N = f 2^k -> N1 = f 2^a" with the number of nodes using each
    fft_splits = {}
    for f, logn, logn1 in con.fft_sizes():
        if f:
            key = f"{f}*2^{logn} -> N1 {f}*2^{logn1}"
            fft_splits[key] = fft_splits.get(key, 0) + 1
    tot_bytes, type_bytes = model_bytes(layouts)

    for _ in range(args.warmup):
        con.train_step(lr=1e-2)
    torch.cuda.synchronize()
    launches_per_step = con.get_info()["launches_per_step"]

    # ---------------- timed region (device time, CUDA events on the console's stream) ----------------
    # the graph is replayed without per-launch events: the headline carries no instrumentation
    clocks = ClockSampler(dev)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if args.profiler_range:
        torch.cuda.profiler.start()
    ev0.record(con.stream)
    for _ in range(args.steps):
        losses = con.train_step(lr=1e-2)
    ev1.record(con.stream)
    torch.cuda.synchronize()
    if args.profiler_range:
        torch.cuda.profiler.stop()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    elapsed_ms = ev0.elapsed_time(ev1)
    elapsed_ms, job_track_seconds = aggregate_over_ranks(elapsed_ms, track_seconds, world)
    ms_per_step = elapsed_ms / args.steps
    value = job_track_seconds / (ms_per_step / 1e3)
    finite = bool(torch.isfinite(losses).all().item())

    # ---------------- stage split: a separate pass with CUDA events around every launch ----------------
    prof_steps = max(1, args.prof_steps)
    con.set_profiling(True)
    con.train_step(lr=1e-2)               # captures the instrumented graph
    torch.cuda.synchronize()
    con.reset_kernel_times()
    pa = torch.cuda.Event(enable_timing=True)
    pb = torch.cuda.Event(enable_timing=True)
    pa.record(con.stream)
    for _ in range(prof_steps):
        con.train_step(lr=1e-2)
    pb.record(con.stream)
    torch.cuda.synchronize()
    prof_ms_per_step = pa.elapsed_time(pb) / prof_steps
    stage = con.stage_times()
    fam = con.kernel_times()
    con.set_profiling(False)
    con.train_step(lr=1e-2)               # back to the uninstrumented graph for the legs below
    torch.cuda.synchronize()

    # roofline of the dominant stage (largest device time per step among the processor types): its algorithmic
    # bytes (5 stereo FP32 streams per node-sample) over its CUDA-event time per step; the whole step the same
    # way; the FP32-ALU fraction of the FFT stages under the flop model; and the four-step row kernel against
    # the bytes of its own FFT grid (an implementation figure, kept for comparison)
    peak, peak_kind = measured_peaks()
    stage_step = {k: v[0] / prof_steps for k, v in stage.items()}
    proc_stages = {k: v for k, v in stage_step.items() if k in "ecnsgdr"}
    dom = max(proc_stages, key=lambda k: proc_stages[k])
    dom_ms = proc_stages[dom]
    stage_achieved = type_bytes[dom] / (dom_ms / 1e3) / 1e9
    step_achieved = tot_bytes / (ms_per_step / 1e3) / 1e9
    sm_clk = clk.get("sm_max_mhz") or 2070.0
    fpk = fp32_peak_tflops(sm_clk)
    flops = model_flops(layouts)
    alu = {}
    for k, fl in flops.items():
        t = stage_step.get(k, 0.0)
        if fl > 0 and t > 0:
            tf = fl / (t / 1e3) / 1e12
            alu[k] = {"model_gflop": fl / 1e9, "ms_per_step": t, "achieved_tflops": tf, "frac": tf / fpk}
    roofline = {"bound": "hbm", "kernel": f"stage {dom} (every fwd+bwd launch of its type, per step)",
                "achieved": stage_achieved, "peak": peak, "unit": "GB/s", "frac": stage_achieved / peak,
                "traffic": None, "model_bytes": type_bytes[dom], "ms_per_step": dom_ms,
                "byte_model": "5 stereo FP32 streams per node-sample (fwd reads u, writes y; bwd reads dy, u, "
                              "writes du)",
                "peak_source": f"{peak_kind} hbm_gbs (copy burst)",
                "step": {"achieved": step_achieved, "frac": step_achieved / peak, "model_bytes": tot_bytes,
                         "ms_per_step": ms_per_step},
                "alu": {"peak_tflops": fpk, "peak_source": f"{N_SM} SMs x {FP32_LANES} FP32 lanes x 2 x {sm_clk:.0f} MHz",
                        "flop_model": "FFTs only, 2.5 n log2 n per real FFT of size n", "stages": alu},
                "instrumented_ms_per_step": prof_ms_per_step}
    fam_step = {k: (v[0] / prof_steps, v[1] / prof_steps) for k, v in fam.items() if v[1] > 0}
    ptypes = con.processor_types()
    grid_points = sum(int(f) << int(logn) for (f, logn, _), t in zip(con.fft_sizes(), ptypes) if f and t in "dr")
    if "row_bwd2" in fam_step and grid_points:
        launches = fam_step["row_bwd2"][1]
        ms_launch = fam_step["row_bwd2"][0] / launches
        bytes_launch = KERNEL_BYTES_PER_POINT["row_bwd2"] * grid_points / launches
        achieved = bytes_launch / (ms_launch / 1e3) / 1e9
        traffic = None
        if ROW_BWD2_DRAM_BYTES_PER_POINT and KERNEL_SRC_SHA1 == kernel_src_sha1():
            traffic = ROW_BWD2_DRAM_BYTES_PER_POINT * grid_points / launches
        roofline["kernel_grid"] = {"kernel": "k_row_bwd2", "achieved": achieved, "frac": achieved / peak,
                                   "traffic": traffic, "bytes_per_launch": bytes_launch, "ms_per_launch": ms_launch,
                                   "launches_per_step": launches,
                                   "byte_model": f"{KERNEL_BYTES_PER_POINT['row_bwd2']} B per complex point of the "
                                                 f"FFT grid, {grid_points} points"}

    # ---------------- one launch per node (same kernels, one-by-one processing) ----------------
    per_node = None
    if args.per_node_steps > 0:
        con.set_launch_mode(True)
        con.train_step(lr=1e-2)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(con.stream)
        for _ in range(args.per_node_steps):
            con.train_step(lr=1e-2)
        b.record(con.stream)
        torch.cuda.synchronize()
        pn_total, pn_units = aggregate_over_ranks(a.elapsed_time(b), track_seconds, world)
        pn_ms = pn_total / args.per_node_steps
        per_node = {"value": pn_units / (pn_ms / 1e3), "ms_per_step": pn_ms,
                    "batched_speedup": pn_ms / ms_per_step}
        con.set_launch_mode(False)

    # ---------------- end to end through the public API, host buffers ----------------
    e2e = None
    if args.e2e_steps > 0:
        pinned_src = [torch.as_tensor(s).pin_memory() for s in sources]
        pinned_tgt = [torch.as_tensor(m).pin_memory() for m in mixes]
        host_losses = torch.empty(con.n_songs, 7, dtype=torch.float32).pin_memory()
        h2d = sum(s.numel() * 4 + t.numel() * 4 for s, t in zip(pinned_src, pinned_tgt))
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            for s in range(con.n_songs):
                con.update_audio_host(s, pinned_src[s].numpy(), pinned_tgt[s].numpy())
            l = con.train_step(lr=1e-2)
            host_losses.copy_(l, non_blocking=False)
        torch.cuda.synchronize()
        e2e_total_ms, e2e_units = aggregate_over_ranks(1e3 * (time.perf_counter() - t0), track_seconds, world)
        e2e_s = e2e_total_ms / 1e3 / args.e2e_steps
        e2e = {"value": e2e_units / e2e_s, "unit": "track-s/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(host_losses.numel() * 4), "ms_per_step": 1e3 * e2e_s}

    # ---------------- CPU baseline: the oracle on a bounded sample ----------------
    cpu = None
    if rank == 0 and args.cpu_baseline_steps > 0:
        torch.set_num_threads(os.cpu_count() or 1)
        lay, desc = cpu_sample_layout()
        tt, ts = 0.0, 0.0
        for _ in range(args.cpu_baseline_steps):
            dt, tsec, cores = oracle_sample_step(lay)
            tt += dt
            ts += tsec
        cpu = {"value": ts / tt, "unit": "track-s/s", "cores": torch.get_num_threads(), "kind": "oracle",
               "sample": desc + f", {args.cpu_baseline_steps} steps"}

    serving, long_song, search = None, None, None
    dev_bytes = info["device_bytes"]
    if args.serve_jobs > 0 or args.long_steps > 0 or args.search_train > 0:
        con.close()
        del con
        torch.cuda.synchronize()
    if args.long_steps > 0:
        long_song = long_song_run(args, rank)
    if args.search_train > 0:
        search = search_run(args, rank)
    if args.serve_jobs > 0:
        prepared = prepare_serving_jobs(args, rank)
        rates = [float(r) for r in args.serve_sweep.split(",")] if args.serve_sweep else [args.serve_rate]
        sweep = [serving_run(args, rank, r, prepared) for r in rates]
        serving = sweep[0] if len(sweep) == 1 else {"sweep": sweep}

    if rank == 0:
        line = {"metric": metric, "value": value, "unit": "track-s/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config, "roofline": roofline,
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches_per_step * args.steps),
                "clocks": clk, "per_node": per_node, "losses_finite": finite,
                "stages_ms_per_step": stage_step,
                "kernel_families_ms_per_step": {k: v[0] for k, v in fam_step.items()},
                "device_bytes": dev_bytes, "fft_splits": fft_splits, "console_create_s": create_s,
                "long_song": long_song, "serving": serving, "search": search}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()

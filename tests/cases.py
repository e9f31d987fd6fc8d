"""Shared builders for parity cases: the same seeded inputs feed the FP64 oracle and the CUDA console."""
from __future__ import annotations

import dataclasses
import json
import os
from typing import List, Optional, Sequence

import numpy as np

import workloads as W
from oracle import console as OC
from oracle import loss as OL
from oracle import graph as OG

LOSS_FIELDS = ("La", "Llr", "Lm", "Ls", "Lg", "Lp", "total")


@dataclasses.dataclass
class Case:
    layouts: List[W.SongLayout]
    types: str
    sources: list
    targets: list
    noise: Optional[np.ndarray]
    ptypes: List[str]
    params: np.ndarray
    n_fft: Sequence[int]
    n_mels: int
    oracle: OC.Console
    fs: int = W.FS
    warmup: int = 0


def make_case(layouts: Sequence[W.SongLayout], types: str = "ecnsgdr", seed: int = 0, n_fft=(512, 2048, 8192),
              n_mels: int = 96, a_weighting: bool = True, warmup: int = 0, param_key=None, fs: int = W.FS) -> Case:
    layouts = list(layouts)
    songs = [OC.SongSpec(l.num_tracks, l.num_subgroups, l.track_group, l.num_samples) for l in layouts]
    sources = [W.song_sources(l, (seed, i), fs) for i, l in enumerate(layouts)]
    ptypes = W.processor_types(layouts, types)
    n_rev = sum(t == "r" for t in ptypes)
    noise = W.reverb_noise((seed,), max(1, n_rev), fs) if n_rev else None
    ldesc = OL.LossDesc(sample_rate=float(fs), n_fft=tuple(n_fft), n_mels=n_mels, a_weighting=a_weighting,
                        warmup_samples=warmup)
    desc = OC.ConsoleDesc(sample_rate=float(fs), types=types, loss=ldesc)
    gt, keep = W.ground_truth(ptypes, (seed, 77))
    targets = OC.Console(songs, sources, None, noise, desc).render_targets(gt, keep)
    oracle = OC.Console(songs, sources, targets, noise, desc)
    params = W.init_params(ptypes, (seed, 5) if param_key is None else param_key)
    return Case(layouts, types, sources, targets, noise, ptypes, params, tuple(n_fft), n_mels, oracle, fs, warmup)


def gpu_console(case: Case, **cfg_kw):
    """The CUDA console of a case: same songs, sources, targets, noises, sample rate and loss settings."""
    import paper_2509_15948_gb300 as M
    songs = [M.Song(l.num_tracks, l.num_subgroups, l.track_group, l.num_samples) for l in case.layouts]
    kw = dict(types=case.types, n_fft=case.n_fft, n_mels=case.n_mels, sample_rate=float(case.fs),
              warmup_samples=case.warmup)
    kw.update(cfg_kw)
    return M.Console(songs, case.sources, case.targets, case.noise, M.ConsoleConfig(**kw))


def rel_l2(a, b) -> float:
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / den) if den > 0 else float(np.linalg.norm(a - b))


def oracle_with_delay_taps(case: Case, alpha_p: float):
    """Oracle losses, gradients and mixes, plus for every delay processor, from the forward/backward of the same
    call: (dL/dh, its 39-tap FIRs c_m, |u| its input's magnitude, dL/dy_bar = w dL/dy its wet adjoint)."""
    import torch
    from oracle import processors as OP
    cap = []
    orig = OP.DelayScatter.apply

    def hook(c, zr, zi, D, L):
        t = orig(c, zr, zi, D, L)
        if t.requires_grad:
            t.retain_grad()
            cap.append((t, c.detach().numpy()))
        return t

    OP.DelayScatter.apply = hook
    try:
        x = torch.tensor(np.asarray(case.params, np.float64), dtype=torch.float64, requires_grad=True)
        res = case.oracle.forward(x, alpha_p=alpha_p, keep_outputs=True)
        dprocs = [p for p in case.oracle.procs if p.type == "d"]
        for p in dprocs:
            res[p.song]["outputs"][p.index].retain_grad()
        sum(r["total"] for r in res).backward()
    finally:
        OP.DelayScatter.apply = orig
    losses = np.array([[float(r[k].detach()) for k in ("La", "Llr", "Lm", "Ls", "Lg", "Lp", "total")] for r in res])
    grads = x.grad.detach().numpy().copy()
    mixes = [r["mix"].detach().numpy() for r in res]
    q = np.asarray(case.params, np.float64)[case.oracle.n_proc_params:]
    taps = {}
    for p, (t, c) in zip(dprocs, cap):
        o = res[p.song]["outputs"]
        u_abs = np.abs(o[("in", p.index)].detach().numpy())
        dybar = o[p.index].grad.numpy() / (1.0 + np.exp(-q[p.index]))
        taps[p.index] = (t.grad.numpy(), c, u_abs, dybar)
    return losses, grads, mixes, taps


def lag_correlation(a, b, nh: int, n0: int = -19):
    """c[j] = sum_n a[n] b[n - j] at the tap lags j = n0 .. n0 + nh - 1 (both [2][L]), per channel, FP64."""
    L = a.shape[1]
    M = 1 << int(np.ceil(np.log2(2 * L + nh)))
    lags = (np.arange(nh) + n0) % M
    return np.stack([np.fft.irfft(np.fft.rfft(a[ch], M) * np.conj(np.fft.rfft(b[ch], M)), M)[lags] for ch in range(2)])


def delay_term_rms(case: Case, alpha_p: float = 1e-3, D: int = None, n0: int = -19) -> dict:
    """Per delay processor and channel: rms over the tap lags of A[j] = sum_n |dL/dy_bar[n]| |u[n - j]|, the
    magnitudes of the terms whose sum is dL/dh[j] (dL/dy_bar taken as w dL/dy from the oracle's intermediates).
    Near an optimum dL/dh cancels strongly (A is 4-2000x its rms), and FP32 rounding of the upstream adjoint
    bounds dL/dh's accuracy by a fraction of A rather than of dL/dh."""
    import torch
    D = D or int(round(0.1 * case.fs))
    params = torch.tensor(np.asarray(case.params, np.float64), requires_grad=True)
    res = case.oracle.forward(params, alpha_p=alpha_p, keep_outputs=True)
    for r in res:
        for v in r["outputs"].values():
            if isinstance(v, torch.Tensor) and v.requires_grad:
                v.retain_grad()
    sum(r["total"] for r in res).backward()
    q = np.asarray(case.params, np.float64)[case.oracle.n_proc_params:]
    out = {}
    for p in case.oracle.procs:
        if p.type != "d":
            continue
        o = res[p.song]["outputs"]
        u = np.abs(o[("in", p.index)].detach().numpy())
        db = np.abs(o[p.index].grad.numpy()) / (1.0 + np.exp(-q[p.index]))
        L = u.shape[1]
        nh = 20 * D + 38                      # taps of Eq. (17): 20 slots of D plus the 39-tap FIR span
        M = 1 << int(np.ceil(np.log2(2 * L + nh)))
        lags = (np.arange(nh) + n0) % M
        rms = np.zeros(2)
        for ch in range(2):
            c = np.fft.irfft(np.fft.rfft(db[ch], M) * np.conj(np.fft.rfft(u[ch], M)), M)
            rms[ch] = np.sqrt(np.mean(c[lags] ** 2))
        out[p.index] = rms
    return out


def delay_slot_conditioning(case: Case, taps: dict, D: int = None, term_rms: dict = None):
    """Per delay processor, channel and tap m: kappa = |g_m| / (rms(dL/dh) ||c_m|| ||s'||), the ratio of the
    Eq. (19) inner product g_m to its Cauchy-Schwarz scale (how far g_m stands above cancellation).  With
    term_rms (delay_term_rms) the scale uses the rms of the summed term magnitudes instead of rms(dL/dh)."""
    from oracle import processors as OP
    D = D or int(round(0.1 * case.fs))
    out = {}
    for p in case.oracle.procs:
        if p.type != "d":
            continue
        dh, cvals = taps[p.index][:2]
        kap = np.zeros((2, 20))
        for ch in range(2):
            rms = term_rms[p.index][ch] if term_rms is not None else np.sqrt(np.mean(dh[ch] ** 2))
            for m in range(20):
                o = p.offset + (ch * 20 + m) * 22
                z = complex(case.params[o], case.params[o + 1])
                sp = OP.surrogate_impulse_dz(z / max(1.0, abs(z)), D)
                G = np.lib.stride_tricks.sliding_window_view(dh[ch, m * D: m * D + D + 38], 39) @ cvals[ch, m]
                scale = rms * np.linalg.norm(cvals[ch, m]) * np.linalg.norm(sp)
                kap[ch, m] = abs(np.sum(G * np.conj(sp))) / scale if scale > 0 else 0.0
        out[p.index] = kap
    return out


def grad_groups(case: Case):
    """Index arrays of the gradient per processor type (parameters) and of the dry/wet logits."""
    procs = case.oracle.procs
    out = {}
    for t in "ecnsgdr":
        idx = [np.arange(p.offset, p.offset + p.count) for p in procs if p.type == t]
        if idx:
            out[t] = np.concatenate(idx)
    out["q"] = np.arange(case.oracle.n_proc_params, case.oracle.n_params)
    return out


def record_error(test: str, quantity: str, err: float, plain_bound: float, bound: float, **extra):
    """Append one measured parity error (with the plain bound of the quantity and the bound the test applied) to
    the JSON-lines file named by MG_PARITY_REPORT, when that variable is set; a no-op otherwise."""
    path = os.environ.get("MG_PARITY_REPORT")
    if not path:
        return
    rec = {"test": test, "quantity": quantity, "err": float(err), "plain_bound": float(plain_bound),
           "bound": float(bound)}
    rec.update({k: v.item() if hasattr(v, "item") else v for k, v in extra.items()})
    with open(path, "a") as f:
        f.write(json.dumps(rec) + "\n")


def current_test() -> str:
    return os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]


def console_graph(layout, types="ecnsgdr"):
    """The console of one song as a graph (Sec. 1.2): input -> chain per track, mix node -> chain per subgroup,
    output summing the subgroup chains, then the ungrouped tracks; processors numbered in the console's
    canonical order."""
    chain = [t for t in "ecnsgdr" if t in types]
    ntype, track, edges = [], [], []

    def node(t, k=-1):
        ntype.append(t)
        track.append(k)
        return len(ntype) - 1

    def add_chain(src):
        last = src
        for t in chain:
            v = node("ecnsgdr".index(t))
            edges.append((last, v))
            last = v
        return last
    K, S = layout.num_tracks, layout.num_subgroups
    inputs = [node(OG.INPUT, k) for k in range(K)]
    # processors must come in canonical order (tracks' chains, then subgroups' chains), so nodes are created
    # chain by chain; the mix nodes get their edges after the track chains exist
    track_out = [add_chain(inputs[k]) for k in range(K)]
    group_out = []
    for g in range(S):
        m = node(OG.MIX)
        for k in range(K):
            if layout.track_group[k] == g:
                edges.append((track_out[k], m))
        group_out.append(add_chain(m))
    o = node(OG.OUTPUT)
    for g in range(S):
        edges.append((group_out[g], o))
    for k in range(K):
        if layout.track_group[k] < 0:
            edges.append((track_out[k], o))
    return ntype, track, edges


def random_dag(n_tracks: int, n_proc: int, n_mix: int, seed: int):
    """A seeded random processing graph: the inputs, then processors (every type at least once) and mix nodes in a
    random order, each with one to three predecessors among the nodes before it, and the output fed by every
    node nothing else reads (so that every node reaches the output).  Edges run from lower to higher index."""
    rng = np.random.default_rng(seed)
    ntype = [OG.INPUT] * n_tracks
    track = list(range(n_tracks))
    kinds = list(range(7)) + [int(t) for t in rng.integers(0, 7, n_proc - 7)] + [OG.MIX] * n_mix
    rng.shuffle(kinds)
    edges = []
    for t in kinds:
        v = len(ntype)
        k = int(rng.integers(1, 4))
        preds = sorted(set(int(u) for u in rng.integers(0, v, k)))
        edges += [(u, v) for u in preds]
        ntype.append(int(t))
        track.append(-1)
    o = len(ntype)
    ntype.append(OG.OUTPUT)
    track.append(-1)
    has_succ = {u for u, _ in edges}
    for v in range(o):
        if v not in has_succ:
            edges.append((v, o))
    return ntype, track, edges

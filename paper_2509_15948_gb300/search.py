"""Mixing-graph search (Alg. 2 with brute-force sampling, Alg. 3 with dry/wet sampling, and the hybrid of the
two; Sec. 6.1-6.3) on the CUDA console.

Every song of a console runs its own search.  The songs advance together: one mg_prune_scores call evaluates
the next trials of every song at once, because a song's audio loss L_a depends only on its own processors, and
each song submits a window of its next trials drawn on the assumption that they fail (_run_trials), which the
batched scorer evaluates over one base render.  The decisions equal those of one trial at a time.  Training
between rounds is the console's CUDA-graph step (forward, backward, Adam).

Readings where the paper is silent:
  * N_t is fixed when the round starts; the candidate count is k = max(1, floor(N_t r_t + 0.5)) capped at
    |V_t| (the rounding of Alg. 3 can give 0, which would never end the round);
  * the least-weight nodes are ordered by (w, processor index), w = sigmoid(q) in double precision from the
    FP32 logits;
  * SampleType draws from the remaining types kept in chain order e c n s g d r with the splitmix64
    generator (Steele, Lea, Flood 2014): index = next() mod |T_c|; one generator per song, seeded with
    song_seed(seed, song);
  * a type whose node set V_t has become empty leaves T_c when it is drawn (the draw is consumed);
  * a failed trial with k > 1 halves r_t, a failed trial with k = 1 removes the type;
  * L_min is the unmasked L_a after the initial training and is only updated by accepted trials (Alg. 3);
  * the sparsity weight alpha_p rises linearly from 0 to alpha_p_max over the first ramp_steps fine-tuning
    steps (Sec. 6.3: 0 to 1e-4 over the first 4k of 6k steps) and stays there;
  * brute force: the pool holds the song's present processors in ascending order, v = pool[next() mod |pool|],
    and a tried processor leaves the pool whatever the outcome; hybrid: brute force on iterations 4, 8, ...
"""
from __future__ import annotations

import dataclasses
import time
from typing import Dict, List, Optional, Sequence

import numpy as np

TYPE_ORDER = "ecnsgdr"
_M64 = (1 << 64) - 1


class SplitMix64:
    """splitmix64 (Steele, Lea, Flood, OOPSLA 2014): state += golden gamma, then two xor-shift-multiply
    rounds and a final xor-shift."""

    def __init__(self, seed: int):
        self.s = seed & _M64

    def next(self) -> int:
        self.s = (self.s + 0x9E3779B97F4A7C15) & _M64
        x = self.s
        x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & _M64
        return x ^ (x >> 31)


def song_seed(seed: int, song: int) -> int:
    """Seed of song `song`'s type sampler."""
    return (seed * 0x100000001B3 + song + 1) & _M64


def dry_wet_weights(q: np.ndarray) -> np.ndarray:
    """w = sigmoid(q) in double precision (Sec. 3.1 dry/wet weights)."""
    q = np.asarray(q, np.float64)
    return 1.0 / (1.0 + np.exp(-q))


@dataclasses.dataclass
class Trial:
    song: int
    type: str
    candidates: tuple          # processor indices (console-wide) switched off by the trial
    la: float                  # L_a of the song with the trial mask
    accepted: bool


class _SongRound:
    """State of one song's pruning round (Alg. 3, inner loop)."""

    def __init__(self, procs: Sequence[int], types: Sequence[str], w: np.ndarray, l_min: float, rng: SplitMix64):
        self.w = w
        self.tc = [t for t in TYPE_ORDER if any(types[i] == t for i in procs)]
        self.V = {t: [i for i in procs if types[i] == t] for t in self.tc}
        self.N = {t: len(self.V[t]) for t in self.tc}
        self.r = {t: 0.1 for t in self.tc}
        self.removed: set = set()     # processors switched off by accepted trials
        self.l_min = float(l_min)
        self.rng = rng
        self.pending: Optional[tuple] = None

    def advance(self) -> bool:
        """Draws the next trial; False when the round of this song is over."""
        while self.tc:
            t = self.tc[self.rng.next() % len(self.tc)]
            if not self.V[t]:
                self.tc.remove(t)
                continue
            k = min(max(1, int(np.floor(self.N[t] * self.r[t] + 0.5))), len(self.V[t]))
            order = sorted(self.V[t], key=lambda i: (self.w[i], i))
            self.pending = (t, tuple(order[:k]))
            return True
        self.pending = None
        return False

    def resolve(self, la: float, tau: float) -> Trial:
        t, cand = self.pending
        ok = la < self.l_min + tau
        if ok:
            self.l_min = min(self.l_min, la)
            self.removed.update(cand)
            drop = set(cand)
            self.V[t] = [i for i in self.V[t] if i not in drop]
            self.pending = None
        else:
            self.fail()
        return t, cand, ok

    def fail(self):
        """The state after the pending trial fails: r_t halves (k > 1) or the type leaves T_c (k = 1)."""
        t, cand = self.pending
        if len(cand) > 1:
            self.r[t] /= 2.0
        else:
            self.tc.remove(t)
        self.pending = None

    def clone(self) -> "_SongRound":
        c = _SongRound.__new__(_SongRound)
        c.w, c.tc, c.V, c.N, c.r = self.w, list(self.tc), {t: list(v) for t, v in self.V.items()}, self.N, dict(self.r)
        c.removed, c.l_min, c.rng, c.pending = set(self.removed), self.l_min, SplitMix64(0), self.pending
        c.rng.s = self.rng.s
        return c

    def candidates(self):
        return self.pending[1]


def _run_trials(con, songs, tau: float, window: int, on_trial) -> None:
    """Runs the trials of every song's round (objects with advance / resolve / fail / clone / candidates).

    Every prune_scores call carries, per song, its next trials up to the song's window, drawn on a copy of its
    state on the assumption that each of them fails (the next trial of a round follows from the state alone).
    The results are taken in order up to the song's first accepted trial: every mask taken up to there is
    exactly the mask of a one-trial-at-a-time round (a song's L_a depends only on its own processors), so the
    decisions and scores are those of that round; the song's later masks lacked the accepted candidates and
    are discarded.  A song's window doubles (up to `window`) when all its trials were taken and shrinks to
    twice what was taken otherwise.  window = 1 is the plain round, one mask per call."""
    P = con.n_processors
    active = [sr.advance() for sr in songs]
    win = [min(window, 4)] * len(songs)
    while any(active):
        chains = []
        for s, sr in enumerate(songs):
            chain = []
            if active[s]:
                st = sr.clone()
                while True:
                    chain.append(st.candidates())
                    if len(chain) >= win[s]:
                        break
                    st.fail()
                    if not st.advance():
                        break
            chains.append(chain)
        masks = np.ones((max(len(c) for c in chains), P), np.uint8)
        for s, sr in enumerate(songs):
            for i in sr.removed:
                masks[:, i] = 0
            for b, cand in enumerate(chains[s]):
                for i in cand:
                    masks[b, i] = 0
        la = con.prune_scores(masks).cpu().numpy().astype(np.float64)
        for s, sr in enumerate(songs):
            taken = 0
            for b, cand in enumerate(chains[s]):
                assert tuple(sr.candidates()) == tuple(cand)
                ok = on_trial(s, sr, float(la[b, s]))
                taken += 1
                active[s] = sr.advance()
                if ok or not active[s]:
                    break
            if chains[s]:
                win[s] = min(window, 2 * win[s]) if taken == len(chains[s]) else max(1, min(window, 2 * taken))


def dry_wet_round(con, l_min: Sequence[float], tau: float, rngs: Sequence[SplitMix64],
                  w: Optional[np.ndarray] = None, window: int = 16) -> tuple:
    """One pruning round of Alg. 3 for every song of `con`, in lockstep.

    Returns (keep mask [P] uint8 over all processors, updated L_min per song, list of Trial)."""
    types = con.processor_types()
    _, _, song_of = con.layout()
    present = con.present()
    if w is None:
        w = dry_wet_weights(con.get_params().cpu().numpy()[con.n_proc_params:])
    P = con.n_processors
    songs = []
    for s in range(con.n_songs):
        procs = [i for i in range(P) if song_of[i] == s and present[i]]
        songs.append(_SongRound(procs, types, w, l_min[s], rngs[s]))
    trials: List[Trial] = []

    def on_trial(s, sr, la):
        t, cand, ok = sr.resolve(la, tau)
        trials.append(Trial(s, t, cand, la, ok))
        return ok
    _run_trials(con, songs, tau, window, on_trial)
    keep = present.astype(np.uint8).copy()
    for sr in songs:
        for i in sr.removed:
            keep[i] = 0
    return keep, [sr.l_min for sr in songs], trials


class _SongBrute:
    """State of one song's brute-force round: every pool processor is tried alone (Sec. 6.2)."""

    def __init__(self, procs: Sequence[int], l_min: float, rng: SplitMix64):
        self.pool = sorted(procs)
        self.removed: set = set()
        self.l_min = float(l_min)
        self.rng = rng
        self.pending: Optional[int] = None

    def advance(self) -> bool:
        if not self.pool:
            self.pending = None
            return False
        self.pending = self.pool[self.rng.next() % len(self.pool)]
        return True

    def resolve(self, la: float, tau: float):
        v = self.pending
        ok = la < self.l_min + tau
        if ok:
            self.l_min = min(self.l_min, la)
            self.removed.add(v)
        self.pool.remove(v)
        self.pending = None
        return v, ok

    def fail(self):
        self.pool.remove(self.pending)
        self.pending = None

    def clone(self) -> "_SongBrute":
        c = _SongBrute.__new__(_SongBrute)
        c.pool, c.removed, c.l_min, c.pending = list(self.pool), set(self.removed), self.l_min, self.pending
        c.rng = SplitMix64(0)
        c.rng.s = self.rng.s
        return c

    def candidates(self):
        return (self.pending,)


def brute_force_round(con, l_min: Sequence[float], tau: float, rngs: Sequence[SplitMix64], window: int = 16) -> tuple:
    """One pruning round with brute-force sampling for every song of `con`: every processor of a song is tried
    alone, one at a time.  Pool in ascending processor order, v = pool[next() mod |pool|], a tried processor
    leaves the pool whatever the outcome.  Trials are submitted in speculative windows (_run_trials).
    Returns (keep mask [P], updated L_min per song, list of Trial)."""
    types = con.processor_types()
    _, _, song_of = con.layout()
    present = con.present()
    P = con.n_processors
    songs = [_SongBrute([i for i in range(P) if song_of[i] == s and present[i]], l_min[s], rngs[s])
             for s in range(con.n_songs)]
    trials: List[Trial] = []

    def on_trial(s, sr, la):
        v, ok = sr.resolve(la, tau)
        trials.append(Trial(s, types[v], (v,), la, ok))
        return ok
    _run_trials(con, songs, tau, window, on_trial)
    keep = present.astype(np.uint8).copy()
    for sr in songs:
        for i in sr.removed:
            keep[i] = 0
    return keep, [sr.l_min for sr in songs], trials


def uses_brute_force(iteration: int, every: int = 4) -> bool:
    """Hybrid sampling (Sec. 6.2): brute force on every 4th pruning iteration (1-based), dry/wet otherwise."""
    return iteration % every == 0


def node_deltas(con, max_masks: int = 64) -> np.ndarray:
    """Delta_i = L_a(G minus v_i) - L_a(G) for every present processor (Sec. 7.2; NaN for absent ones).
    Mask j switches off the j-th present processor of every song at once (a song's L_a depends only on its
    own processors), and up to max_masks masks go to the GPU per prune_scores call."""
    _, _, song_of = con.layout()
    present = con.present()
    P = con.n_processors
    per_song = [[i for i in range(P) if song_of[i] == s and present[i]] for s in range(con.n_songs)]
    n = max((len(v) for v in per_song), default=0)
    base = con.prune_scores(np.ones((1, P), np.uint8))[0].cpu().numpy().astype(np.float64)
    out = np.full(P, np.nan)
    for j0 in range(0, n, max_masks):
        js = range(j0, min(n, j0 + max_masks))
        masks = np.ones((len(js), P), np.uint8)
        for r, j in enumerate(js):
            for v in per_song:
                if j < len(v):
                    masks[r, v[j]] = 0
        la = con.prune_scores(masks).cpu().numpy().astype(np.float64)
        for r, j in enumerate(js):
            for s, v in enumerate(per_song):
                if j < len(v):
                    out[v[j]] = la[r, s] - base[s]
    return out


class CropFeeder:
    """Random fixed-length segments (the training regime of Sec. 5.1: every step draws a 3.8 s segment; the
    loss skips its first second through the console's warmup_samples).  Before each training step every
    song's dry tracks and target in the crop-length console `con` are replaced by a crop of the full-length
    audio, at an offset drawn with the song's splitmix64 generator: next() mod (L_full - crop + 1)."""

    def __init__(self, con, sources, targets, seed: int = 0):
        import torch
        self.con = con
        dev = con.device
        as_dev = lambda x: (x if isinstance(x, torch.Tensor) else torch.as_tensor(np.asarray(x, np.float32))).to(
            dev, torch.float32).contiguous()
        self.src = [as_dev(x) for x in sources]
        self.tgt = [as_dev(x) for x in targets]
        self.crop = [song.num_samples for song in con.songs]
        for s, (x, c) in enumerate(zip(self.src, self.crop)):
            if x.shape[1] < c or self.tgt[s].shape[1] != x.shape[1]:
                raise ValueError(f"song {s}: full-length audio shorter than the crop or target length mismatch")
        self.rngs = [SplitMix64(song_seed(seed, 1000 + s)) for s in range(len(self.src))]
        self.last: List[int] = []

    def next(self) -> List[int]:
        self.last = []
        for s, (x, t, c) in enumerate(zip(self.src, self.tgt, self.crop)):
            off = self.rngs[s].next() % (x.shape[1] - c + 1)
            self.con.update_audio(s, x[:, off:off + c], t[:, off:off + c])
            self.last.append(off)
        return self.last


@dataclasses.dataclass
class SearchResult:
    present: np.ndarray            # processors left after the last round
    l_min: List[float]             # per song
    la_final: List[float]          # per song, unmasked L_a of the pruned graph after the last fine-tuning
    pruning_ratio: List[float]     # per song: pruned processors / initial processors (Sec. 6.1)
    trials: List[List[Trial]]      # per round
    seconds: Dict[str, float]      # wall time of training, rounds and fine-tuning


def alpha_p_at(step: int, ramp_steps: int, alpha_p_max: float) -> float:
    """Sparsity weight after `step` fine-tuning steps (linear ramp, Sec. 6.3)."""
    if ramp_steps <= 0:
        return alpha_p_max
    return alpha_p_max * min(1.0, step / ramp_steps)


def search(con, n_iter: int, train_steps: int, finetune_steps: int, lr: float = 1e-2, tau: float = 0.01,
           seed: int = 0, alpha_p_max: float = 1e-4, ramp_steps: Optional[int] = None,
           method: str = "dry_wet", feeder: Optional[CropFeeder] = None, eval_con=None,
           window: int = 16) -> SearchResult:
    """Alg. 2 / Alg. 3 on every song of `con`: train, L_min from the unmasked graph, then n_iter rounds of
    {pruning round, structural prune, fine-tuning}.  method: "dry_wet" (Alg. 3), "brute_force" (every
    processor tried alone) or "hybrid" (brute force on every 4th round, dry/wet otherwise; the paper's
    default).  With a CropFeeder every training step runs on fresh random crops; trials and L_min are then
    evaluated by eval_con (the same songs at full length; parameters copied from `con` before every round,
    both consoles pruned alike), or by `con` on its current crops when eval_con is None."""
    if method not in ("dry_wet", "brute_force", "hybrid"):
        raise ValueError(method)
    ev = eval_con if eval_con is not None else con

    def train(steps, alpha):
        for _ in range(steps):
            if feeder is not None:
                feeder.next()
            if alpha is not None:
                con.set_alpha_p(alpha())
            con.train_step(lr)

    def sync_eval():
        if eval_con is not None:
            eval_con.set_params(con.get_params())
    if ramp_steps is None:
        ramp_steps = (2 * n_iter * finetune_steps) // 3
    _, _, song_of = con.layout()
    present0 = con.present().copy()
    init_count = [int(np.sum(present0[song_of == s])) for s in range(con.n_songs)]
    rngs = [SplitMix64(song_seed(seed, s)) for s in range(con.n_songs)]
    sync = lambda: con.stream.synchronize()       # the console's stream only (other consoles may be capturing)
    secs = {"train": 0.0, "rounds": 0.0, "finetune": 0.0}

    t0 = time.perf_counter()
    con.set_alpha_p(0.0)
    train(train_steps, None)
    ones = np.ones((1, con.n_processors), np.uint8)
    sync_eval()
    l_min = ev.prune_scores(ones)[0].cpu().numpy().astype(np.float64).tolist()
    sync()
    secs["train"] += time.perf_counter() - t0

    all_trials, ft = [], [0]

    def ramp():
        a = alpha_p_at(ft[0], ramp_steps, alpha_p_max)
        ft[0] += 1
        return a

    for it in range(1, n_iter + 1):
        t0 = time.perf_counter()
        sync_eval()
        brute = method == "brute_force" or (method == "hybrid" and uses_brute_force(it))
        keep, l_min, trials = (brute_force_round if brute else dry_wet_round)(ev, l_min, tau, rngs, window=window)
        con.prune(keep)
        if eval_con is not None:
            eval_con.prune(keep)
        sync()
        secs["rounds"] += time.perf_counter() - t0
        all_trials.append(trials)
        t0 = time.perf_counter()
        train(finetune_steps, ramp)
        sync()
        secs["finetune"] += time.perf_counter() - t0
    sync_eval()
    la = ev.prune_scores(ones)[0].cpu().numpy().astype(np.float64).tolist()
    present = con.present().copy()
    ratio = [1.0 - int(np.sum(present[song_of == s])) / max(1, init_count[s]) for s in range(con.n_songs)]
    return SearchResult(present, l_min, la, ratio, all_trials, secs)


def presence_scores(truth: np.ndarray, pred: np.ndarray, types: Sequence[str]) -> Dict[str, Dict[str, float]]:
    """Binary classification of processor presence (one decision per chain and type): accuracy, precision,
    recall and F1 per type and micro-averaged ("mu"); positive = present; a ratio with nothing in its
    denominator counts as 1.0."""
    truth = np.asarray(truth).astype(bool)
    pred = np.asarray(pred).astype(bool)
    ty = np.array(list(types))

    def one(sel):
        counts = {}
        for name, a, b in (("tp", True, True), ("fp", False, True), ("fn", True, False), ("tn", False, False)):
            counts[name] = int(np.count_nonzero((truth[sel] == a) & (pred[sel] == b)))
        tp, fp, fn, tn = counts["tp"], counts["fp"], counts["fn"], counts["tn"]
        ratio = lambda n, d: n / d if d > 0 else 1.0
        precision, recall = ratio(tp, tp + fp), ratio(tp, tp + fn)
        if tp + fp > 0 and tp + fn > 0:
            f1 = ratio(2.0 * precision * recall, precision + recall)
        else:
            f1 = ratio(2.0 * tp, 2.0 * tp + fp + fn)
        return {"accuracy": ratio(tp + tn, tp + tn + fp + fn), "precision": precision, "recall": recall, "f1": f1}

    out = {t: one(ty == t) for t in TYPE_ORDER if np.any(ty == t)}
    out["mu"] = one(np.ones(len(ty), bool))
    return out


def consistency_check(con, make_console, init_params, n_iter: int, train_steps: int, finetune_steps: int,
                      **search_kw) -> Dict[str, Dict[str, float]]:
    """Consistency analysis (Sec. 7.3): the pruned graph of `con` (after its search) is taken as a synthetic
    ground truth; its own mixes become the targets of a fresh console (make_console(targets) builds it over the
    same songs), the search is run again from init_params, and the two processor sets are compared per type."""
    _, mixes = con.forward_loss(with_mix=True)
    con2 = make_console([m.detach().clone() for m in mixes])
    try:
        con2.set_params(init_params)
        search(con2, n_iter, train_steps, finetune_steps, **search_kw)
        return presence_scores(con.present(), con2.present(), con.processor_types())
    finally:
        con2.close()

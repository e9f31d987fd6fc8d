"""Mixing console G_c (Sec. 1.2, Sec. 4) and its objective (Eqs. 20-23, 26), FP64 (oracle; test infrastructure).

Structure (Sec. 1.2, console type string iecnsgdrmecnsgdro of Sec. 4.2):
  * every track k: input i (the mono source on both channels) -> chain of the enabled processor types in
    the fixed order e c n s g d r;
  * every subgroup s: mix m (sum of its tracks' chain outputs, Eq. 3) -> the same chain;
  * output o: sum of the subgroup chain outputs plus the chain outputs of tracks that belong to no
    subgroup (reading: the paper's consoles route every track through a subgroup; the plain workload
    sends two tracks straight to the output).
Every processor is followed by the dry/wet blend of Eq. (2b) with w = sigmoid(q) * mask (Sec. 5.1, Alg. 3).

Canonical processor order: song -> chain (tracks, then subgroups) -> type in chain order.  The flat
parameter vector holds every processor's parameters in that order, followed by one dry/wet logit q per
processor in the same order.  Reverb noises are indexed by the rank of the reverb among all reverbs.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from . import processors as P
from .loss import LossDesc, audio_loss, gain_staging

F64 = torch.float64
TYPE_ORDER = "ecnsgdr"
PARAM_COUNT = {"e": 1024, "c": 4, "n": 4, "s": 1, "g": 2, "d": 880, "r": 768}


@dataclasses.dataclass
class SongSpec:
    num_tracks: int
    num_subgroups: int
    track_group: List[int]
    num_samples: int

    @property
    def num_chains(self):
        return self.num_tracks + self.num_subgroups


@dataclasses.dataclass
class Proc:
    song: int
    chain: int        # 0..K-1 tracks, K..K+S-1 subgroups
    type: str
    offset: int       # first parameter index
    count: int
    index: int        # processor index (dry/wet logit / mask position)
    rev: int          # rank among reverbs (-1 otherwise)


@dataclasses.dataclass
class ConsoleDesc:
    sample_rate: float = 44100.0
    types: str = TYPE_ORDER
    alpha_g: float = 1e-3
    loss: LossDesc = dataclasses.field(default_factory=LossDesc)


def layout(songs: Sequence[SongSpec], types: str = TYPE_ORDER):
    """Processors in canonical order, total processor-parameter count and number of processors."""
    chain = [t for t in TYPE_ORDER if t in types]
    procs: List[Proc] = []
    off = 0
    rev = 0
    for si, s in enumerate(songs):
        for c in range(s.num_chains):
            for t in chain:
                procs.append(Proc(si, c, t, off, PARAM_COUNT[t], len(procs), rev if t == "r" else -1))
                off += PARAM_COUNT[t]
                rev += t == "r"
    return procs, off, len(procs)


def schedule_string(types: str = TYPE_ORDER) -> str:
    """Type string of the console's node-subset sequence (Sec. 4.2): i, chain, m, chain, o."""
    chain = "".join(t for t in TYPE_ORDER if t in types)
    return "i" + chain + "m" + chain + "o"


class Console:
    """FP64 console over one or more songs (songs are independent; losses are per song)."""

    def __init__(self, songs: Sequence[SongSpec], sources: Sequence[np.ndarray], targets: Optional[Sequence[np.ndarray]],
                 reverb_noise: Optional[np.ndarray], desc: ConsoleDesc = ConsoleDesc()):
        self.songs = list(songs)
        self.desc = desc
        self.procs, self.n_proc_params, self.n_procs = layout(self.songs, desc.types)
        self.n_params = self.n_proc_params + self.n_procs
        self.sources = [torch.tensor(np.asarray(s, np.float32), dtype=F64) for s in sources]
        self.targets = [torch.tensor(np.asarray(t, np.float32), dtype=F64) for t in (targets or [])]
        n_rev = sum(p.type == "r" for p in self.procs)
        self.fir_len = int(round(2 * desc.sample_rate))
        self.noise_spec = []
        if n_rev:
            assert reverb_noise is not None and reverb_noise.shape[0] >= n_rev
            self.noise_spec = [P.reverb_noise_stft(torch.tensor(np.asarray(reverb_noise[i], np.float32), dtype=F64))
                               for i in range(n_rev)]
        self.D = P.delay_slot(desc.sample_rate)
        self.by_song_chain: Dict[tuple, List[Proc]] = {}
        for p in self.procs:
            self.by_song_chain.setdefault((p.song, p.chain), []).append(p)

    # ------------------------------------------------------------------------------------------
    def _process(self, p: Proc, u: torch.Tensor, pbar: torch.Tensor) -> torch.Tensor:
        if p.type == "g":
            return P.gain_pan(u, pbar)
        if p.type == "s":
            return P.stereo_imager(u, pbar)
        if p.type == "e":
            return P.equalizer(u, pbar)
        if p.type == "r":
            return P.reverb(u, pbar, self.noise_spec[p.rev], self.fir_len)
        if p.type == "c":
            return P.dynamics(u, pbar, gate=False)
        if p.type == "n":
            return P.dynamics(u, pbar, gate=True)
        if p.type == "d":
            return P.multitap_delay(u, pbar, self.D)
        raise ValueError(p.type)

    def _chain(self, song: int, chain: int, u: torch.Tensor, params, w, present, outs):
        """Runs one chain; outs[i] receives processor i's output and outs[("in", i)] its input."""
        lg = torch.zeros((), dtype=F64)
        for p in self.by_song_chain.get((song, chain), []):
            outs[("in", p.index)] = u
            if present is not None and not present[p.index]:
                outs[p.index] = u
                continue
            ybar = self._process(p, u, params[p.offset: p.offset + p.count])
            if p.type in "erd":
                lg = lg + gain_staging(ybar, u)
            u = P.dry_wet(u, ybar, w[p.index])
            outs[p.index] = u
        return u, lg

    def forward(self, params: torch.Tensor, mask=None, present=None, alpha_p: float = 0.0,
                keep_outputs: bool = False) -> List[Dict[str, torch.Tensor]]:
        """Render every song and evaluate Eqs. (20), (22), (26).  params: fp64 [n_params].
        mask: optional {0,1}[P] multiplied into w; present: optional {0,1}[P] structural presence
        (absent processors are bypassed and left out of L_g and L_p)."""
        q = params[self.n_proc_params:]
        w = torch.sigmoid(q)
        if mask is not None:
            w = w * torch.as_tensor(np.asarray(mask, np.float64), dtype=F64)
        res = []
        for si, s in enumerate(self.songs):
            outs: Dict[int, torch.Tensor] = {}
            lg = torch.zeros((), dtype=F64)
            track_out = []
            for k in range(s.num_tracks):
                u = torch.stack([self.sources[si][k], self.sources[si][k]])
                y, l = self._chain(si, k, u, params, w, present, outs)
                track_out.append(y)
                lg = lg + l
            mix = torch.zeros(2, s.num_samples, dtype=F64)
            for g in range(s.num_subgroups):
                u = torch.zeros(2, s.num_samples, dtype=F64)
                for k in range(s.num_tracks):
                    if s.track_group[k] == g:
                        u = u + track_out[k]
                y, l = self._chain(si, s.num_tracks + g, u, params, w, present, outs)
                lg = lg + l
                mix = mix + y
            for k in range(s.num_tracks):
                if s.track_group[k] < 0:
                    mix = mix + track_out[k]
            if self.targets:
                la = audio_loss(mix, self.targets[si], self.desc.loss)
            else:
                z = torch.zeros((), dtype=F64)
                la = {"a": z, "lr": z, "m": z, "s": z}
            lp = torch.zeros((), dtype=F64)
            for p in self.procs:
                if p.song == si and (present is None or present[p.index]):
                    lp = lp + w[p.index]
            total = la["a"] + self.desc.alpha_g * lg + alpha_p * lp
            r = {"mix": mix, "La": la["a"], "Llr": la["lr"], "Lm": la["m"], "Ls": la["s"], "Lg": lg, "Lp": lp,
                 "total": total}
            if keep_outputs:
                r["outputs"] = outs
            res.append(r)
        return res

    def loss_and_grad(self, params: np.ndarray, mask=None, present=None, alpha_p: float = 0.0):
        """Per-song losses [n_songs, 7] (La, Llr, Lm, Ls, Lg, Lp, total), d(sum_songs total)/d params, mixes."""
        x = torch.tensor(np.asarray(params, np.float64), dtype=F64, requires_grad=True)
        res = self.forward(x, mask, present, alpha_p)
        tot = sum(r["total"] for r in res)
        tot.backward()
        losses = np.array([[float(r[k].detach()) for k in ("La", "Llr", "Lm", "Ls", "Lg", "Lp", "total")] for r in res])
        return losses, x.grad.detach().numpy().copy(), [r["mix"].detach().numpy() for r in res]

    def losses(self, params: np.ndarray, mask=None, present=None, alpha_p: float = 0.0):
        with torch.no_grad():
            res = self.forward(torch.tensor(np.asarray(params, np.float64), dtype=F64), mask, present, alpha_p)
        losses = np.array([[float(r[k].detach()) for k in ("La", "Llr", "Lm", "Ls", "Lg", "Lp", "total")] for r in res])
        return losses, [r["mix"].numpy() for r in res]

    def render_targets(self, params: np.ndarray, w: np.ndarray) -> List[np.ndarray]:
        """Mix of every song with explicit dry/wet weights w [P] (ground-truth rendering), float32."""
        x = torch.tensor(np.asarray(params, np.float64), dtype=F64)
        keep_q = x.clone()
        # w enters Eq. (2b) directly: pass through a mask on sigmoid(+inf) = 1
        keep_q[self.n_proc_params:] = float("inf")
        with torch.no_grad():
            res = self.forward(keep_q, mask=np.asarray(w, np.float64))
        return [r["mix"].numpy().astype(np.float32) for r in res]

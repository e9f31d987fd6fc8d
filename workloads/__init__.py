"""Seeded synthetic inputs for the mixing-console hot path.

This module is shared by the CPU oracle tests, the GPU parity tests and the
benchmark.  It holds random draws only: console layouts (track counts,
subgroup assignment, lengths), dry source audio, reverb noise, ground-truth
processor parameters and initial parameters.  None of the mixing method's
arithmetic (processors, loss, gradients) lives here.

The paper's data (MedleyDB, MixingSecrets, an internal set; stereo 30 kHz,
17.6-28.8 tracks per song, Sec. 5.2 and Sec. 7.6) is not available, so these
generators stand in with audio of the same shape: mono tracks made of pink
noise bursts and exponentially decaying sine notes, peak normalised to -6 dBFS.
"""
from __future__ import annotations

import dataclasses
from typing import List, Sequence

import numpy as np

FS = 44100
TYPE_ORDER = "ecnsgdr"  # chain order of the seven processor types (console string iecnsgdrmecnsgdro)

# Parameter counts per processor type (Sec. 3: g 2, s 1, e 1024, r 768, c 4, n 4, d 880).
PARAM_COUNT = {"e": 1024, "c": 4, "n": 4, "s": 1, "g": 2, "d": 880, "r": 768}

PEAK = 0.501  # -6 dBFS


@dataclasses.dataclass
class SongLayout:
    """One song: K mono tracks of L samples, S subgroups; track_group[k] in [0,S) or -1 (straight to the mix)."""

    num_tracks: int
    num_subgroups: int
    track_group: List[int]
    num_samples: int

    def __post_init__(self):
        assert len(self.track_group) == self.num_tracks
        assert all(-1 <= g < self.num_subgroups for g in self.track_group)

    @property
    def num_chains(self) -> int:
        return self.num_tracks + self.num_subgroups


def _rng(*key: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(k) & 0xFFFFFFFF for k in key])))


# ---------------------------------------------------------------------------------------------
# console layouts of the five workloads
# ---------------------------------------------------------------------------------------------

def layout_plain(num_samples: int = 2 * FS) -> SongLayout:
    """4 tracks, one subgroup of tracks 0 and 1, tracks 2 and 3 straight to the mix (2 s by default)."""
    return SongLayout(4, 1, [0, 0, -1, -1], num_samples)


def layout_single_search(num_samples: int = 10 * FS) -> SongLayout:
    """16 tracks in 4 subgroups of 4 (10 s by default)."""
    return SongLayout(16, 4, [k // 4 for k in range(16)], num_samples)


def layout_uneven_batch(num_songs: int = 64, seed: int = 2, min_s: float = 5.0, max_s: float = 30.0,
                        min_k: int = 4, max_k: int = 32, max_groups: int = 8) -> List[SongLayout]:
    """Songs with K ~ U{min_k..max_k} tracks, S ~ U{1..max_groups} subgroups (S <= K), tracks assigned
    round-robin to subgroups, length ~ U[min_s, max_s] seconds."""
    rng = _rng(0x5EED, seed)
    out = []
    for _ in range(num_songs):
        k = int(rng.integers(min_k, max_k + 1))
        s = int(rng.integers(1, max_groups + 1))
        s = min(s, k)
        L = int(round(rng.uniform(min_s, max_s) * FS))
        out.append(SongLayout(k, s, [t % s for t in range(k)], L))
    return out


def layout_long(num_samples: int = 60 * FS) -> SongLayout:
    """64 tracks in 8 subgroups of 8 (60 s by default)."""
    return SongLayout(64, 8, [k // 8 for k in range(64)], num_samples)


# ---------------------------------------------------------------------------------------------
# dry sources
# ---------------------------------------------------------------------------------------------

def _pink_bursts(rng: np.random.Generator, L: int, fs: int) -> np.ndarray:
    white = rng.standard_normal(L)
    spec = np.fft.rfft(white)
    f = np.arange(spec.shape[0], dtype=np.float64)
    f[0] = 1.0
    spec = spec / np.sqrt(f)
    spec[0] = 0.0
    pink = np.fft.irfft(spec, n=L)
    pink /= max(np.std(pink), 1e-12)
    env = np.zeros(L)
    ramp = max(1, int(round(0.005 * fs)))
    t = 0
    on = bool(rng.integers(0, 2))
    while t < L:
        dur = max(1, int(round(rng.exponential(0.5) * fs)))
        if on:
            seg = np.ones(min(dur, L - t))
            r = min(ramp, seg.shape[0] // 2)
            if r > 0:
                seg[:r] = np.linspace(0.0, 1.0, r, endpoint=False)
                seg[-r:] = np.linspace(1.0, 0.0, r, endpoint=False)
            env[t:t + seg.shape[0]] = seg
        t += dur
        on = not on
    return pink * env


def _notes(rng: np.random.Generator, L: int, fs: int) -> np.ndarray:
    out = np.zeros(L)
    n = int(rng.poisson(4.0 * L / fs))
    for _ in range(n):
        t0 = int(rng.integers(0, L))
        f = float(np.exp(rng.uniform(np.log(55.0), np.log(1760.0))))
        tau = float(rng.uniform(0.1, 1.0))
        amp = float(rng.uniform(0.3, 1.0))
        phase = float(rng.uniform(0.0, 2.0 * np.pi))
        m = min(L - t0, int(5.0 * tau * fs))
        tt = np.arange(m) / fs
        out[t0:t0 + m] += amp * np.sin(2.0 * np.pi * f * tt + phase) * np.exp(-tt / tau)
    return out


def source_track(key: Sequence[int], L: int, fs: int = FS) -> np.ndarray:
    """One mono dry track (float32 [L]), peak -6 dBFS, seeded by `key`."""
    rng = _rng(0x50C, *key)
    x = _pink_bursts(rng, L, fs) * rng.uniform(0.2, 1.0) + _notes(rng, L, fs) * rng.uniform(0.2, 1.0)
    pk = np.max(np.abs(x))
    if pk > 0:
        x = x * (PEAK / pk)
    return x.astype(np.float32)


def song_sources(layout: SongLayout, key: Sequence[int], fs: int = FS) -> np.ndarray:
    """All K mono tracks of one song, float32 [K][L]."""
    return np.stack([source_track(tuple(key) + (k,), layout.num_samples, fs) for k in range(layout.num_tracks)])


def reverb_noise(key: Sequence[int], n_nodes: int, fs: int = FS) -> np.ndarray:
    """Fixed uniform noise of the reverbs (Sec. 3.4): float32 [n_nodes][2 (mid, side)][2*fs], U(-1, 1)."""
    rng = _rng(0xAEB, *key)
    return rng.uniform(-1.0, 1.0, size=(n_nodes, 2, 2 * fs)).astype(np.float32)


# ---------------------------------------------------------------------------------------------
# parameters
# ---------------------------------------------------------------------------------------------

def chain_types(type_mask: str = TYPE_ORDER) -> str:
    """Enabled processor types of every chain, in chain order."""
    return "".join(t for t in TYPE_ORDER if t in type_mask)


def processor_types(layouts: Sequence[SongLayout], type_mask: str = TYPE_ORDER) -> List[str]:
    """Processor types in canonical order: song -> chain (tracks, then subgroups) -> type in chain order."""
    ct = chain_types(type_mask)
    out: List[str] = []
    for lay in layouts:
        for _ in range(lay.num_chains):
            out.extend(ct)
    return out


def init_params(types: Sequence[str], key: Sequence[int]) -> np.ndarray:
    """Initial parameters ~ N(0, 0.1^2) (Sec. 5.1): processor parameters in canonical order, then one
    dry/wet logit per processor.  float32."""
    rng = _rng(0x1417, *key)
    n = sum(PARAM_COUNT[t] for t in types) + len(types)
    return (0.1 * rng.standard_normal(n)).astype(np.float32)


def _gt_proc(rng: np.random.Generator, t: str) -> np.ndarray:
    if t == "g":
        return rng.uniform(-1.0, 1.0, 2)
    if t == "s":
        return rng.uniform(-1.0, 0.5, 1)
    if t == "e":
        knots = rng.uniform(-1.0, 1.0, 8)
        return np.interp(np.arange(1024), np.linspace(0, 1023, 8), knots)
    if t == "r":
        out = np.empty((2, 2, 192))
        out[:, 0] = rng.uniform(-6.0, -3.0, (2, 192))
        out[:, 1] = rng.uniform(-1.0, 1.0, (2, 192))
        return out.reshape(-1)
    if t in "cn":
        lo_t, hi_t = (-8.0, -2.0) if t == "c" else (-14.0, -8.0)
        return np.array([rng.uniform(4.0, 9.0), rng.uniform(lo_t, hi_t), rng.uniform(-1.0, 1.0), rng.uniform(0.0, 2.0)])
    if t == "d":
        out = np.empty((2, 20, 22))
        rad = rng.uniform(0.9, 1.0, (2, 20))
        ang = rng.uniform(-np.pi, np.pi, (2, 20))
        out[:, :, 0] = rad * np.cos(ang)
        out[:, :, 1] = rad * np.sin(ang)
        out[:, :, 2:] = rng.uniform(-5.0, -3.0, (2, 20, 20))
        return out.reshape(-1)
    raise ValueError(t)


def ground_truth(types: Sequence[str], key: Sequence[int]):
    """Seeded ground-truth graph: keep round(P/3) processors (seeded permutation) with parameters uniform
    in their ranges.  Returns (params float32 [n_params] with the dry/wet logits zero, keep uint8 [P]).
    The target is rendered with dry/wet weights w = keep (1 kept, 0 removed)."""
    rng = _rng(0x67, *key)
    P = len(types)
    keep = np.zeros(P, np.uint8)
    keep[rng.permutation(P)[: int(round(P / 3))]] = 1
    chunks = [_gt_proc(rng, t) for t in types]
    params = np.concatenate(chunks + [np.zeros(P)]).astype(np.float32)
    return params, keep

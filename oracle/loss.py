"""Sec. 5.1 audio loss (Eqs. 20-21) and gain-staging regulariser (Eq. 22), FP64 (oracle; test infrastructure).

Readings where the paper is silent (repeated in the design notes):
  * STFT: periodic Hann window, hop n_fft / hop_div, no centre padding; frames that start before
    `warmup` samples are dropped (the paper drops the first second, Sec. 5.1).
  * A-weighting (Sec. 5.1): the analytic IEC 61672 A-curve magnitude, normalised to 0 dB at 1 kHz,
    multiplies every STFT bin (instead of a time-domain pre-filter).
  * magnitude sqrt(re^2 + im^2 + 1e-8) of the weighted spectrum; Mel: `n_mels` HTK-formula triangles
    over 0..fs/2, unnormalised (n_mels = 0 keeps the linear bins).
  * Eq. (21) "/N": the L1 log term is the element-wise mean over frames x bands x channels of the
    channel set; the log uses ln(Y + 1e-5); the Frobenius norms run over the same elements.
  * channel sets: lr = {left, right}, m = {left + right}, s = {left - right}.
  * Eq. (22): log of the l2 norm taken as 0.5 ln(sum x^2 + 1e-12).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, Sequence

import numpy as np
import torch

from .processors import stft

F64 = torch.float64
LOG_EPS = 1e-5
MAG_EPS = 1e-8
NORM_EPS = 1e-12


@dataclasses.dataclass
class LossDesc:
    sample_rate: float = 44100.0
    n_fft: Sequence[int] = (512, 2048, 8192)
    hop_div: int = 4
    n_mels: int = 96
    a_weighting: bool = True
    warmup_samples: int = 0
    alpha_lr: float = 0.5
    alpha_m: float = 0.25
    alpha_s: float = 0.25


def a_weight_gain(freqs: np.ndarray) -> np.ndarray:
    """IEC 61672 A-weighting magnitude R_A(f) / R_A(1000 Hz)."""
    def ra(f):
        f2 = np.asarray(f, np.float64) ** 2
        return (12194.0 ** 2 * f2 * f2) / ((f2 + 20.6 ** 2) * np.sqrt((f2 + 107.7 ** 2) * (f2 + 737.9 ** 2)) * (f2 + 12194.0 ** 2))
    return ra(freqs) / ra(1000.0)


def hz_to_mel(f):
    return 2595.0 * np.log10(1.0 + np.asarray(f, np.float64) / 700.0)


def mel_to_hz(m):
    return 700.0 * (10.0 ** (np.asarray(m, np.float64) / 2595.0) - 1.0)


def mel_filterbank(n_fft: int, n_mels: int, fs: float) -> np.ndarray:
    """HTK-formula triangular filters, unnormalised: [n_mels, n_fft/2 + 1]."""
    fk = np.arange(n_fft // 2 + 1) * fs / n_fft
    edges = mel_to_hz(np.linspace(0.0, hz_to_mel(fs / 2.0), n_mels + 2))
    W = np.zeros((n_mels, fk.shape[0]))
    for b in range(n_mels):
        lo, ce, hi = edges[b], edges[b + 1], edges[b + 2]
        W[b] = np.maximum(0.0, np.minimum((fk - lo) / (ce - lo), (hi - fk) / (hi - ce)))
    return W


def spectrogram(x: torch.Tensor, n_fft: int, desc: LossDesc) -> torch.Tensor:
    """Weighted (Mel) magnitude spectrogram of one channel x [L] -> [frames, bands]."""
    hop = n_fft // desc.hop_div
    first = -(-desc.warmup_samples // hop)
    X = stft(x, n_fft, hop, first)
    fk = np.arange(n_fft // 2 + 1) * desc.sample_rate / n_fft
    A = torch.tensor(a_weight_gain(fk) if desc.a_weighting else np.ones_like(fk), dtype=F64)
    mag = torch.sqrt(A ** 2 * (X.real ** 2 + X.imag ** 2) + MAG_EPS)
    if desc.n_mels > 0:
        W = torch.tensor(mel_filterbank(n_fft, desc.n_mels, desc.sample_rate), dtype=F64)
        return mag @ W.T
    return mag


def channel_sets(x: torch.Tensor) -> Dict[str, torch.Tensor]:
    """Stereo [2, L] -> {'lr': [2, L], 'm': [1, L], 's': [1, L]}."""
    return {"lr": x, "m": (x[0] + x[1])[None], "s": (x[0] - x[1])[None]}


def mrstft_set(yhat: torch.Tensor, y: torch.Tensor, desc: LossDesc) -> torch.Tensor:
    """Eq. (21) for one channel set (yhat, y: [C, L]): sum over resolutions of the mean absolute
    log-spectral distance plus the spectral convergence ||Y - Yhat||_F / ||Y||_F."""
    total = torch.zeros((), dtype=F64)
    for n_fft in desc.n_fft:
        Y = torch.stack([spectrogram(y[c], n_fft, desc) for c in range(y.shape[0])])
        Yh = torch.stack([spectrogram(yhat[c], n_fft, desc) for c in range(yhat.shape[0])])
        if Y.numel() == 0:
            continue
        logd = torch.mean(torch.abs(torch.log(Y + LOG_EPS) - torch.log(Yh + LOG_EPS)))
        sc = torch.linalg.norm((Y - Yh).reshape(-1)) / torch.linalg.norm(Y.reshape(-1))
        total = total + logd + sc
    return total


def audio_loss(yhat: torch.Tensor, y: torch.Tensor, desc: LossDesc) -> Dict[str, torch.Tensor]:
    """Eq. (20): L_a = a_lr L_lr + a_m L_m + a_s L_s.  yhat (prediction), y (target): [2, L]."""
    sh, st = channel_sets(yhat), channel_sets(y.to(F64))
    parts = {k: mrstft_set(sh[k], st[k], desc) for k in ("lr", "m", "s")}
    parts["a"] = combine(parts["lr"], parts["m"], parts["s"], desc)
    return parts


def combine(l_lr, l_m, l_s, desc: LossDesc):
    """Eq. (20) weighted sum."""
    return desc.alpha_lr * l_lr + desc.alpha_m * l_m + desc.alpha_s * l_s


def log_l2(x: torch.Tensor) -> torch.Tensor:
    return 0.5 * torch.log(torch.sum(x * x) + NORM_EPS)


def gain_staging(ybar: torch.Tensor, u: torch.Tensor) -> torch.Tensor:
    """One term of Eq. (22): | log ||(y_bar)_mid||_2 - log ||(u)_mid||_2 |, mid = left + right."""
    return torch.abs(log_l2(ybar[0] + ybar[1]) - log_l2(u[0] + u[1]))

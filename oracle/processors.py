"""Sec. 3 differentiable processors, FP64, plain PyTorch CPU ops (oracle; test infrastructure only).

Every function takes a stereo input u of shape [2, L] (row 0 left, row 1 right) and a parameter
vector p_bar, and returns the wet output y_bar = f(u, p_bar) of Eq. (2a).  The dry/wet blend of
Eq. (2b) is `dry_wet`.  Convolutions use the FFT as a library primitive (exact linear convolution
up to rounding); `direct_conv` is the brute-force definition used by the pins.

Readings where the paper is silent or garbled (each is repeated in the design notes):
  * zero-phase FIR (Eq. 7): taps n in [-(N-1)/2, (N-1)/2] (the printed range is off by one) and the
    symmetric Hann window v[n] = (1 + cos(2 pi n / (N-1))) / 2 with v[0] = 1.
  * reverb (Sec. 3.4): STFT with a periodic Hann window, no centre padding; 193 bins of the 384-point
    FFT, the last (Nyquist) bin reusing parameter 191; H_delta = -0.05 softplus(p_delta); inverse STFT by
    overlap-add normalised by the summed squared window (0 where no frame covers a sample); stereo FIR
    h_l = h_m + h_s, h_r = h_m - h_s; causal convolution truncated to the input length.
  * compressor / noisegate (Sec. 3.5-3.6): alpha = sigmoid(p0), T = p1, W = exp(p2), R = 1 + exp(p3);
    the envelope is the exact one-pole recursion of Eq. (11) (the paper's truncation length of Eq. 12 is
    not given); G_u = ln(g + 1e-8).
  * multitap delay (Sec. 3.7): slot length D = round(0.1 fs); d_m = (m-1) D + (round(D ((-arg z_m) mod 2pi)
    / 2pi) mod D), decided in double precision; c_m is the Eq. (7) FIR with N = 39 centred on d_m.  The
    surrogate of Eq. (18) uses N = D and z clamped to the unit disk; its gradient uses the real part of
    the surrogate and the PyTorch complex-gradient convention; sgn(z*) of Eq. (19) is read as the radial
    direction z/|z|.
"""
from __future__ import annotations

import math

import numpy as np
import torch

F64 = torch.float64

EQ_TAPS = 2047        # Sec. 3.3: N = 2047, 1024 parameters
DELAY_FIR_TAPS = 39   # Sec. 3.7: 39-tap c_m, 20 log-magnitudes
DELAY_TAPS = 20       # Sec. 3.7: M = 20 delays per channel
REVERB_NFFT = 384     # Sec. 3.4: FFT 384, hop 192
REVERB_HOP = 192
REVERB_BINS = 192     # parameters per log-magnitude vector
ENV_EPS = 1e-8        # G_u = ln(g + eps)
DELAY_GAMMA = 0.01    # Sec. 3.7: regulariser strength


# ------------------------------------------------------------------------------------------------
# convolution helpers
# ------------------------------------------------------------------------------------------------

def _next_pow2(n: int) -> int:
    return 1 << max(0, (n - 1).bit_length())


def fft_conv(x: torch.Tensor, taps: torch.Tensor, n0: int) -> torch.Tensor:
    """y[n] = sum_j taps[..., j] x[..., n - (n0 + j)] for n in [0, L): linear convolution of x (zero outside
    [0, L)) with an FIR whose first tap sits at time n0, truncated to the input length."""
    L = x.shape[-1]
    nh = taps.shape[-1]
    nfft = _next_pow2(L + nh - 1)
    c = torch.fft.irfft(torch.fft.rfft(x, nfft) * torch.fft.rfft(taps, nfft), nfft)[..., : L + nh - 1]
    if n0 <= 0:
        return c[..., -n0: -n0 + L]
    pad = torch.zeros(c.shape[:-1] + (n0,), dtype=c.dtype)
    return torch.cat([pad, c[..., : L - n0]], -1)


def direct_conv(x: np.ndarray, taps: np.ndarray, n0: int) -> np.ndarray:
    """Brute-force definition of `fft_conv` (numpy, one output at a time); for pins on small inputs."""
    L = x.shape[-1]
    y = np.zeros(L)
    for n in range(L):
        acc = 0.0
        for j in range(taps.shape[-1]):
            m = n - (n0 + j)
            if 0 <= m < L:
                acc += taps[j] * x[m]
        y[n] = acc
    return y


# ------------------------------------------------------------------------------------------------
# Eq. (2b) dry/wet, Eq. (4) gain/panning, Eqs. (5)-(6) stereo imager
# ------------------------------------------------------------------------------------------------

def dry_wet(u: torch.Tensor, ybar: torch.Tensor, w: torch.Tensor) -> torch.Tensor:
    """Eq. (2b): y = w y_bar + (1 - w) u."""
    return w * ybar + (1.0 - w) * u


def gain_pan(u: torch.Tensor, p: torch.Tensor) -> torch.Tensor:
    """Eq. (4): y_bar[c] = exp(p[c]) u[c]; p holds the two per-channel log gains."""
    return torch.exp(p)[:, None] * u


def stereo_imager(u: torch.Tensor, p: torch.Tensor) -> torch.Tensor:
    """Eqs. (5)-(6): mid = l + r, side = exp(p) (l - r); back to l/r with the halves."""
    mid = u[0] + u[1]
    side = torch.exp(p[0]) * (u[0] - u[1])
    return torch.stack([(mid + side) / 2.0, (mid - side) / 2.0])


# ------------------------------------------------------------------------------------------------
# Eqs. (7)-(8) zero-phase FIR equalizer
# ------------------------------------------------------------------------------------------------

def hann_symmetric(N: int) -> torch.Tensor:
    """v[n] = (1 + cos(2 pi n / (N-1))) / 2 for n in [-(N-1)/2, (N-1)/2] (v[0] = 1, zero at both ends)."""
    half = (N - 1) // 2
    n = torch.arange(-half, half + 1, dtype=F64)
    return 0.5 * (1.0 + torch.cos(2.0 * math.pi * n / (N - 1)))


def zero_phase_fir(logmag: torch.Tensor, N: int) -> torch.Tensor:
    """Eq. (7): h[n] = v[n] (1/N) sum_k exp(P[k]) w_N^{kn}, w_N = exp(+j 2 pi / N), for n in
    [-(N-1)/2, (N-1)/2].  The log-magnitudes give P[k] for k = 0..(N-1)/2 and the mirror P[N-k] = P[k]
    makes the response real and even.  Returns taps [..., N]; tap 0 sits at n = -(N-1)/2."""
    half = (N - 1) // 2
    assert logmag.shape[-1] == half + 1
    P = torch.cat([logmag, logmag[..., 1:].flip(-1)], -1)
    h_circ = torch.fft.ifft(torch.exp(P).to(torch.complex128), dim=-1).real   # (1/N) sum_k e^{P_k} w^{kn}
    h = torch.roll(h_circ, half, dims=-1)                                       # index j <-> n = j - half
    return hann_symmetric(N) * h


def equalizer(u: torch.Tensor, p: torch.Tensor) -> torch.Tensor:
    """Eq. (8): the same zero-phase FIR of Eq. (7) (N = 2047) on both channels."""
    h = zero_phase_fir(p, EQ_TAPS)
    return fft_conv(u, h, -(EQ_TAPS - 1) // 2)


# ------------------------------------------------------------------------------------------------
# Sec. 3.4 reverb, Eqs. (9)-(10)
# ------------------------------------------------------------------------------------------------

def hann_periodic(n: int) -> torch.Tensor:
    j = torch.arange(n, dtype=F64)
    return 0.5 * (1.0 - torch.cos(2.0 * math.pi * j / n))


def stft(x: torch.Tensor, n_fft: int, hop: int, first_frame: int = 0) -> torch.Tensor:
    """Frames t = first_frame.. with t hop + n_fft <= len(x), periodic Hann window, no centre padding;
    returns the one-sided spectrum [..., frames, n_fft/2 + 1]."""
    fr = x.unfold(-1, n_fft, hop)[..., first_frame:, :]
    return torch.fft.rfft(fr * hann_periodic(n_fft), dim=-1)


def istft_ola(spec: torch.Tensor, n_fft: int, hop: int, length: int) -> torch.Tensor:
    """Inverse of `stft`: inverse FFT of every frame, window, overlap-add, divide by the summed squared
    window where it is above 1e-11 (zero elsewhere).  spec [F, n_fft/2 + 1] -> [length]."""
    win = hann_periodic(n_fft)
    frames = torch.fft.irfft(spec, n_fft, dim=-1) * win
    out = torch.zeros(length, dtype=F64)
    env = torch.zeros(length, dtype=F64)
    for t in range(spec.shape[0]):
        s = t * hop
        out = out.index_add(0, torch.arange(s, s + n_fft), frames[t])
        env[s: s + n_fft] += win * win
    safe = env > 1e-11
    return torch.where(safe, out / torch.where(safe, env, torch.ones_like(env)), torch.zeros_like(out))


def reverb_noise_stft(noise: torch.Tensor) -> torch.Tensor:
    """STFT U_x[k, m] of the fixed mid and side noises (noise [2, 2 fs]) -> [2, F, 193]."""
    return stft(noise.to(F64), REVERB_NFFT, REVERB_HOP)


def reverb_fir(p: torch.Tensor, noise_spec: torch.Tensor, fir_len: int) -> torch.Tensor:
    """Eqs. (9)-(10): H_x = U_x * M_x with M_x[k, m] = exp(H0_x[k] + (m-1) H_delta_x[k]) for frames
    m = 1..F, inverse STFT to the time-domain responses h_m, h_s and the stereo FIR
    (h_m + h_s, h_m - h_s).  p = [x in (mid, side)][(H0, p_delta)][192].  Returns [2, fir_len]."""
    pp = p.reshape(2, 2, REVERB_BINS)
    F = noise_spec.shape[1]
    m1 = torch.arange(F, dtype=F64)[:, None]        # m - 1
    hs = []
    for x in range(2):
        h0 = torch.cat([pp[x, 0], pp[x, 0, -1:]])              # 193 bins, Nyquist reuses bin 191
        hd = -0.05 * torch.nn.functional.softplus(torch.cat([pp[x, 1], pp[x, 1, -1:]]))
        mask = torch.exp(h0[None, :] + m1 * hd[None, :])
        hs.append(istft_ola(noise_spec[x] * mask, REVERB_NFFT, REVERB_HOP, fir_len))
    return torch.stack([hs[0] + hs[1], hs[0] - hs[1]])


def reverb(u: torch.Tensor, p: torch.Tensor, noise_spec: torch.Tensor, fir_len: int) -> torch.Tensor:
    """Channel-wise causal convolution of u with the stereo reverb FIR (Sec. 3.4)."""
    h = reverb_fir(p, noise_spec, fir_len)
    return fft_conv(u, h, 0)


# ------------------------------------------------------------------------------------------------
# Sec. 3.5-3.6 compressor and noisegate, Eqs. (11)-(16)
# ------------------------------------------------------------------------------------------------

def envelope(x: torch.Tensor, alpha: torch.Tensor) -> torch.Tensor:
    """Eq. (11) with a single alpha: g[n] = alpha g[n-1] + (1 - alpha) x[n], g[-1] = 0.  Computed exactly as
    the causal convolution of x with the untruncated impulse response (1 - alpha) alpha^n of Eq. (12)."""
    L = x.shape[-1]
    n = torch.arange(L, dtype=F64)
    h = (1.0 - alpha) * torch.exp(n * torch.log(alpha))
    return fft_conv(x, h, 0)


def envelope_loop(x: np.ndarray, alpha: float) -> np.ndarray:
    """Eq. (11) by the plain recursion (pins only)."""
    g = np.zeros_like(x, dtype=np.float64)
    prev = 0.0
    for i in range(x.shape[0]):
        prev = alpha * prev + (1.0 - alpha) * x[i]
        g[i] = prev
    return g


def dyn_params(p: torch.Tensor):
    """alpha = sigmoid(p0), T = p1, W = exp(p2), R = 1 + exp(p3)."""
    return torch.sigmoid(p[0]), p[1], torch.exp(p[2]), 1.0 + torch.exp(p[3])


def compressor_gain_law(Gu, T, W, R):
    """Eqs. (13)-(14): quadratic-knee compressor gain computer."""
    above = T + (Gu - T) / R
    mid = Gu + (1.0 / R - 1.0) * (Gu - T + W) ** 2 / (4.0 * W)
    return torch.where(Gu >= T + W, above, torch.where(Gu >= T - W, mid, Gu))


def noisegate_gain_law(Gu, T, W, R):
    """Eq. (16) with the above-threshold branch G_u (Sec. 3.6)."""
    mid = Gu + (1.0 - R) * (Gu - T - W) ** 2 / (4.0 * W)
    below = T + R * (Gu - T)
    return torch.where(Gu >= T + W, Gu, torch.where(Gu >= T - W, mid, below))


def dynamics(u: torch.Tensor, p: torch.Tensor, gate: bool) -> torch.Tensor:
    """Sec. 3.5 (compressor) / Sec. 3.6 (noisegate): mid energy -> Eq. (11) envelope -> log ->
    gain law -> Eq. (15) y_bar_x = exp(G_y - G_u) u_x."""
    alpha, T, W, R = dyn_params(p)
    x = (u[0] + u[1]) ** 2
    g = envelope(x, alpha)
    Gu = torch.log(g + ENV_EPS)
    Gy = noisegate_gain_law(Gu, T, W, R) if gate else compressor_gain_law(Gu, T, W, R)
    return torch.exp(Gy - Gu)[None, :] * u


# ------------------------------------------------------------------------------------------------
# Sec. 3.7 multitap delay, Eqs. (17)-(19)
# ------------------------------------------------------------------------------------------------

def delay_slot(fs: float) -> int:
    return int(round(0.1 * fs))


def delay_positions(zr: np.ndarray, zi: np.ndarray, D: int) -> np.ndarray:
    """Integer delays d_m (0-based m: d_m = m D + offset) from the angular frequencies, in double precision:
    z = exp(-j 2 pi d / D) yields the impulse delta[n - d] through Eq. (18) with w_D = exp(+j 2 pi / D)."""
    ang = np.arctan2(np.asarray(zi, np.float64), np.asarray(zr, np.float64))
    ph = np.mod(-ang, 2.0 * np.pi)
    off = np.mod(np.rint(D * ph / (2.0 * np.pi)).astype(np.int64), D)
    m = np.arange(zr.shape[-1])
    return m * D + off


def surrogate_impulse(z: complex, D: int) -> np.ndarray:
    """Eq. (18) with N = D: s[n] = (1/D) sum_k z^k w_D^{kn}, n in [0, D) (complex)."""
    k = np.arange(D)
    return np.fft.ifft(np.power(complex(z), k))


def surrogate_impulse_dz(z: complex, D: int) -> np.ndarray:
    """d s[n] / d z = (1/D) sum_k k z^(k-1) w_D^{kn} (s is holomorphic in z)."""
    k = np.arange(D)
    a = np.zeros(D, np.complex128)
    a[1:] = k[1:] * np.power(complex(z), k[1:] - 1)
    return np.fft.ifft(a)


class DelayScatter(torch.autograd.Function):
    """h_d[n] = sum_m c_m[n - d_m] (Eq. 17) with the exact integer delays in the forward pass and the
    Eq. (19) straight-through gradient for z_m in the backward pass:
        g_m   = sum_n dL/dh_tilde_m[n] * conj(d h_tilde_m[n] / dz)      (h_tilde = Re of Eq. 18, z clamped
                                                                       to the unit disk)
        dz_m  = sgn(g_m) + gamma (|z_m| - 1) z_m / |z_m|,  sgn(0) = 0
    where dL/dh_tilde_m[n] = sum_j dL/dh_d[d_base_m + n + j] c_m[j] (slot m, n in [0, D)).
    Inputs: c [2, 20, 39] (tap 0 at -19), zr, zi [2, 20].  Output taps [2, 20 D + 38], tap 0 at n = -19."""

    @staticmethod
    def forward(ctx, c, zr, zi, D: int, L: int):
        d = delay_positions(zr.detach().numpy(), zi.detach().numpy(), D)   # [2, 20]
        ntaps = DELAY_TAPS * D + DELAY_FIR_TAPS - 1
        out = torch.zeros(2, ntaps, dtype=F64)
        for ch in range(2):
            for m in range(DELAY_TAPS):
                s = int(d[ch, m])
                out[ch, s: s + DELAY_FIR_TAPS] += c[ch, m]
        ctx.save_for_backward(c, zr, zi)
        ctx.d = d
        ctx.D = D
        ctx.L = L
        return out

    @staticmethod
    def backward(ctx, dtaps):
        c, zr, zi = ctx.saved_tensors
        d, D = ctx.d, ctx.D
        dc = torch.zeros_like(c)
        dzr = torch.zeros_like(zr)
        dzi = torch.zeros_like(zi)
        dt = dtaps.detach().numpy().copy()
        # dL/dh[t] = sum_n dL/dy[n] u[n - t] vanishes identically for lags t >= L (no overlap); drop the
        # rounding residue there so that sgn(0) = 0 holds for slots beyond the signal
        dt[:, ctx.L + DELAY_FIR_TAPS // 2:] = 0.0
        cc = c.detach().numpy()
        for ch in range(2):
            for m in range(DELAY_TAPS):
                s = int(d[ch, m])
                dc[ch, m] = dtaps[ch, s: s + DELAY_FIR_TAPS]
                seg = dt[ch, m * D: m * D + D + DELAY_FIR_TAPS - 1]
                G = np.lib.stride_tricks.sliding_window_view(seg, DELAY_FIR_TAPS) @ cc[ch, m]   # [D]
                z = complex(float(zr[ch, m]), float(zi[ch, m]))
                r = abs(z)
                zc = z / max(1.0, r)
                g = np.sum(G * np.conj(surrogate_impulse_dz(zc, D)))
                sg = g / abs(g) if abs(g) > 0 else 0.0
                radial = DELAY_GAMMA * (r - 1.0) * (z / r) if r > 0 else 0.0
                tot = sg + radial
                dzr[ch, m] = tot.real
                dzi[ch, m] = tot.imag
        return dc, dzr, dzi, None, None


def delay_fir(p: torch.Tensor, D: int, L: int) -> torch.Tensor:
    """Eq. (17) FIR of both channels from p = [ch][m][(Re z, Im z, 20 log-magnitudes)], for an input of
    L samples."""
    pp = p.reshape(2, DELAY_TAPS, 22)
    c = zero_phase_fir(pp[:, :, 2:], DELAY_FIR_TAPS)     # [2, 20, 39]
    return DelayScatter.apply(c, pp[:, :, 0], pp[:, :, 1], D, L)


def multitap_delay(u: torch.Tensor, p: torch.Tensor, D: int) -> torch.Tensor:
    """Sec. 3.7: channel-wise convolution with the per-channel multitap FIRs (first tap at n = -19)."""
    h = delay_fir(p, D, u.shape[-1])
    return fft_conv(u, h, -(DELAY_FIR_TAPS - 1) // 2)

"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: values the paper prints, closed forms,
special cases that reduce to a textbook or library routine, invariants, or brute force on tiny inputs.
"""
import math
import os

import numpy as np
import pytest
import torch

from oracle import processors as P
from oracle import loss as Lo
from oracle import console as C
from oracle import adam as A

GOLD = os.path.join(os.path.dirname(__file__), "golden")
F64 = torch.float64


def t64(x):
    return torch.tensor(np.asarray(x, np.float64), dtype=F64)


def rng(seed=0):
    return np.random.default_rng(seed)


# ------------------------------------------------------------------------------------------------
# Eq. (2b), Eq. (4), Eqs. (5)-(6)
# ------------------------------------------------------------------------------------------------

def test_dry_wet_bypass_and_full_wet():
    u = t64(rng().standard_normal((2, 100)))
    yb = t64(rng(1).standard_normal((2, 100)))
    assert torch.equal(P.dry_wet(u, yb, torch.tensor(0.0, dtype=F64)), u)   # w = 0 is an exact bypass
    assert torch.allclose(P.dry_wet(u, yb, torch.tensor(1.0, dtype=F64)), yb, rtol=0, atol=0)


def test_gain_pan_special_values():
    u = t64(rng().standard_normal((2, 50)))
    y = P.gain_pan(u, t64([math.log(2.0), 0.0]))
    assert torch.allclose(y[0], 2.0 * u[0], rtol=1e-15, atol=0) and torch.allclose(y[1], u[1], rtol=0, atol=0)
    y = P.gain_pan(u, t64([0.0, math.log(0.25)]))
    assert torch.allclose(y[1], 0.25 * u[1], rtol=1e-15, atol=0) and torch.allclose(y[0], u[0])


def test_stereo_imager_identity_mono_and_midside():
    u = t64(rng().standard_normal((2, 64)))
    assert torch.allclose(P.stereo_imager(u, t64([0.0])), u, rtol=0, atol=1e-15)   # identity at p = 0
    mono = P.stereo_imager(u, t64([-60.0]))                                        # side removed -> mono
    assert torch.allclose(mono[0], (u[0] + u[1]) / 2, atol=1e-12) and torch.allclose(mono[1], mono[0], atol=1e-12)
    y = P.stereo_imager(u, t64([0.7]))
    assert torch.allclose(y[0] + y[1], u[0] + u[1], atol=1e-12)                     # mid preserved
    assert torch.allclose(y[0] - y[1], math.exp(0.7) * (u[0] - u[1]), atol=1e-12)   # side scaled


# ------------------------------------------------------------------------------------------------
# Eqs. (7)-(8) zero-phase FIR and convolution
# ------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("N", [7, 39, 2047])
def test_zero_phase_fir_flat_is_unit_impulse(N):
    h = P.zero_phase_fir(torch.zeros((N + 1) // 2, dtype=F64), N).numpy()
    ref = np.zeros(N)
    ref[(N - 1) // 2] = 1.0
    assert np.allclose(h, ref, atol=1e-14)


@pytest.mark.parametrize("N", [7, 39])
def test_zero_phase_fir_brute_force_and_sampled_response(N):
    half = (N - 1) // 2
    lm = rng(3).uniform(-2, 2, half + 1)
    h = P.zero_phase_fir(t64(lm), N).numpy()
    # brute force of Eq. (7) with complex arithmetic, w_N = exp(+j 2 pi / N)
    Pk = np.concatenate([lm, lm[1:][::-1]])
    for j, n in enumerate(range(-half, half + 1)):
        v = 0.5 * (1 + math.cos(2 * math.pi * n / (N - 1)))
        s = sum(math.e ** Pk[k] * complex(math.cos(2 * math.pi * k * n / N), math.sin(2 * math.pi * k * n / N)) for k in range(N))
        assert abs(h[j] - v * s.real / N) < 1e-12 and abs(s.imag) < 1e-9
    assert np.allclose(h, h[::-1], atol=1e-14)     # even, hence zero phase
    assert h[0] == 0.0 and h[-1] == 0.0           # the symmetric Hann window vanishes at both ends


@pytest.mark.parametrize("n0", [-5, 0, 3])
def test_fft_conv_matches_direct(n0):
    r = rng(4)
    x = r.standard_normal(37)
    taps = r.standard_normal(11)
    y = P.fft_conv(t64(x), t64(taps), n0).numpy()
    assert np.allclose(y, P.direct_conv(x, taps, n0), atol=1e-12)


def test_equalizer_flat_is_identity():
    u = t64(rng(5).standard_normal((2, 3000)))
    y = P.equalizer(u, torch.zeros(1024, dtype=F64))
    assert torch.allclose(y, u, atol=1e-12)


# ------------------------------------------------------------------------------------------------
# Sec. 3.5-3.6 envelope and gain laws
# ------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("alpha", [0.3, 0.99, 0.9999])
def test_envelope_matches_recursion(alpha):
    x = rng(6).uniform(0, 1, 2000) ** 3
    g = P.envelope(t64(x), torch.tensor(alpha, dtype=F64)).numpy()
    assert np.allclose(g, P.envelope_loop(x, alpha), rtol=1e-9, atol=1e-14)


def test_envelope_alpha_zero_is_energy():
    x = rng(7).uniform(0, 1, 500)
    g = P.envelope(t64(x), torch.tensor(1e-300, dtype=F64)).numpy()
    assert np.allclose(g, x, rtol=1e-12)


def test_compressor_below_threshold_is_unity_gain():
    u = t64(0.3 * rng(8).standard_normal((2, 4000)))
    p = t64([0.0, 10.0, 0.0, 1.0])    # T = 10 (energy e^10) is never reached
    assert torch.allclose(P.dynamics(u, p, gate=False), u, rtol=1e-14, atol=0)


def test_noisegate_above_threshold_is_unity_gain():
    u = t64(0.3 * rng(9).standard_normal((2, 4000)) + 0.5)
    p = t64([0.0, -40.0, 0.0, 1.0])   # every level is above T + W
    assert torch.allclose(P.dynamics(u, p, gate=True), u, rtol=1e-14, atol=0)


def test_compressor_ratio_one_is_identity_law():
    G = t64(np.linspace(-10, 5, 301))
    assert torch.allclose(P.compressor_gain_law(G, -2.0, 1.0, 1.0), G, atol=1e-14)


def test_gain_law_static_points():
    # textbook static curves (Giannoulis et al.): above the knee the compressor maps G -> T + (G - T)/R,
    # the gate below the knee maps G -> T + R (G - T).
    assert float(P.compressor_gain_law(t64(2.0), -2.0, 1.0, 4.0)) == pytest.approx(-1.0, abs=1e-15)
    assert float(P.noisegate_gain_law(t64(-10.0), -4.0, 1.0, 3.0)) == pytest.approx(-22.0, abs=1e-15)


@pytest.mark.parametrize("law", ["c", "n"])
def test_gain_laws_are_c1_at_knee_edges(law):
    T, W, R = -3.0, 0.7, 2.5
    f = (lambda g: P.compressor_gain_law(g, T, W, R)) if law == "c" else (lambda g: P.noisegate_gain_law(g, T, W, R))
    for edge in (T - W, T + W):
        d = 1e-7
        lo, at, hi = (float(f(t64(edge + s))) for s in (-d, 0.0, d))
        assert abs(hi - lo) < 1e-5
        s_lo = (float(f(t64(edge - d))) - float(f(t64(edge - 2 * d)))) / d
        s_hi = (float(f(t64(edge + 2 * d))) - float(f(t64(edge + d)))) / d
        assert abs(s_lo - s_hi) < 1e-5


# ------------------------------------------------------------------------------------------------
# Sec. 3.4 reverb
# ------------------------------------------------------------------------------------------------

def test_istft_inverts_stft_where_covered():
    x = t64(rng(10).standard_normal(5000))
    spec = P.stft(x, 384, 192)
    y = P.istft_ola(spec, 384, 192, 5000).numpy()
    F = spec.shape[0]
    cover = (F - 1) * 192 + 384
    assert np.allclose(y[1:cover], x.numpy()[1:cover], atol=1e-10)
    assert np.all(y[cover:] == 0.0)


def test_reverb_unit_mask_returns_the_noise():
    noise = t64(rng(11).uniform(-1, 1, (2, 8000)))
    spec = P.reverb_noise_stft(noise)
    p = torch.zeros(2, 2, 192, dtype=F64)
    p[:, 1] = -80.0   # softplus(-80) ~ 1.8e-35: no decay; H0 = 0: unit mask
    h = P.reverb_fir(p.reshape(-1), spec, 8000).numpy()
    F = spec.shape[1]
    cover = (F - 1) * 192 + 384
    nm, ns = noise.numpy()
    assert np.allclose(h[0, 1:cover], (nm + ns)[1:cover], atol=1e-10)
    assert np.allclose(h[1, 1:cover], (nm - ns)[1:cover], atol=1e-10)


def test_reverb_conv_matches_direct():
    r = rng(12)
    noise = t64(r.uniform(-1, 1, (2, 1200)))
    spec = P.reverb_noise_stft(noise)
    p = t64(r.normal(0, 0.3, 768))
    h = P.reverb_fir(p, spec, 1200).numpy()
    u = r.standard_normal((2, 300))
    y = P.reverb(t64(u), p, spec, 1200).numpy()
    for c in range(2):
        assert np.allclose(y[c], P.direct_conv(u[c], h[c], 0), atol=1e-10)


# ------------------------------------------------------------------------------------------------
# Sec. 3.7 multitap delay
# ------------------------------------------------------------------------------------------------

def test_surrogate_on_bin_is_exact_impulse():
    D = 4410
    for d in (0, 1, 1234, 4409):
        z = np.exp(-2j * np.pi * d / D)
        s = P.surrogate_impulse(z, D)
        ref = np.zeros(D)
        ref[d] = 1.0
        assert np.allclose(s, ref, atol=1e-9)
        assert P.delay_positions(np.array([z.real]), np.array([z.imag]), D)[0] == d


def test_surrogate_closed_form_and_derivative():
    D = 4410
    z = 0.93 * np.exp(1j * 0.77)
    n = np.arange(D)
    w = np.exp(2j * np.pi * n / D)
    closed = (1 - z ** D) / (D * (1 - z * w))       # geometric series of Eq. (18)
    assert np.allclose(P.surrogate_impulse(z, D), closed, atol=1e-12)
    h = 1e-6
    fd = (P.surrogate_impulse(z + h, D) - P.surrogate_impulse(z - h, D)) / (2 * h)
    assert np.allclose(P.surrogate_impulse_dz(z, D), fd, atol=1e-6)


def test_delay_forward_matches_sparse_direct_conv():
    r = rng(13)
    D = 50
    p = torch.zeros(2, 20, 22, dtype=F64)
    ang = r.uniform(-np.pi, np.pi, (2, 20))
    p[:, :, 0] = t64(np.cos(ang))
    p[:, :, 1] = t64(np.sin(ang))
    p[:, :, 2:] = t64(r.uniform(-2, 0, (2, 20, 20)))
    u = r.standard_normal((2, 700))
    y = P.multitap_delay(t64(u), p.reshape(-1), D).numpy()
    c = P.zero_phase_fir(p[:, :, 2:], 39).numpy()
    for ch in range(2):
        ref = np.zeros(700)
        for m in range(20):
            off = int(np.mod(np.rint(D * np.mod(-ang[ch, m], 2 * np.pi) / (2 * np.pi)), D))
            dm = m * D + off
            for j in range(-19, 20):
                sh = dm + j          # y[n] += c_m[j] u[n - sh]
                if 0 <= sh < 700:
                    ref[sh:] += c[ch, m, j + 19] * u[ch, : 700 - sh]
                elif sh < 0:
                    ref[: 700 + sh] += c[ch, m, j + 19] * u[ch, -sh:]
        assert np.allclose(y[ch], ref, atol=1e-10)


def test_delay_straight_through_gradient():
    """The z gradient is the closed-form sgn(sum_n G[n] conj(d h_tilde/dz)) + gamma (|z|-1) z/|z|."""
    r = rng(14)
    D = 4410
    p = torch.zeros(2, 20, 22, dtype=F64)
    rad = r.uniform(0.2, 1.3, (2, 20))
    ang = r.uniform(-np.pi, np.pi, (2, 20))
    p[:, :, 0] = t64(rad * np.cos(ang))
    p[:, :, 1] = t64(rad * np.sin(ang))
    p[:, :, 2:] = t64(r.uniform(-2, 0, (2, 20, 20)))
    p.requires_grad_(True)
    taps = P.delay_fir(p.reshape(-1), D, 10 ** 6)
    wts = t64(r.standard_normal(taps.shape))
    (taps * wts).sum().backward()
    g = p.grad.numpy()
    c = P.zero_phase_fir(p.detach()[:, :, 2:], 39).numpy()
    n = np.arange(D)
    w = np.exp(2j * np.pi * n / D)
    for ch in range(2):
        for m in (0, 7, 19):
            z = complex(rad[ch, m] * np.cos(ang[ch, m]), rad[ch, m] * np.sin(ang[ch, m]))
            zc = z / max(1.0, abs(z))
            # closed-form derivative of (1 - z^D) / (D (1 - z w^n))
            ds = (-D * zc ** (D - 1) * (1 - zc * w) + (1 - zc ** D) * w) / (D * (1 - zc * w) ** 2)
            seg = wts.numpy()[ch, m * D: m * D + D + 38]
            G = np.array([seg[q: q + 39] @ c[ch, m] for q in range(D)])
            gm = np.sum(G * np.conj(ds))
            ref = gm / abs(gm) + 0.01 * (abs(z) - 1) * z / abs(z)
            assert abs(g[ch, m, 0] - ref.real) < 1e-8 and abs(g[ch, m, 1] - ref.imag) < 1e-8
    # the FIR log-magnitudes get the exact gradient: sum of the upstream weights under each tap
    lm_fd_idx = (1, 3, 5)
    eps = 1e-6
    pp = p.detach().clone()
    pp[lm_fd_idx] += eps
    up = float((P.delay_fir(pp.reshape(-1), D, 10 ** 6) * wts).sum())
    pp[lm_fd_idx] -= 2 * eps
    dn = float((P.delay_fir(pp.reshape(-1), D, 10 ** 6) * wts).sum())
    assert abs((up - dn) / (2 * eps) - g[lm_fd_idx]) < 1e-6


# ------------------------------------------------------------------------------------------------
# Sec. 5.1 loss
# ------------------------------------------------------------------------------------------------

def test_table_rows_reproduce_printed_audio_loss():
    desc = Lo.LossDesc()
    n = 0
    for line in open(os.path.join(GOLD, "table2_3_loss_rows.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, la, llr, lm, ls = line.split()
        assert abs(Lo.combine(float(llr), float(lm), float(ls), desc) - float(la)) <= 1e-3 + 1e-12, name
        n += 1
    assert n == 8


def test_a_weighting_matches_iec_table():
    for line in open(os.path.join(GOLD, "a_weighting_iec61672.txt")):
        if line.startswith("#") or not line.strip():
            continue
        f, db, _ = map(float, line.split())
        assert abs(20 * math.log10(Lo.a_weight_gain(np.array([f]))[0]) - db) <= 0.051, f


def test_mel_filterbank_shape_and_peaks():
    assert abs(Lo.hz_to_mel(700.0) - 2595.0 * math.log10(2.0)) < 1e-9
    assert abs(Lo.mel_to_hz(Lo.hz_to_mel(1234.5)) - 1234.5) < 1e-9
    W = Lo.mel_filterbank(8192, 96, 44100.0)
    assert W.shape == (96, 4097) and W.min() >= 0.0 and W.max() <= 1.0
    # every band above the lowest few has its peak close to 1 at its centre bin
    assert np.all(W[10:].max(axis=1) > 0.9)


def test_loss_is_zero_for_identical_signals():
    x = t64(rng(15).standard_normal((2, 9000)))
    parts = Lo.audio_loss(x, x, Lo.LossDesc())
    for k in ("lr", "m", "s", "a"):
        assert float(parts[k]) == 0.0


def test_linear_mrstft_matches_scipy_stft():
    scipy_signal = pytest.importorskip("scipy.signal")
    r = rng(16)
    y = r.standard_normal((2, 6000))
    yh = y + 0.3 * r.standard_normal((2, 6000))
    desc = Lo.LossDesc(n_fft=(256, 1024), n_mels=0, a_weighting=False)
    got = Lo.audio_loss(t64(yh), t64(y), desc)

    def mag(x, n):
        win = scipy_signal.get_window("hann", n, fftbins=True)
        _, _, Z = scipy_signal.stft(x, nperseg=n, noverlap=n - n // 4, window=win, boundary=None, padded=False,
                                    detrend=False, return_onesided=True)
        Z = Z * win.sum()           # scipy scales by 1/sum(window)
        return np.sqrt(np.abs(Z.T) ** 2 + 1e-8)

    def setloss(a, b):
        tot = 0.0
        for n in (256, 1024):
            Y = np.stack([mag(ch, n) for ch in b])
            Yh = np.stack([mag(ch, n) for ch in a])
            tot += np.mean(np.abs(np.log(Y + 1e-5) - np.log(Yh + 1e-5))) + np.linalg.norm(Y - Yh) / np.linalg.norm(Y)
        return tot

    ref = {"lr": setloss(yh, y), "m": setloss(yh[:1] + yh[1:], y[:1] + y[1:]), "s": setloss(yh[:1] - yh[1:], y[:1] - y[1:])}
    for k in ref:
        assert float(got[k]) == pytest.approx(ref[k], rel=1e-10)


# ------------------------------------------------------------------------------------------------
# console structure
# ------------------------------------------------------------------------------------------------

def _golden_schedule():
    lines = [l.split() for l in open(os.path.join(GOLD, "console_schedule.txt")) if l.strip() and not l.startswith("#")]
    return lines[0][0], {t: int(n) for t, n in lines[1:]}


def test_schedule_string_and_param_counts():
    sched, counts = _golden_schedule()
    assert C.schedule_string() == sched
    assert C.PARAM_COUNT == counts
    procs, npp, P_ = C.layout([C.SongSpec(4, 1, [0, 0, -1, -1], 1000)])
    assert P_ == 35 and npp == 5 * sum(counts.values())          # 4 tracks + 1 subgroup, 7 processors each
    assert [p.type for p in procs[:7]] == list("ecnsgdr")


def test_adam_first_step_closed_form():
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    p, m, v = A.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    assert np.allclose(p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)   # m_hat = g, v_hat = g^2


def test_adam_later_steps_closed_form():
    """Kingma-Ba bias correction at t = 2 and 3 (Sec. 5.1 optimiser).  With a constant gradient g the corrected
    moments are exactly g and g^2 at every t (m_t = (1 - b1^t) g), so every step moves by -lr g / (|g| + eps);
    with gradients g1 then g2 the corrected moments at t = 2 are (b1 g1 + g2) / (1 + b1) and
    (b2 g1^2 + g2^2) / (1 + b2) (the geometric sums divided by 1 - b^2 = (1 - b)(1 + b)).  A wrong exponent in
    either correction, or the moments updated in the other order, fails one of these."""
    g = np.array([0.5, -2.0, 1e-3, 3.0])
    p, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    for t in (1, 2, 3):
        p, m, v = A.adam_step(p, g, m, v, t, lr=0.01)
        assert np.allclose(p, -0.01 * t * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15), t
    b1, b2 = 0.9, 0.999
    g1 = np.array([0.5, -2.0, 1e-3, 3.0])
    g2 = np.array([-1.5, 0.25, 2e-3, 3.0])
    p1, m1, v1 = A.adam_step(np.ones(4), g1, np.zeros(4), np.zeros(4), 1, lr=0.01)
    p2, _, _ = A.adam_step(p1, g2, m1, v1, 2, lr=0.01)
    mhat = (b1 * g1 + g2) / (1.0 + b1)
    vhat = (b2 * g1 ** 2 + g2 ** 2) / (1.0 + b2)
    assert np.allclose(p2, p1 - 0.01 * mhat / (np.sqrt(vhat) + 1e-8), rtol=1e-12, atol=1e-15)
    # decoupled weight decay: p <- p (1 - lr wd) before the moment step
    p3, _, _ = A.adam_step(np.full(4, 2.0), g, np.zeros(4), np.zeros(4), 1, lr=0.01, weight_decay=0.1)
    assert np.allclose(p3, 2.0 * (1 - 0.001) - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)


# ------------------------------------------------------------------------------------------------
# Eq. (22) gain staging: closed-form values
# ------------------------------------------------------------------------------------------------

def test_gain_staging_closed_forms():
    """Eq. (22): |log ||y_bar_mid||_2 - log ||u_mid||_2| with mid = left + right.
    * y_bar = 2 u gives ln 2 (not 2 ln 2: the log of the norm, not of the energy);
    * a sine of amplitude A over whole periods, on both channels, has ||mid||^2 = (2A)^2 L / 2;
    * the mid is the channel sum: (2x, 0) and (x, x) have the same mid, so the term is 0, while a left-only or
      per-channel-energy reading would give ln 2 or ln sqrt 2; (x, -x) has a silent mid (the 1e-12 floor)."""
    r = rng(21)
    u = t64(r.standard_normal((2, 5000)))
    assert float(Lo.gain_staging(2.0 * u, u)) == pytest.approx(math.log(2.0), rel=1e-12)
    assert float(Lo.gain_staging(u, 0.25 * u)) == pytest.approx(math.log(4.0), rel=1e-12)
    L, A_, B_ = 4800, 0.3, 1.7
    n = np.arange(L)
    s = np.sin(2 * np.pi * 12 * n / L)                      # 12 whole periods
    us, ys = t64(np.stack([A_ * s, A_ * s])), t64(np.stack([B_ * s, B_ * s]))
    assert float(Lo.log_l2(us[0] + us[1])) == pytest.approx(0.5 * math.log((2 * A_) ** 2 * L / 2), rel=1e-12)
    assert float(Lo.gain_staging(ys, us)) == pytest.approx(math.log(B_ / A_), rel=1e-12)
    x = t64(r.standard_normal(3000))
    both = torch.stack([x, x])
    left = torch.stack([2.0 * x, torch.zeros_like(x)])
    assert float(Lo.gain_staging(left, both)) == pytest.approx(0.0, abs=1e-12)
    anti = torch.stack([x, -x])
    expect = abs(0.5 * math.log(1e-12) - 0.5 * math.log(float(torch.sum((2 * x) ** 2))))
    assert float(Lo.gain_staging(anti, both)) == pytest.approx(expect, rel=1e-12)


def test_console_gain_staging_sums_lti_nodes():
    """L_g of a console (Eq. 22 summed over the equalizer, reverb and delay nodes): a flat Eq. (7) response
    exp(c) is the impulse exp(c) delta (v[0] = 1), so an equalizer with every log-magnitude equal to c scales
    its input by exp(c) and contributes |c|, whatever its dry/wet weight; gain/pan nodes contribute nothing."""
    L = 3000
    r = rng(22)
    songs = [C.SongSpec(2, 1, [0, -1], L)]
    src = [r.standard_normal((2, L)).astype(np.float32)]
    con = C.Console(songs, src, None, None, C.ConsoleDesc(types="eg"))
    params = np.zeros(con.n_params)
    consts = {}
    for p in con.procs:
        if p.type == "e":
            c = float(r.uniform(-1.5, 1.5))
            params[p.offset:p.offset + p.count] = c
            consts[p.index] = c
        else:
            params[p.offset:p.offset + p.count] = r.normal(0, 0.5, p.count)
    params[con.n_proc_params:] = r.normal(0, 1.0, con.n_procs)
    with torch.no_grad():
        res = con.forward(t64(params))
    assert float(res[0]["Lg"]) == pytest.approx(sum(abs(c) for c in consts.values()), rel=1e-9)


# ------------------------------------------------------------------------------------------------
# Sec. 3.4 reverb decay (Eq. 10), frame by frame
# ------------------------------------------------------------------------------------------------

def _one_bin_spec(F, k0):
    spec = torch.zeros(F, 193, dtype=torch.complex128)
    spec[:, k0] = 1.0
    return spec


@pytest.mark.parametrize("k0", [5, 192])
def test_reverb_decay_frame_by_frame(k0):
    """Eq. (10): the mask of frame m (1-based) is exp(H0[k] + (m - 1) H_delta[k]), read with
    H_delta = -0.05 softplus(p_delta).  A noise spectrum holding 1 in bin k0 of every frame is masked and
    inverted; at the centre of frame t (0-based, sample t hop + n/2) only that frame's window is nonzero and
    equals 1 (periodic Hann, hop n/2), and the window-sum there is 1, so the FIR sample is the inverse DFT of
    the single bin at n/2: (2/n) a_t (-1)^k0 for an inner bin and a_t / n for the Nyquist bin, a_t the mask.
    So h[centre of frame 0] fixes exp(H0) (no decay at the first frame), and the ratio of consecutive centres
    is exp(H_delta) whatever the frame.  k0 = 192 is the Nyquist bin, which reuses parameter 191."""
    n, hop, F = 384, 192, 40
    L = (F - 1) * hop + n
    h0m, pdm = 0.7, 0.4              # mid: H0 and p_delta of the probed bin
    h0s, pds = -0.3, -1.2            # side
    p = torch.zeros(2, 2, 192, dtype=F64)
    pk = min(k0, 191)
    p[0, 0, :] = -9.0                # every other bin is irrelevant (zero noise); keep them distinct anyway
    p[1, 0, :] = -9.0
    p[0, 0, pk], p[0, 1, pk] = h0m, pdm
    p[1, 0, pk], p[1, 1, pk] = h0s, pds
    spec = torch.stack([_one_bin_spec(F, k0), _one_bin_spec(F, k0)])
    h = P.reverb_fir(p.reshape(-1), spec, L).numpy()
    hm, hs = (h[0] + h[1]) / 2, (h[0] - h[1]) / 2           # h_l = h_m + h_s, h_r = h_m - h_s
    scale = (1.0 / n) if k0 == n // 2 else (2.0 / n) * (-1.0) ** k0

    def softplus(x):
        return math.log1p(math.exp(x))

    for hx, h0, pd in ((hm, h0m, pdm), (hs, h0s, pds)):
        centres = np.array([hx[t * hop + n // 2] for t in range(F)])
        assert centres[0] == pytest.approx(scale * math.exp(h0), rel=1e-10)
        decay = math.exp(-0.05 * softplus(pd))
        assert np.allclose(centres[1:] / centres[:-1], decay, rtol=1e-10, atol=0)
        assert np.allclose(centres, scale * np.exp(h0 - 0.05 * softplus(pd) * np.arange(F)), rtol=1e-10, atol=0)


# ------------------------------------------------------------------------------------------------
# Sec. 5.1 warm-up: which frames the loss keeps
# ------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("warmup", [0, 1, 127, 128, 129, 1000, 44100])
def test_warmup_drops_frames_starting_before_it(warmup):
    """Frames that start before `warmup` samples are dropped (Sec. 5.1 leaves the first second out of the
    loss).  Checked against a hand count of the frame starts t hop < warmup, and by value: two signals that
    differ only before the warm-up give a zero loss, while a difference at the second sample of the first kept
    frame does not (so that frame is not dropped too)."""
    n_fft, hop = 512, 128
    L = 60000
    x = t64(rng(23).standard_normal(L))
    desc0 = Lo.LossDesc(n_fft=(n_fft,), n_mels=0, a_weighting=False, warmup_samples=0)
    descw = Lo.LossDesc(n_fft=(n_fft,), n_mels=0, a_weighting=False, warmup_samples=warmup)
    full = Lo.spectrogram(x, n_fft, desc0)
    kept = Lo.spectrogram(x, n_fft, descw)
    starts = [t * hop for t in range(full.shape[0])]
    dropped = sum(1 for s in starts if s < warmup)
    assert kept.shape[0] == full.shape[0] - dropped
    assert torch.equal(kept, full[dropped:])
    if warmup == 0:
        return
    y = torch.stack([x, x.flip(0)])
    yh = y.clone()
    yh[:, :warmup] += 0.5                   # differs only before the warm-up
    parts = Lo.audio_loss(yh, y, Lo.LossDesc(n_fft=(n_fft,), hop_div=4, n_mels=0, a_weighting=False,
                                             warmup_samples=warmup))
    assert float(parts["a"]) == 0.0
    # sample s0 + 1, s0 = ceil(warmup / hop) hop the start of the first kept frame (its window is 0 at s0):
    # only frames starting at or before it cover it, and of those only the first kept frame is kept
    s0 = dropped * hop
    yh2 = y.clone()
    yh2[:, s0 + 1] += 0.5
    parts2 = Lo.audio_loss(yh2, y, Lo.LossDesc(n_fft=(n_fft,), hop_div=4, n_mels=0, a_weighting=False,
                                               warmup_samples=warmup))
    assert float(parts2["a"]) > 0.0

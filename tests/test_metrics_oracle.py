"""Pins of the evaluation metrics oracle (Sec. 5.3): closed forms of SI-SDR and of each feature."""
import numpy as np
import pytest

from oracle import metrics as OM

FS = 44100.0


def test_si_sdr_closed_forms():
    rng = np.random.default_rng(0)
    ref = rng.standard_normal((2, 1000))
    noise = rng.standard_normal((2, 1000))
    noise -= (noise.ravel() @ ref.ravel()) / (ref.ravel() @ ref.ravel()) * ref     # orthogonal to ref
    est = 3.0 * ref + 0.5 * noise
    expect = 10 * np.log10(np.sum((3.0 * ref) ** 2) / np.sum((0.5 * noise) ** 2))
    assert OM.si_sdr(est, ref) == pytest.approx(expect, abs=1e-9)
    assert OM.si_sdr(-2.0 * ref + 1e-3 * noise, ref) == pytest.approx(OM.si_sdr(ref + -5e-4 * noise, ref), abs=1e-9)


def test_feature_closed_forms():
    n = int(8 * FS)
    t = np.arange(n) / FS
    s = np.sin(2 * np.pi * 1000.0 * t)
    f = OM.features(np.stack([s, 0.5 * s]), FS)
    assert f["rms"] == pytest.approx([np.sqrt(0.5), 0.5 * np.sqrt(0.5)], rel=1e-6)
    assert f["cf"] == pytest.approx([np.sqrt(2), np.sqrt(2)], rel=1e-4)
    assert f["sw"][0] == pytest.approx(0.5 / 1.5)                     # |l - r| / |l + r| = 0.5 / 1.5
    assert f["si"][0] == pytest.approx((1 - 0.25) / (1 + 0.25))
    # a 1 kHz sine puts its energy in the 920-1080 Hz band (index 8)
    assert int(np.argmax(f["bs"])) == 8
    mono = OM.features(np.stack([s, s]), FS)
    assert mono["sw"][0] == 0.0 and mono["si"][0] == 0.0


def test_mir_distances_equal_inputs_and_segmenting():
    rng = np.random.default_rng(1)
    y = rng.standard_normal((2, int(17 * FS)))
    d = OM.mir_distances(y, y, FS)
    assert all(v == -np.inf for v in d.values())
    assert len(OM.segments(y, FS)) == 2 and len(OM.segments(y[:, :1000], FS)) == 1
    # a 2x gain changes RMS by rms and leaves CF and SI unchanged
    d2 = OM.mir_distances(2 * y, y, FS)
    assert d2["cf"] == -np.inf and d2["si"] == -np.inf and d2["sw"] == -np.inf
    r = [OM.features(sg, FS)["rms"] for sg in OM.segments(y, FS)]
    assert d2["rms"] == pytest.approx(np.log10(np.mean(np.concatenate(r) ** 2)))

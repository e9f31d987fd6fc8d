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


def test_classification_metrics_hand_counts():
    types = list("eeeegg")
    truth = [1, 1, 0, 0, 1, 0]
    pred = [1, 0, 1, 0, 1, 1]
    m = OM.classification_metrics(truth, pred, types)
    # e: tp 1, fn 1, fp 1, tn 1 -> accuracy 0.5, precision 0.5, recall 0.5, f1 0.5
    assert m["e"] == {"accuracy": 0.5, "precision": 0.5, "recall": 0.5, "f1": 0.5}
    # g: tp 1, fp 1 -> accuracy 0.5, precision 0.5, recall 1, f1 2/3
    assert m["g"]["precision"] == 0.5 and m["g"]["recall"] == 1.0 and m["g"]["f1"] == pytest.approx(2 / 3)
    # micro: tp 2, fp 2, fn 1, tn 1
    assert m["mu"]["accuracy"] == pytest.approx(3 / 6) and m["mu"]["precision"] == 0.5
    assert m["mu"]["recall"] == pytest.approx(2 / 3) and m["mu"]["f1"] == pytest.approx(2 * 0.5 * (2 / 3) / (0.5 + 2 / 3))
    perfect = OM.classification_metrics(truth, truth, types)
    assert all(v == 1.0 for d in perfect.values() for v in d.values())

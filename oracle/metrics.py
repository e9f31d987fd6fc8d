"""Evaluation metrics of the matched mix (Sec. 5.3): SI-SDR and the MIR feature distances of Eq. (27)
(oracle; test infrastructure).  FP64 numpy, the plain definitions.

Readings (the paper names the features and cites their source without formulas):
  * SI-SDR (Le Roux et al. 2019) over the stereo signal flattened: alpha = <y_hat, y> / ||y||^2,
    SI-SDR = 10 log10(||alpha y||^2 / ||alpha y - y_hat||^2), y the target (reference), y_hat the estimate;
  * segments: disjoint full 8 s segments from the start (a song shorter than 8 s is one segment);
  * RMS: per channel sqrt(mean x^2) (K = 2); crest factor: per channel max |x| / RMS (K = 2);
  * stereo width: ||l - r|| / ||l + r|| (K = 1); stereo imbalance: (||l||^2 - ||r||^2) / (||l||^2 + ||r||^2)
    (K = 1); a quotient with a zero denominator is 0;
  * Bark spectrum: the mid signal (l + r) / 2 in frames of 8192 samples with hop 8192 and a periodic Hann
    window (full frames inside the segment), mean power |X_k|^2 over the frames, summed over the 24 Zwicker
    critical bands (edges below), 10 log10(band power + 1e-12) (K = 24);
  * d_x = log10 of the mean over segments and the K entries of the squared feature difference (Eq. 27).
"""
from __future__ import annotations

from typing import Dict

import numpy as np

SEG_SECONDS = 8.0
BARK_FRAME = 8192
BARK_EDGES_HZ = (0, 100, 200, 300, 400, 510, 630, 770, 920, 1080, 1270, 1480, 1720, 2000, 2320, 2700, 3150,
                 3700, 4400, 5300, 6400, 7700, 9500, 12000, 15500)


def si_sdr(est: np.ndarray, ref: np.ndarray) -> float:
    e = np.asarray(est, np.float64).ravel()
    r = np.asarray(ref, np.float64).ravel()
    alpha = float(e @ r) / float(r @ r)
    target = alpha * r
    res = target - e
    return 10.0 * np.log10(float(target @ target) / float(res @ res))


def _div(a: float, b: float) -> float:
    return a / b if b != 0.0 else 0.0


def segments(x: np.ndarray, fs: float):
    n = int(round(SEG_SECONDS * fs))
    L = x.shape[1]
    if L < n:
        return [x]
    return [x[:, k * n:(k + 1) * n] for k in range(L // n)]


def features(seg: np.ndarray, fs: float) -> Dict[str, np.ndarray]:
    l, r = np.asarray(seg[0], np.float64), np.asarray(seg[1], np.float64)
    rms = np.sqrt(np.array([np.mean(l * l), np.mean(r * r)]))
    peak = np.array([np.max(np.abs(l)), np.max(np.abs(r))])
    cf = np.array([_div(peak[0], rms[0]), _div(peak[1], rms[1])])
    sw = np.array([_div(np.linalg.norm(l - r), np.linalg.norm(l + r))])
    el, er = float(l @ l), float(r @ r)
    si = np.array([_div(el - er, el + er)])
    mid = 0.5 * (l + r)
    nfr = mid.shape[0] // BARK_FRAME
    win = 0.5 * (1.0 - np.cos(2.0 * np.pi * np.arange(BARK_FRAME) / BARK_FRAME))
    power = np.zeros(BARK_FRAME // 2 + 1)
    for f in range(nfr):
        X = np.fft.rfft(mid[f * BARK_FRAME:(f + 1) * BARK_FRAME] * win)
        power += np.abs(X) ** 2
    if nfr:
        power /= nfr
    freqs = np.arange(BARK_FRAME // 2 + 1) * fs / BARK_FRAME
    bands = np.array([power[(freqs >= BARK_EDGES_HZ[b]) & (freqs < BARK_EDGES_HZ[b + 1])].sum()
                      for b in range(len(BARK_EDGES_HZ) - 1)])
    bs = 10.0 * np.log10(bands + 1e-12)
    return {"rms": rms, "cf": cf, "sw": sw, "si": si, "bs": bs}


def mir_distances(est: np.ndarray, ref: np.ndarray, fs: float) -> Dict[str, float]:
    """Eq. (27) for x in RMS, CF, SW, SI, BS."""
    se, sr = segments(np.asarray(est), fs), segments(np.asarray(ref), fs)
    acc: Dict[str, float] = {}
    cnt: Dict[str, int] = {}
    for a, b in zip(se, sr):
        fa, fb = features(a, fs), features(b, fs)
        for k in fa:
            acc[k] = acc.get(k, 0.0) + float(np.sum((fa[k] - fb[k]) ** 2))
            cnt[k] = cnt.get(k, 0) + fa[k].size
    return {k: float(np.log10(acc[k] / cnt[k])) if acc[k] > 0 else -np.inf for k in acc}


def classification_metrics(truth, pred, types, type_order: str = "ecnsgdr") -> Dict[str, Dict[str, float]]:
    """Consistency check (Sec. 7.3): processors present in the pruned graph G (truth) against those present
    after re-running the search on G's own mix (pred), one binary decision per (input or subgroup chain, type).
    Per type and micro-averaged (key "mu") accuracy, precision, recall and F1; positive = present.  A metric with
    a zero denominator is reported as 1.0 when its numerator is zero as well (nothing to get wrong)."""
    truth = np.asarray(truth, bool)
    pred = np.asarray(pred, bool)
    types = np.asarray(list(types))

    def stats(sel):
        t, p = truth[sel], pred[sel]
        tp = int(np.sum(t & p))
        fp = int(np.sum(~t & p))
        fn = int(np.sum(t & ~p))
        tn = int(np.sum(~t & ~p))
        div = lambda a, b: a / b if b else 1.0
        prec, rec = div(tp, tp + fp), div(tp, tp + fn)
        f1 = div(2 * prec * rec, prec + rec) if (tp + fp and tp + fn) else div(2 * tp, 2 * tp + fp + fn)
        return {"accuracy": div(tp + tn, tp + tn + fp + fn), "precision": prec, "recall": rec, "f1": f1}

    out = {t: stats(types == t) for t in type_order if np.any(types == t)}
    out["mu"] = stats(np.ones(truth.shape, bool))
    return out

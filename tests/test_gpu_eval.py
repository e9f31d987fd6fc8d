"""Evaluation metrics (Sec. 5.3) on the GPU against the metric oracle on the same FP32 mix and target (GPU)."""
import numpy as np
import pytest

import workloads as W
import paper_2509_15948_gb300 as M
from oracle import metrics as OM

pytestmark = pytest.mark.gpu


def test_evaluate_matches_the_metric_oracle():
    lays = [W.SongLayout(3, 1, [0, -1, 0], 400000), W.SongLayout(2, 0, [-1, -1], 30011),
            W.SongLayout(4, 2, [0, 1, 0, -1], 720000)]
    rng = np.random.default_rng(3)
    sources = [W.song_sources(l, (9, i)) for i, l in enumerate(lays)]
    targets = []
    for src in sources:
        mono = src.sum(axis=0)
        targets.append(np.stack([0.4 * mono, 0.25 * mono]).astype(np.float32)
                       + 0.01 * rng.standard_normal((2, src.shape[1])).astype(np.float32))
    types = W.processor_types(lays)
    noise = W.reverb_noise((9,), sum(t == "r" for t in types))
    con = M.Console([M.Song(l.num_tracks, l.num_subgroups, l.track_group, l.num_samples) for l in lays],
                    sources, targets, noise, M.ConsoleConfig())
    con.set_params(W.init_params(types, (9, 5)))
    _, mixes = con.forward_loss(with_mix=True)
    got = con.evaluate().cpu().numpy()
    for s, (mix, tgt) in enumerate(zip(mixes, targets)):
        mix = mix.cpu().numpy().astype(np.float64)
        assert got[s, 0] == pytest.approx(OM.si_sdr(mix, tgt), abs=1e-3)
        d = OM.mir_distances(mix, tgt, 44100.0)
        for j, k in enumerate(("rms", "cf", "sw", "si", "bs")):
            assert got[s, 1 + j] == pytest.approx(d[k], abs=1e-4), (s, k, got[s, 1 + j], d[k])

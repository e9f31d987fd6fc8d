"""Host logic of the search driver (Alg. 3) against the oracle's one-song round, without a GPU.

A fake console stands in for the CUDA one: its L_a of song s under a mask is a fixed base plus a fixed
(signed) cost for every switched-off processor of s, so some trials are accepted and some fail."""
import numpy as np
import pytest

from oracle import search as OS
from paper_2509_15948_gb300 import search as GS


class FakeTensor:
    def __init__(self, a):
        self.a = np.asarray(a)

    def cpu(self):
        return self

    def numpy(self):
        return self.a

    def __getitem__(self, i):
        return FakeTensor(self.a[i])


class FakeConsole:
    def __init__(self, song_sizes, types_str="ecnsgdr", seed=0):
        rng = np.random.default_rng(seed)
        self.types, self.song = [], []
        for s, nchains in enumerate(song_sizes):
            for _ in range(nchains):
                for t in types_str:
                    self.types.append(t)
                    self.song.append(s)
        self.song = np.array(self.song, np.int32)
        self.n_processors = len(self.types)
        self.n_songs = len(song_sizes)
        self.n_proc_params = 10
        self.q = rng.normal(0.0, 1.0, self.n_processors)
        self.cost = rng.normal(0.0, 0.01, self.n_processors)   # accepted when base + sum(cost) < l_min + tau
        self.base = rng.uniform(0.2, 0.6, self.n_songs)
        self._present = np.ones(self.n_processors, np.uint8)
        self.calls = 0

    def processor_types(self):
        return list(self.types)

    def layout(self):
        return None, None, self.song

    def present(self):
        return self._present

    def get_params(self):
        return FakeTensor(np.concatenate([np.zeros(self.n_proc_params), self.q]).astype(np.float32))

    def la(self, mask):
        return np.array([self.base[s] + np.sum(self.cost[(self.song == s) & (mask == 0)])
                         for s in range(self.n_songs)])

    def prune_scores(self, masks):
        self.calls += 1
        return FakeTensor(np.stack([self.la(m) for m in masks]).astype(np.float32))


def oracle_song_round(con, s, l_min, tau, seed):
    """The oracle's Alg. 3 round on song s alone (processor indices local to the song)."""
    idx = np.nonzero(con.song == s)[0]
    w = GS.dry_wet_weights(con.get_params().numpy()[con.n_proc_params:])
    types = [con.types[i] for i in idx]

    def evaluate(local_mask):
        full = np.ones(con.n_processors, np.uint8)
        full[idx] = local_mask
        return float(np.float32(con.la(full)[s]))

    m, lm, trace = OS.dry_wet_round(w[idx], types, np.ones(len(idx), np.uint8), l_min, tau, evaluate,
                                    OS.SplitMix64(seed))
    return idx, m, lm, trace


def test_splitmix64_matches_published_output():
    g = GS.SplitMix64(0)
    assert g.next() == 0xE220A8397B1DCDAF


@pytest.mark.parametrize("window", [1, 3, 16])
@pytest.mark.parametrize("tau", [0.0, 0.01])
def test_lockstep_round_equals_per_song_oracle_rounds(tau, window):
    """Speculative windows (several trials per song and call, taken up to the first accepted one) give the
    one-trial-at-a-time decisions; window 1 is one call per trial step."""
    con = FakeConsole([3, 1, 5, 2], seed=7)
    l_min = [float(np.float32(b)) for b in con.base]
    rngs = [GS.SplitMix64(GS.song_seed(11, s)) for s in range(con.n_songs)]
    keep, lm, trials = GS.dry_wet_round(con, l_min, tau, rngs, window=window)
    steps = max(sum(1 for t in trials if t.song == s) for s in range(con.n_songs))
    if window == 1:
        assert con.calls == steps
    else:
        assert con.calls < steps
    for s in range(con.n_songs):
        idx, m, olm, trace = oracle_song_round(con, s, l_min[s], tau, GS.song_seed(11, s))
        mine = [(t.type, tuple(int(i) for i in t.candidates), t.la, t.accepted) for t in trials if t.song == s]
        theirs = [(t, tuple(int(idx[i]) for i in c), la, ok) for (t, c, la, ok) in trace]
        assert mine == theirs, s
        assert np.array_equal(keep[idx], m)
        assert lm[s] == olm
    assert 0 < int(np.sum(keep == 0)) < con.n_processors     # the fixture both prunes and keeps


def test_round_skips_absent_processors():
    con = FakeConsole([2, 2], seed=3)
    con._present[::3] = 0
    rngs = [GS.SplitMix64(GS.song_seed(5, s)) for s in range(con.n_songs)]
    keep, _, trials = GS.dry_wet_round(con, list(con.base), 0.01, rngs)
    absent = np.nonzero(con._present == 0)[0]
    assert all(i not in absent for t in trials for i in t.candidates)
    assert np.all(keep[absent] == 0)


def test_alpha_p_ramp():
    assert GS.alpha_p_at(0, 100, 1e-4) == 0.0
    assert GS.alpha_p_at(50, 100, 1e-4) == pytest.approx(5e-5)
    assert GS.alpha_p_at(400, 100, 1e-4) == 1e-4


@pytest.mark.parametrize("window", [1, 4, 16])
@pytest.mark.parametrize("tau", [0.0, 0.01])
def test_lockstep_brute_force_equals_per_song_oracle_rounds(tau, window):
    con = FakeConsole([2, 1, 3], seed=5)
    l_min = [float(np.float32(b)) for b in con.base]
    rngs = [GS.SplitMix64(GS.song_seed(4, s)) for s in range(con.n_songs)]
    keep, lm, trials = GS.brute_force_round(con, l_min, tau, rngs, window=window)
    if window > 1:
        assert con.calls < max(sum(1 for t in trials if t.song == s) for s in range(con.n_songs))
    for s in range(con.n_songs):
        idx = np.nonzero(con.song == s)[0]

        def evaluate(local_mask):
            full = np.ones(con.n_processors, np.uint8)
            full[idx] = local_mask
            return float(np.float32(con.la(full)[s]))

        m, olm, trace = OS.brute_force_round(np.ones(len(idx), np.uint8), l_min[s], tau, evaluate,
                                             OS.SplitMix64(GS.song_seed(4, s)))
        mine = [(t.candidates[0], t.la, t.accepted) for t in trials if t.song == s]
        assert mine == [(int(idx[v]), la, ok) for (v, la, ok) in trace]
        assert np.array_equal(keep[idx], m) and lm[s] == olm


def test_node_deltas_match_the_oracle_definition():
    con = FakeConsole([2, 3], seed=8)
    con._present[4] = 0
    d = GS.node_deltas(con, max_masks=5)
    for s in range(con.n_songs):
        idx = np.nonzero(con.song == s)[0]
        base = float(np.float32(con.la(np.ones(con.n_processors, np.uint8))[s]))

        def evaluate(local_mask):
            full = np.ones(con.n_processors, np.uint8)
            full[idx] = local_mask
            return float(np.float32(con.la(full)[s]))

        od = OS.node_deltas(base, evaluate, con._present[idx])
        assert np.allclose(d[idx], od, equal_nan=True, rtol=0, atol=1e-12)


def test_hybrid_uses_brute_force_every_fourth_round():
    assert [GS.uses_brute_force(n) for n in range(1, 9)] == [OS.uses_brute_force(n) for n in range(1, 9)]


def test_presence_scores_equal_the_oracle_definition():
    from oracle import metrics as OMet
    rng = np.random.default_rng(2)
    types = [t for t in "ecnsgdr" for _ in range(9)]
    for _ in range(10):
        truth = rng.random(len(types)) < 0.5
        pred = rng.random(len(types)) < 0.5
        assert GS.presence_scores(truth, pred, types) == OMet.classification_metrics(truth, pred, types)
    assert GS.presence_scores(truth, truth, types)["mu"]["f1"] == 1.0

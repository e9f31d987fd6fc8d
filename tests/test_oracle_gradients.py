"""Oracle gradients against central finite differences (FP64, step 1e-4) on tiny consoles, the
pruned-equals-masked invariant, and hand-traced runs of Alg. 3 (CPU only)."""
import numpy as np
import pytest

import workloads as W
from oracle import console as C
from oracle import loss as Lo
from oracle import search as S

TINY_LOSS = Lo.LossDesc(n_fft=(128, 256, 512), n_mels=16)


def tiny_console(L=3000, types="ecnsgdr", seed=0):
    lay = W.SongLayout(2, 1, [0, -1], L)
    songs = [C.SongSpec(lay.num_tracks, lay.num_subgroups, lay.track_group, L)]
    src = [W.song_sources(lay, (99, seed))]
    ptypes = W.processor_types([lay], types)
    noise = W.reverb_noise((99, seed), max(1, sum(t == "r" for t in ptypes)))
    desc = C.ConsoleDesc(types=types, loss=TINY_LOSS)
    gt, keep = W.ground_truth(ptypes, (99, seed))
    tgt = C.Console(songs, src, None, noise, desc).render_targets(gt, keep)
    cons = C.Console(songs, src, tgt, noise, desc)
    return cons, ptypes


def _fd_indices(cons, rng):
    idx = []
    for p in cons.procs:
        n = p.count
        if p.type == "d":
            cand = [k for k in range(n) if k % 22 >= 2]          # FIR log-magnitudes only (z is straight-through)
        else:
            cand = list(range(n))
        idx.extend(p.offset + int(k) for k in rng.choice(cand, size=min(3, len(cand)), replace=False))
        idx.append(cons.n_proc_params + p.index)               # dry/wet logit
    return idx


@pytest.mark.parametrize("types", ["ecnsgdr", "gs", "cn", "erd"])
def test_gradients_match_central_differences(types):
    cons, ptypes = tiny_console(types=types)
    rng = np.random.default_rng(1)
    params = W.init_params(ptypes, (5,)).astype(np.float64)
    alpha_p = 1e-3
    _, grad, _ = cons.loss_and_grad(params, alpha_p=alpha_p)
    h = 1e-4
    for i in _fd_indices(cons, rng):
        pp = params.copy()
        pp[i] += h
        up = cons.losses(pp, alpha_p=alpha_p)[0][:, 6].sum()
        pp[i] -= 2 * h
        dn = cons.losses(pp, alpha_p=alpha_p)[0][:, 6].sum()
        fd = (up - dn) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-5 * abs(grad[i]) + 1e-7 * max(1.0, abs(up)), (i, fd, grad[i])


def test_pruned_console_equals_masked_console():
    cons, ptypes = tiny_console()
    params = W.init_params(ptypes, (6,)).astype(np.float64)
    drop = np.ones(len(ptypes), np.uint8)
    drop[[0, 3, 9, 13]] = 0
    lm, mm = cons.losses(params, mask=drop)
    lp, mp = cons.losses(params, present=drop)
    assert np.array_equal(mm[0], mp[0])
    assert lm[0, 0] == lp[0, 0]


def test_splitmix64_reference_output():
    g = S.SplitMix64(0)
    assert g.next() == 0xE220A8397B1DCDAF   # published first output for seed 0 (Vigna's reference code)


def _scripted(costs, base=1.0):
    def ev(mask):
        return base + float(np.sum(np.asarray(costs)[np.asarray(mask) == 0]))
    return ev


def test_alg3_single_type_drop_after_unit_failure():
    P_ = 10
    w = np.linspace(0.1, 1.0, P_)
    costs = np.zeros(P_)
    costs[3] = 0.02
    m, lmin, trace = S.dry_wet_round(w, ["g"] * P_, np.ones(P_, int), 1.0, 0.01, _scripted(costs), S.SplitMix64(7))
    assert [t[1] for t in trace] == [(0,), (1,), (2,), (3,)]
    assert [t[3] for t in trace] == [True, True, True, False]
    assert list(np.where(m == 0)[0]) == [0, 1, 2] and lmin == 1.0


def test_alg3_ratio_halving_and_threshold_update():
    P_ = 40
    w = np.linspace(0.01, 0.4, P_)
    costs = np.zeros(P_)
    costs[6] = 0.02
    costs[0] = -0.005          # pruning node 0 improves the match: L_min moves down (Alg. 3)
    m, lmin, trace = S.dry_wet_round(w, ["e"] * P_, np.ones(P_, int), 1.0, 0.01, _scripted(costs), S.SplitMix64(3))
    # k = 4 -> accept {0..3}; k = 4 {4..7} fails (node 6) -> r halves; k = 2 {4,5} accepted;
    # k = 2 {6,7} fails -> r halves; k = 1 {6} fails -> type dropped
    assert [t[1] for t in trace] == [(0, 1, 2, 3), (4, 5, 6, 7), (4, 5), (6, 7), (6,)]
    assert [t[3] for t in trace] == [True, False, True, False, False]
    assert lmin == pytest.approx(0.995)
    assert list(np.where(m == 0)[0]) == [0, 1, 2, 3, 4, 5]


def test_alg3_skips_absent_processors_and_types():
    types = ["e", "e", "g", "g", "r"]
    present = [1, 0, 1, 1, 0]
    w = [0.5, 0.1, 0.2, 0.3, 0.0]
    m, _, trace = S.dry_wet_round(w, types, present, 1.0, 0.01, _scripted(np.zeros(5)), S.SplitMix64(11))
    tried = sorted(i for t in trace for i in t[1])
    assert tried == [0, 2, 3] and m[1] == 1 and m[4] == 1


def test_brute_force_round_tries_every_processor_once_and_keeps_the_costly_ones():
    # nodes 2 and 5 cost more than tau: never pruned; node 0 improves the match (L_min moves down); the rest
    # are free.  The outcome does not depend on the draw order.
    costs = np.zeros(8)
    costs[2] = costs[5] = 0.02
    costs[0] = -0.005
    present = np.ones(8, int)
    present[7] = 0
    m, lmin, trace = S.brute_force_round(present, 1.0, 0.01, _scripted(costs), S.SplitMix64(5))
    assert sorted(t[0] for t in trace) == [0, 1, 2, 3, 4, 5, 6]
    assert list(np.where(m == 0)[0]) == [0, 1, 3, 4, 6] and m[7] == 1
    assert lmin == pytest.approx(0.995)
    assert all(ok == (t[0] not in (2, 5)) for t in trace for ok in [t[2]])


def test_brute_force_round_order_decides_between_two_partial_costs():
    # two nodes of cost 0.006 each: the first tried fits under tau, the second then does not
    costs = np.zeros(4)
    costs[1] = costs[3] = 0.006
    m, _, trace = S.brute_force_round(np.ones(4, int), 1.0, 0.01, _scripted(costs), S.SplitMix64(9))
    tried = [t[0] for t in trace if t[0] in (1, 3)]
    assert m[tried[0]] == 0 and m[tried[1]] == 1
    # the draw is pool[next() mod |pool|] over the pool in ascending order
    g, pool = S.SplitMix64(9), [0, 1, 2, 3]
    first = pool[g.next() % 4]
    assert trace[0][0] == first


def test_hybrid_schedule_and_node_deltas():
    assert [S.uses_brute_force(n) for n in range(1, 13)] == [n % 4 == 0 for n in range(1, 13)]
    costs = np.array([0.1, -0.2, 0.0, 0.3])
    d = S.node_deltas(1.0, _scripted(costs), [1, 1, 0, 1])
    assert np.allclose(d[[0, 1, 3]], costs[[0, 1, 3]]) and np.isnan(d[2])

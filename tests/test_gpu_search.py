"""Alg. 3 search on the CUDA console against the oracle (GPU).

The round is replayed twice: (a) through the oracle's round logic with the GPU's own evaluations, which
must give the identical trial sequence and pruned set; (b) trial by trial with the oracle's FP64 L_a at the
same masks and parameters.  Alg. 3 decides on d = L_a(trial) - L_min < tau, a difference of two losses of
nearly the same mix, so (b) holds d to the gradient bound (1e-3 relative, plus 1e-6 of L_a for rounding,
plus the L_a floor below) and requires the same decision wherever |d - tau| exceeds twice that bound.  With no
near-tie the oracle's own search takes the same decisions in the same order, so its pruned set is the GPU's.
L_a itself is held to 1e-5 relative plus the change of the oracle's L_a when its mix moves by white noise of
relative L2 1e-5 (the log-spectral term of Eq. 21 is sensitive on near-silent bins, so FP32 rounding of the mix
shifts L_a by a nearly constant amount that cancels in d)."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import loss as OL
from oracle import search as OS
from paper_2509_15948_gb300 import search as GS
from tests.cases import make_case, gpu_console

pytestmark = pytest.mark.gpu

LA_TOL = 1e-5
D_TOL = 1e-3


def test_dry_wet_round_matches_oracle():
    tau = 0.01
    # start near the ground-truth graph, so that the mix has the target's level and L_a the paper's scale
    # (at the initial parameters the raw reverb magnitudes make the mix ~1e5 times louder than the target)
    seed_case = 1
    case = make_case([W.layout_plain(88200)], seed=seed_case)
    gt, gt_keep = W.ground_truth(case.ptypes, (seed_case, 77))
    npp = case.oracle.n_proc_params
    start = gt.copy()
    start[npp:] = np.where(gt_keep == 1, 4.0, -4.0)
    con = gpu_console(case)
    con.set_params(start)
    for _ in range(5):
        con.train_step(1e-2)
    params = con.get_params().cpu().numpy()
    P = con.n_processors
    l_min0 = float(con.prune_scores(np.ones((1, P), np.uint8))[0, 0])
    seed = GS.song_seed(3, 0)
    keep, lm, trials = GS.dry_wet_round(con, [l_min0], tau, [GS.SplitMix64(seed)])
    assert len(trials) >= 3

    # (a) the oracle's round logic on the GPU's evaluations
    w = GS.dry_wet_weights(params[con.n_proc_params:])
    gpu_eval = lambda m: float(con.prune_scores(np.asarray(m, np.uint8)[None, :])[0, 0])
    m, olm, trace = OS.dry_wet_round(w, con.processor_types(), np.ones(P, np.uint8), l_min0, tau, gpu_eval,
                                     OS.SplitMix64(seed))
    assert [(t.type, tuple(t.candidates), t.la, t.accepted) for t in trials] == \
           [(t, tuple(c), la, ok) for (t, c, la, ok) in trace]
    assert np.array_equal(keep, m) and lm[0] == olm

    # (b) FP64 oracle losses at every trial mask
    full, mixes = case.oracle.losses(params)
    mix = torch.tensor(mixes[0], dtype=torch.float64)
    tgt = torch.tensor(case.targets[0], dtype=torch.float64)
    noise = torch.tensor(np.random.default_rng(0).standard_normal(mix.shape))
    noise *= 1e-5 * mix.norm() / noise.norm()
    floor = abs(float(OL.audio_loss(mix + noise, tgt, case.oracle.desc.loss)["a"]) - full[0, 0])
    l_min_o, l_min_g = full[0, 0], l_min0
    assert abs(l_min_g - l_min_o) <= LA_TOL * abs(l_min_o) + floor
    removed, near_ties = set(), 0
    for t in trials:
        mask = np.ones(P, np.uint8)
        mask[list(removed | set(t.candidates))] = 0
        row, mix_t = case.oracle.losses(params, mask=mask)
        la_o = row[0, 0]
        assert abs(t.la - la_o) <= LA_TOL * abs(la_o) + floor, (t, la_o, floor)
        d_g, d_o = t.la - l_min_g, la_o - l_min_o
        tol = D_TOL * abs(d_o) + 1e-6 * abs(la_o) + floor
        assert abs(d_g - d_o) <= tol, (t, d_g, d_o, tol)
        if abs(d_o - tau) <= 2 * tol:
            near_ties += 1
        else:
            assert (d_o < tau) == t.accepted, (t, d_o)
        if t.accepted:
            l_min_o, l_min_g = min(l_min_o, la_o), min(l_min_g, t.la)
            removed |= set(t.candidates)
    print(f"trials {len(trials)}, pruned {int(np.sum(keep == 0))} of {P}, near ties {near_ties}, "
          f"L_a floor {floor:.3g}")
    assert near_ties == 0       # every decision is resolved: the pruned set is the oracle's


def near_ground_truth_console(seed_case=1, steps=5):
    case = make_case([W.layout_plain(88200)], seed=seed_case)
    gt, gt_keep = W.ground_truth(case.ptypes, (seed_case, 77))
    start = gt.copy()
    start[case.oracle.n_proc_params:] = np.where(gt_keep == 1, 4.0, -4.0)
    con = gpu_console(case)
    con.set_params(start)
    for _ in range(steps):
        con.train_step(1e-2)
    return case, con


def la_floor(case, params):
    full, mixes = case.oracle.losses(params)
    mix = torch.tensor(mixes[0], dtype=torch.float64)
    tgt = torch.tensor(case.targets[0], dtype=torch.float64)
    noise = torch.tensor(np.random.default_rng(0).standard_normal(mix.shape))
    noise *= 1e-5 * mix.norm() / noise.norm()
    return full, abs(float(OL.audio_loss(mix + noise, tgt, case.oracle.desc.loss)["a"]) - full[0, 0])


def test_brute_force_round_matches_oracle():
    """Brute-force sampling (every processor tried alone): the same two replays as the dry/wet round."""
    tau = 0.01
    case, con = near_ground_truth_console()
    params = con.get_params().cpu().numpy()
    P = con.n_processors
    l_min0 = float(con.prune_scores(np.ones((1, P), np.uint8))[0, 0])
    seed = GS.song_seed(6, 0)
    keep, lm, trials = GS.brute_force_round(con, [l_min0], tau, [GS.SplitMix64(seed)])
    assert len(trials) == P
    gpu_eval = lambda m: float(con.prune_scores(np.asarray(m, np.uint8)[None, :])[0, 0])
    m, olm, trace = OS.brute_force_round(np.ones(P, np.uint8), l_min0, tau, gpu_eval, OS.SplitMix64(seed))
    assert [(t.candidates[0], t.la, t.accepted) for t in trials] == trace
    assert np.array_equal(keep, m) and lm[0] == olm
    full, floor = la_floor(case, params)
    l_min_o, l_min_g = full[0, 0], l_min0
    removed, near_ties = set(), 0
    for t in trials:
        mask = np.ones(P, np.uint8)
        mask[list(removed | set(t.candidates))] = 0
        la_o = case.oracle.losses(params, mask=mask)[0][0, 0]
        d_g, d_o = t.la - l_min_g, la_o - l_min_o
        tol = D_TOL * abs(d_o) + 1e-6 * abs(la_o) + floor
        assert abs(d_g - d_o) <= tol, (t, d_g, d_o, tol)
        if abs(d_o - tau) <= 2 * tol:
            near_ties += 1
        else:
            assert (d_o < tau) == t.accepted, (t, d_o)
        if t.accepted:
            l_min_o, l_min_g = min(l_min_o, la_o), min(l_min_g, t.la)
            removed |= set(t.candidates)
    print(f"brute force: pruned {int(np.sum(keep == 0))} of {P}, near ties {near_ties}")
    assert near_ties == 0


def test_node_deltas_match_oracle():
    """Delta_i = L_a(G minus v_i) - L_a(G) (Sec. 7.2) for every processor, scored with batched masks."""
    case, con = near_ground_truth_console()
    params = con.get_params().cpu().numpy()
    d = GS.node_deltas(con, max_masks=16)
    full, floor = la_floor(case, params)
    od = OS.node_deltas(full[0, 0], lambda m: case.oracle.losses(params, mask=m)[0][0, 0],
                        np.ones(con.n_processors, np.uint8))
    err = np.abs(d - od)
    assert np.all(err <= D_TOL * np.abs(od) + 1e-6 * abs(full[0, 0]) + floor), (err.max(), np.abs(od).max())


def test_search_rounds_prune_and_fine_tune():
    """Four hybrid rounds on a two-song batch: the pruned set is what the trials accepted, the pruned console
    keeps training, and the final losses are finite."""
    case = make_case([W.layout_plain(44100), W.SongLayout(3, 1, [0, -1, 0], 30011)], seed=3)
    con = gpu_console(case)
    con.set_params(case.params)
    res = GS.search(con, n_iter=4, train_steps=10, finetune_steps=3, seed=1, method="hybrid")
    present = con.present()
    accepted = {i for rnd in res.trials for t in rnd if t.accepted for i in t.candidates}
    assert set(np.nonzero(present == 0)[0]) == accepted
    assert all(np.isfinite(res.la_final)) and all(0.0 <= r <= 1.0 for r in res.pruning_ratio)
    for rnd in res.trials:
        for s in range(con.n_songs):
            assert any(t.song == s for t in rnd)
    # hybrid: rounds 1-3 dry/wet (a round starts with k = round(0.1 N_t) candidates), round 4 brute force
    assert all(len(t.candidates) == 1 for t in res.trials[3]) and len(res.trials[3]) >= 1


def test_crop_feeder_equals_a_console_built_on_the_crop():
    """The training regime of Sec. 5.1: a crop-length console fed a random segment computes exactly what a
    console created on that segment computes (losses with a loss warm-up, mixes)."""
    import paper_2509_15948_gb300 as M
    case = make_case([W.layout_plain(88200)], seed=4)
    crop = 44100 + 13
    song = M.Song(4, 1, [0, 0, -1, -1], crop)
    cfg = M.ConsoleConfig(warmup_samples=22050)
    src, tgt = case.sources[0], case.targets[0]
    con = M.Console([song], [src[:, :crop]], [tgt[:, :crop]], case.noise, cfg)
    feeder = GS.CropFeeder(con, [src], [tgt], seed=3)
    off = feeder.next()[0]
    assert 0 <= off <= 88200 - crop
    con.set_params(case.params)
    l1, m1 = con.forward_loss(with_mix=True)
    ref = M.Console([song], [src[:, off:off + crop]], [tgt[:, off:off + crop]], case.noise, cfg)
    ref.set_params(case.params)
    l2, m2 = ref.forward_loss(with_mix=True)
    assert np.array_equal(l1.cpu().numpy(), l2.cpu().numpy())
    assert np.array_equal(m1[0].cpu().numpy(), m2[0].cpu().numpy())
    assert feeder.next()[0] != off or feeder.next()[0] != off     # offsets move


def test_crop_trained_search_evaluated_on_full_songs():
    import paper_2509_15948_gb300 as M
    case = make_case([W.layout_plain(88200)], seed=5)
    crop = 44100
    cfg = M.ConsoleConfig(warmup_samples=11025)
    src, tgt = case.sources[0], case.targets[0]
    con = M.Console([M.Song(4, 1, [0, 0, -1, -1], crop)], [src[:, :crop]], [tgt[:, :crop]], case.noise, cfg)
    full = gpu_console(case)
    con.set_params(case.params)
    res = GS.search(con, n_iter=2, train_steps=6, finetune_steps=3, seed=2,
                    feeder=GS.CropFeeder(con, [src], [tgt], seed=2), eval_con=full)
    assert np.array_equal(con.present(), full.present())
    assert np.isfinite(res.la_final).all() and 0.0 <= res.pruning_ratio[0] <= 1.0
    assert np.array_equal(con.get_params().cpu().numpy(), full.get_params().cpu().numpy())


def test_consistency_check_runs_the_protocol():
    """Sec. 7.3: re-running the search on the pruned graph's own mix recovers most of its processor set."""
    import paper_2509_15948_gb300 as M
    case, con = near_ground_truth_console(seed_case=1, steps=0)
    GS.search(con, n_iter=1, train_steps=5, finetune_steps=3, seed=1)
    songs = [M.Song(l.num_tracks, l.num_subgroups, l.track_group, l.num_samples) for l in case.layouts]
    make = lambda targets: M.Console(songs, case.sources, targets, case.noise, M.ConsoleConfig())
    scores = GS.consistency_check(con, make, con.get_params().cpu().numpy(), n_iter=1, train_steps=5,
                                  finetune_steps=3, seed=1)
    assert set(scores) >= {"mu"} and all(0.0 <= v <= 1.0 for d in scores.values() for v in d.values())
    print("consistency", {k: round(v["f1"], 3) for k, v in scores.items()})


def test_config1_trained_round_replayed_through_oracle():
    """The single-song search configuration (16 tracks x 10 s, 4 subgroups of 4): 2,000 Adam steps at lr 1e-2
    on the GPU from the N(0, 0.1^2) initialisation, then one dry/wet round (Alg. 3, tau = 0.01) from the trained
    parameters.  The oracle replays the round's trial sequence at the same parameters (the pruned-set identity
    protocol): every trial's L_a and d = L_a - L_min against the oracle's FP64 values, and the same decision
    wherever d is not a near tie, so with no near tie the accepted set is the oracle's."""
    tau = 0.01
    case = make_case([W.layout_single_search()], seed=11)
    con = gpu_console(case)
    con.set_params(case.params)
    for _ in range(2000):
        con.train_step(1e-2)
    params = con.get_params().cpu().numpy()
    P = con.n_processors
    l_min_g = float(con.prune_scores(np.ones((1, P), np.uint8))[0, 0])
    _, _, trials = GS.dry_wet_round(con, [l_min_g], tau, [GS.SplitMix64(GS.song_seed(7, 0))])
    assert len(trials) >= 5
    full, floor = la_floor(case, params)
    l_min_o = full[0, 0]
    assert abs(l_min_g - l_min_o) <= LA_TOL * abs(l_min_o) + floor
    removed, near_ties, accepted = set(), 0, 0
    for t in trials:
        mask = np.ones(P, np.uint8)
        mask[list(removed | set(t.candidates))] = 0
        la_o = case.oracle.losses(params, mask=mask)[0][0, 0]
        assert abs(t.la - la_o) <= LA_TOL * abs(la_o) + floor, (t, la_o, floor)
        d_g, d_o = t.la - l_min_g, la_o - l_min_o
        tol = D_TOL * abs(d_o) + 1e-6 * abs(la_o) + floor
        assert abs(d_g - d_o) <= tol, (t, d_g, d_o, tol)
        if abs(d_o - tau) <= 2 * tol:
            near_ties += 1
        else:
            assert (d_o < tau) == t.accepted, (t, d_o)
        if t.accepted:
            accepted += 1
            l_min_o, l_min_g = min(l_min_o, la_o), min(l_min_g, t.la)
            removed |= set(t.candidates)
    print(f"config-1 round: {len(trials)} trials, {accepted} accepted, {len(removed)} of {P} pruned, "
          f"near ties {near_ties}, L_a {full[0, 0]:.4f} after training")
    con.close()

"""Batched candidate scoring (mg_prune_scores, Alg. 2-3 Evaluate) against one full masked render per mask (GPU).

The batched path renders the console once under a base mask and recomputes, for all masks in one pass, only
the nodes each mask changes; every score must equal, bitwise, the score of a full render under that mask (the
same kernels, parameters and work items), and the full renders match the FP64 oracle (test_gpu_parity)."""
import numpy as np
import pytest

import workloads as W
from tests.cases import make_case, gpu_console

pytestmark = pytest.mark.gpu

LOSS_TOL = 1e-5


def _masks(con, rng):
    """Brute-force singletons (one processor off, Sec. 6.2 / Sec. 7.2), dry/wet-sampling style sets of a few
    processors, every processor of one subgroup chain off, one whole song's processors off, random masks, and
    the all-ones mask."""
    P = con.n_processors
    types, _, song = con.layout()
    out = []
    for i in range(0, P, 3):
        m = np.ones(P, np.uint8)
        m[i] = 0
        out.append(m)
    for k in (2, 5, 9):
        m = np.ones(P, np.uint8)
        m[rng.choice(P, k, replace=False)] = 0
        out.append(m)
    m = np.ones(P, np.uint8)
    m[song == song.max()] = 0
    out.append(m)
    for _ in range(3):
        out.append((rng.uniform(size=P) > 0.3).astype(np.uint8))
    out.append(np.ones(P, np.uint8))
    return np.stack(out)


@pytest.mark.parametrize("retain", [1, -1])
def test_batched_scores_equal_full_renders(retain):
    import torch
    lays = [W.SongLayout(3, 1, [0, -1, 0], 30011), W.SongLayout(4, 2, [1, 0, 1, -1], 22050)]
    case = make_case(lays, seed=12)
    con = gpu_console(case, retain_spectra=retain)
    con.set_params(case.params)
    masks = _masks(con, np.random.default_rng(3))
    batched = con.prune_scores(masks).clone()
    con.set_score_mode(True)
    full = con.prune_scores(masks).clone()
    con.set_score_mode(False)
    torch.cuda.synchronize()
    assert torch.equal(batched, full), (batched - full).abs().max().item()
    # one mask per call (the base is the mask itself) and a call after an unmasked forward (its outputs reused)
    for j in (0, 4, len(masks) - 2):
        one = con.prune_scores(masks[j:j + 1])
        assert torch.equal(one[0], full[j])
    con.forward_loss()
    again = con.prune_scores(masks)
    assert torch.equal(again, full)
    # the masked losses agree with the oracle, within the parity bound plus the FP32 floor of the log-spectral
    # term (the change of the oracle's L_a when its mix moves by white noise of relative L2 1e-5): this case has
    # near-silent stretches whose log magnitudes make that floor large
    for j in (1, len(masks) - 3):
        ol, mixes = case.oracle.losses(case.params, mask=masks[j])
        for s in range(2):
            floor = la_floor(case, mixes[s], s, ol[s, 0])
            err = abs(float(full[j, s]) - ol[s, 0])
            assert err <= LOSS_TOL * ol[s, 0] + floor, (j, s, float(full[j, s]), ol[s, 0], floor)
    con.close()


def la_floor(case, mix, s, la):
    import torch
    from oracle import loss as OL
    m = torch.tensor(mix, dtype=torch.float64)
    noise = torch.tensor(np.random.default_rng(0).standard_normal(m.shape))
    noise *= 1e-5 * m.norm() / noise.norm()
    tgt = torch.tensor(case.targets[s], dtype=torch.float64)
    return abs(float(OL.audio_loss(m + noise, tgt, case.oracle.desc.loss)["a"]) - la)


def test_batched_scores_in_chunks_and_full_fallback():
    """A small workspace limit splits the masks into several chunks, and masks whose copies alone exceed it are
    rendered in full: the scores stay bitwise equal to full renders."""
    import torch
    lays = [W.SongLayout(4, 1, [0, 0, -1, -1], 20000)]
    case = make_case(lays, seed=13)
    big = gpu_console(case)
    big.set_params(case.params)
    masks = _masks(big, np.random.default_rng(4))
    big.set_score_mode(True)
    full = big.prune_scores(masks).clone()
    big.close()
    con = gpu_console(case, workspace_limit_bytes=12 << 20, retain_spectra=1)
    con.set_params(case.params)
    got = con.prune_scores(masks)
    torch.cuda.synchronize()
    assert torch.equal(got, full)
    con.close()


def test_pruned_console_scores():
    """After a structural prune the removed processors are bypassed: batched scores of masks over the remaining
    processors equal full renders."""
    import torch
    case = make_case([W.layout_plain(25000)], seed=14)
    con = gpu_console(case)
    con.set_params(case.params)
    rng = np.random.default_rng(5)
    keep = (rng.uniform(size=con.n_processors) > 0.4).astype(np.uint8)
    con.prune(keep)
    masks = _masks(con, rng)
    batched = con.prune_scores(masks).clone()
    con.set_score_mode(True)
    full = con.prune_scores(masks).clone()
    assert torch.equal(batched, full)
    con.close()


def test_consecutive_calls_start_from_the_last_candidates():
    """A call whose base mask equals, song by song, the previous call's base or one of its masks starts from that
    mask's recomputed outputs instead of rendering (the search rounds do this after every accepted trial).  Every
    score still equals a full render bitwise, also after a call whose base matches nothing before it and after an
    unmasked forward in between."""
    import torch
    lays = [W.SongLayout(3, 1, [0, -1, 0], 25011), W.SongLayout(2, 1, [0, 0], 19999)]
    case = make_case(lays, seed=15)
    con = gpu_console(case)
    ref = gpu_console(case)
    for c in (con, ref):
        c.set_params(case.params)
    ref.set_score_mode(True)
    P = con.n_processors
    _, _, song = con.layout()
    rng = np.random.default_rng(6)

    def singles(base, idx):
        out = np.repeat(base[None, :], len(idx), axis=0)
        for r, i in enumerate(idx):
            out[r, i] = 0
        return out
    base = np.ones(P, np.uint8)
    seq = [singles(base, [1, 5, 9, 30])]
    base2 = seq[0][1].copy()                      # the second mask of the first call becomes the base
    base2[song == 1] = seq[0][3][song == 1]       # and song 1 takes the fourth mask's state
    seq.append(singles(base2, [2, 12, 33]))
    seq.append(singles(base2, [3, 4]))            # same base as the call before
    other = np.ones(P, np.uint8)
    other[rng.choice(P, 6, replace=False)] = 0    # matches nothing before: rendered
    seq.append(singles(other, [0, 7, 31]))
    for k, masks in enumerate(seq):
        if k == 3:
            con.forward_loss()                    # an unmasked forward in between
        got = con.prune_scores(masks)
        want = ref.prune_scores(masks)
        torch.cuda.synchronize()
        assert torch.equal(got, want), (k, (got - want).abs().max().item())
    con.close()
    ref.close()

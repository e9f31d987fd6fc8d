"""General processing graphs on the GPU (Sec. 2, Sec. 4, Alg. 1) against the FP64 graph oracle (GPU).

A graph console runs the batched schedule of Alg. 1: per step one aggregation launch (gather and aggregate) and
the step's processors in one launch per kernel (process and store), the backward pass in reverse with the adjoint
sums of nodes read by several others."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import console as OC
from oracle import graph as OG
from oracle import loss as OL
from tests.cases import make_case, console_graph, random_dag, rel_l2

pytestmark = pytest.mark.gpu

MIX_TOL, LOSS_TOL, SET_TOL, GRAD_TOL = 1e-5, 1e-5, 2e-5, 1e-3


def graph_console(ntype, track, edges, sources, target, noise, L, schedule="greedy", **cfg):
    import paper_2509_15948_gb300 as M
    g = M.Graph(ntype, track, edges, schedule=schedule)
    return M.Console([M.Song(sources.shape[0], 0, [], L)], [sources], [target], noise, M.ConsoleConfig(**cfg), graph=g)


def test_console_graph_equals_console_bitwise():
    """The console's own graph (inputs, chains, mix nodes, output) run by the graph engine computes exactly what
    the console computes: the schedule is the console's type string, the sums read their inputs in the same
    order, and every node runs the same kernels on the same data."""
    import paper_2509_15948_gb300 as M
    lay = W.SongLayout(4, 2, [1, 0, 1, -1], 30011)
    case = make_case([lay], seed=31)
    con = M.Console([M.Song(lay.num_tracks, lay.num_subgroups, lay.track_group, lay.num_samples)], case.sources,
                    case.targets, case.noise, M.ConsoleConfig())
    ntype, track, edges = console_graph(lay)
    gcon = graph_console(ntype, track, edges, case.sources[0], case.targets[0], case.noise, lay.num_samples)
    assert M.graph_plan(M.Graph(ntype, track, edges), M.Song(4, 0, [], lay.num_samples))["steps"] == \
        [7] + list(range(7)) + [8] + list(range(7)) + [9]
    for c in (con, gcon):
        c.set_params(case.params)
        c.set_alpha_p(1e-3)
    l1, m1 = con.forward_loss(with_mix=True)
    con.backward()
    l2, m2 = gcon.forward_loss(with_mix=True)
    gcon.backward()
    assert torch.equal(m1[0], m2[0]) and torch.equal(l1, l2)
    assert torch.equal(con.get_grads(), gcon.get_grads())
    for _ in range(2):
        a = con.train_step(1e-2).clone()
        b = gcon.train_step(1e-2).clone()
        assert torch.equal(a, b)
    assert torch.equal(con.get_params(), gcon.get_params())
    con.close()
    gcon.close()


def _oracle_case(ntype, track, edges, n_tracks, L, seed):
    """Sources, a target rendered by the graph oracle from a seeded ground truth (a third of the processors kept),
    reverb noises and initial parameters for a graph."""
    src = W.song_sources(W.SongLayout(n_tracks, 0, [-1] * n_tracks, L), (seed, 0))
    ptypes = ["ecnsgdr"[t] for t in ntype if t < 7]
    noise = W.reverb_noise((seed,), max(1, ptypes.count("r")))
    desc = OC.ConsoleDesc(loss=OL.LossDesc())
    gt, keep = W.ground_truth(ptypes, (seed, 77))
    tgt = OG.GraphOracle(ntype, track, edges, src, None, noise, L, desc).render(gt, keep)
    oracle = OG.GraphOracle(ntype, track, edges, src, tgt, noise, L, desc)
    params = W.init_params(ptypes, (seed, 5))
    return src, tgt, noise, oracle, params, ptypes


def _la_floor(oracle, mix, la):
    m = torch.tensor(np.asarray(mix, np.float64))
    noise = torch.tensor(np.random.default_rng(0).standard_normal(m.shape))
    noise *= 1e-5 * m.norm() / noise.norm()
    return abs(float(OL.audio_loss(m + noise, oracle.target, oracle.desc.loss)["a"]) - la)


@pytest.mark.parametrize("seed", [1, 2, 4, 5])
def test_random_graph_matches_oracle(seed):
    """A seeded random DAG (3 inputs, 14 processors of every type, 2 mix nodes, nodes with up to three inputs
    and several outputs read): mix, losses and gradients against the FP64 graph oracle.  Seed 1's ground truth
    keeps no stereo processor, so its target is exactly mono: the target's side channel is the 1e-8 magnitude
    floor of Eq. (21), which FP32 roundoff of the packed transform (the side spectrum formed as X_L - X_R) reaches,
    so L_s, and L_a and the total that contain it, and the gradients, which carry dL_s, are not compared there
    (as for mono consoles); the mix, L_lr, L_m, L_g and L_p still are."""
    ntype, track, edges = random_dag(3, 14, 2, seed)
    L = 30011
    src, tgt, noise, oracle, params, ptypes = _oracle_case(ntype, track, edges, 3, L, seed)
    ol, og, omix = oracle.loss_and_grad(params, alpha_p=1e-3)
    con = graph_console(ntype, track, edges, src, tgt, noise, L)
    con.set_alpha_p(1e-3)
    con.set_params(params)
    losses, mixes = con.forward_loss(with_mix=True)
    con.backward()
    gl = losses.cpu().numpy()[0]
    gg = con.get_grads().cpu().numpy()
    assert rel_l2(mixes[0].cpu().numpy(), omix) <= MIX_TOL
    floor = _la_floor(oracle, omix, ol[0, 0])
    mono_target = np.array_equal(tgt[0], tgt[1])
    for j, name in enumerate(("La", "Llr", "Lm", "Ls")):
        if mono_target and name in ("La", "Ls"):
            continue
        tol = LOSS_TOL * abs(ol[0, j]) + floor if name == "La" else SET_TOL * abs(ol[0, j])
        assert abs(gl[j] - ol[0, j]) <= tol, (name, gl[j], ol[0, j])
    assert abs(gl[4] - ol[0, 4]) <= LOSS_TOL * sum(t in "erd" for t in ptypes)      # L_g, per LTI node
    assert abs(gl[5] - ol[0, 5]) <= LOSS_TOL * abs(ol[0, 5])                          # L_p
    if mono_target:
        con.close()
        return
    # gradients per processor type (the delay's log-magnitudes; its z entries are Eq. (19) directions, checked
    # for being unit or zero vectors plus the radius term) and the dry/wet logits
    offs = {}
    for v, t in enumerate(ntype):
        if t < 7:
            offs.setdefault("ecnsgdr"[t], []).append(oracle.offset[v])
    for t, starts in offs.items():
        n = OC.PARAM_COUNT[t]
        idx = np.concatenate([np.arange(o, o + n) for o in starts])
        if t == "d":
            blk = idx.reshape(-1, 2, 20, 22)
            lm = blk[:, :, :, 2:].ravel()
            assert rel_l2(gg[lm], og[lm]) <= GRAD_TOL, ("d log-magnitudes", rel_l2(gg[lm], og[lm]))
            continue
        assert rel_l2(gg[idx], og[idx]) <= GRAD_TOL, (t, rel_l2(gg[idx], og[idx]))
    q = np.arange(oracle.n_proc_params, oracle.n_params)
    assert rel_l2(gg[q], og[q]) <= GRAD_TOL
    con.close()


def test_graph_prune_equals_masked_and_schedules_agree():
    """Structural pruning of a graph console equals its masked forward bitwise (a removed processor passes its
    input through), and the greedy and beam schedules give bitwise the same results."""
    ntype, track, edges = random_dag(2, 10, 1, 3)
    L = 20011
    src, tgt, noise, oracle, params, _ = _oracle_case(ntype, track, edges, 2, L, 3)
    a = graph_console(ntype, track, edges, src, tgt, noise, L, schedule="greedy")
    b = graph_console(ntype, track, edges, src, tgt, noise, L, schedule="beam")
    for c in (a, b):
        c.set_params(params)
    la, ma = a.forward_loss(with_mix=True)
    a.backward()
    lb, mb = b.forward_loss(with_mix=True)
    b.backward()
    assert torch.equal(ma[0], mb[0]) and torch.equal(la, lb) and torch.equal(a.get_grads(), b.get_grads())
    keep = (np.random.default_rng(4).uniform(size=a.n_processors) > 0.4).astype(np.uint8)
    lm, mm = a.forward_loss(mask=keep, with_mix=True)
    mm = mm[0].clone()
    a.prune(keep)
    lp, mp = a.forward_loss(with_mix=True)
    assert torch.equal(mp[0], mm) and float(lp[0, 0]) == float(lm[0, 0])
    # the pruned graph against the oracle with the same processors absent
    ol, omix = oracle.forward(torch.tensor(np.asarray(params, np.float64)), present=keep)["La"], None
    assert abs(float(lp[0, 0]) - float(ol)) <= LOSS_TOL * abs(float(ol)) + _la_floor(
        oracle, oracle.forward(torch.tensor(np.asarray(params, np.float64)), present=keep)["mix"].detach().numpy(),
        float(ol))
    a.close()
    b.close()

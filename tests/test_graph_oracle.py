"""Pins of the general-graph oracle (oracle/graph.py; Sec. 2 graphs, Sec. 4) on the CPU.

The graph oracle is checked against the console oracle (itself pinned in test_oracle_pins) on the console's own
graph, against closed forms of the aggregation (a mix node and the output sum their inputs), and against the
plain definition of a topological order."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import console as OC
from oracle import graph as OG
from oracle import loss as OL
from tests.cases import console_graph

INPUT, MIX, OUTPUT = OG.INPUT, OG.MIX, OG.OUTPUT


def test_topological_order_is_the_plain_definition():
    edges = [(0, 2), (1, 2), (2, 3), (1, 3)]
    assert OG.topo_order(4, edges) == [0, 1, 2, 3]
    assert OG.topo_order(3, [(2, 0), (1, 0)]) == [1, 2, 0]
    with pytest.raises(ValueError):
        OG.topo_order(3, [(0, 1), (1, 2), (2, 0)])


def test_mix_and_output_sum_their_inputs():
    """Inputs -> one mix node -> output, and two inputs straight to the output: the mix is the plain sum of the
    sources on both channels (Eq. 3), with no processor in the graph."""
    L = 2000
    src = np.random.default_rng(0).standard_normal((3, L)).astype(np.float32)
    types = [INPUT, INPUT, INPUT, MIX, OUTPUT]
    edges = [(0, 3), (1, 3), (3, 4), (2, 4)]
    g = OG.GraphOracle(types, [0, 1, 2, -1, -1], edges, src, np.zeros((2, L), np.float32), None, L)
    mix = g.render(np.zeros(0), np.zeros(0))
    s = src.astype(np.float64).sum(0)
    assert np.allclose(mix, np.stack([s, s]), atol=1e-6)


def test_gain_chain_closed_form():
    """input -> g -> output with w = 1: the mix is exp(p_c) times the source on channel c (Eq. 4)."""
    L = 1000
    src = np.random.default_rng(1).standard_normal((1, L)).astype(np.float32)
    g = OG.GraphOracle([INPUT, 4, OUTPUT], [0, -1, -1], [(0, 1), (1, 2)], src, None, None, L)
    mix = g.render(np.array([0.3, -0.7, 0.0]), np.array([1.0]))   # the dry/wet logit is replaced by w
    x = src[0].astype(np.float64)
    assert np.allclose(mix[0], np.exp(0.3) * x, rtol=1e-6) and np.allclose(mix[1], np.exp(-0.7) * x, rtol=1e-6)


@pytest.mark.parametrize("layout", [W.SongLayout(3, 1, [0, -1, 0], 3001), W.SongLayout(4, 2, [1, 0, 1, -1], 2500)])
def test_console_graph_equals_console_oracle(layout):
    """The console's own graph through the graph oracle gives the console oracle's mix, losses and gradients."""
    rng = np.random.default_rng(2)
    src = W.song_sources(layout, (9, 0))
    types = W.processor_types([layout])
    noise = W.reverb_noise((9,), sum(t == "r" for t in types))
    desc = OC.ConsoleDesc(loss=OL.LossDesc(n_fft=(256, 1024)))
    spec = OC.SongSpec(layout.num_tracks, layout.num_subgroups, layout.track_group, layout.num_samples)
    tgt = rng.standard_normal((2, layout.num_samples)).astype(np.float32) * 0.1
    con = OC.Console([spec], [src], [tgt], noise, desc)
    params = W.init_params(types, (9, 1))
    lc, gc, mc = con.loss_and_grad(params, alpha_p=1e-3)
    ntype, track, edges = console_graph(layout)
    g = OG.GraphOracle(ntype, track, edges, src, tgt, noise, layout.num_samples, desc)
    assert g.n_params == len(params)
    lg, gg, mg = g.loss_and_grad(params, alpha_p=1e-3)
    assert np.allclose(mg, mc[0], rtol=1e-12, atol=1e-12)
    assert np.allclose(lg, lc, rtol=1e-12, atol=1e-12)
    assert np.allclose(gg, gc, rtol=1e-9, atol=1e-12)

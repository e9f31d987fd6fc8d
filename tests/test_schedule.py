"""Native batched-processing scheduler (Sec. 4, Alg. 1 lines 1-4) against the schedule oracle (host only, no GPU)."""
import time

import numpy as np
import pytest

import workloads as W
import paper_2509_15948_gb300 as M
from oracle import schedule as OSch
from tests.test_schedule_oracle import console_graph, as_string


def random_dag(rng, n, ntypes=3, p=0.3):
    t = [int(x) for x in rng.integers(0, ntypes, n)]
    e = [(u, v) for v in range(n) for u in range(v) if rng.random() < p]
    return t, e


def test_greedy_and_beam_match_the_oracle_on_random_graphs():
    rng = np.random.default_rng(1)
    for _ in range(40):
        t, e = random_dag(rng, int(rng.integers(3, 12)), int(rng.integers(2, 5)))
        g = M.schedule_graph(t, e, "greedy")
        assert g["steps"] == OSch.greedy_schedule(t, e)
        b = M.schedule_graph(t, e, "beam", beam_width=4096)
        assert len(b["steps"]) == len(OSch.optimal_schedule(t, e))
        assert M.schedule_graph(t, e, "beam", beam_width=1)["steps"] == g["steps"]
        for s in (g, b):
            parts = [[v for v in range(len(t)) if s["node_step"][v] == k] for k in range(len(s["steps"]))]
            assert OSch.is_valid_partition(t, e, parts)
            assert [set(p) for p in parts] == [set(q) for q in OSch.subsets(t, e, s["steps"])]


def test_beam_finds_the_shorter_schedule_greedy_misses():
    t = [0, 1, 0, 1, 1, 1, 1, 1]
    e = [(0, 1), (1, 2)]
    assert M.schedule_graph(t, e, "greedy")["steps"] == [1, 0, 1, 0]
    assert M.schedule_graph(t, e, "beam", beam_width=8)["steps"] == [0, 1, 0]


@pytest.mark.parametrize("groups,types,expect", [([0, 0, -1, -1], "ecnsgdr", "iecnsgdrmecnsgdro"),
                                                 ([-1, -1, -1], "ecnsgdr", "iecnsgdro"),
                                                 ([0, 1, 1, -1], "egr", "iegrmegro")])
def test_console_graphs_get_the_canonical_type_string(groups, types, expect):
    t, e = console_graph(groups, types)
    for method in ("greedy", "beam"):
        assert as_string(M.schedule_graph(t, e, method)["steps"]) == expect


def test_order_slices_and_gather_lists():
    rng = np.random.default_rng(4)
    t, e = random_dag(rng, 14, 3, 0.25)
    s = M.schedule_graph(t, e, "beam", beam_width=64)
    order, pos = s["order"], np.argsort(s["order"])
    # every subset is the contiguous slice step_begin[k] .. step_begin[k+1] of the new order
    for k in range(len(s["steps"])):
        members = order[s["step_begin"][k]:s["step_begin"][k + 1]]
        assert all(s["node_step"][v] == k for v in members)
        assert list(members) == sorted(members)
    # the gather lists are the edges in new positions, grouped by the consumer's step
    got = sorted(zip(s["gather_src"].tolist(), s["gather_dst"].tolist()))
    assert got == sorted((int(pos[u]), int(pos[v])) for u, v in e)
    for k in range(len(s["steps"])):
        for i in range(s["gather_begin"][k], s["gather_begin"][k + 1]):
            assert s["node_step"][order[s["gather_dst"][i]]] == k
            assert s["node_step"][order[s["gather_src"][i]]] < k


def test_cycles_and_bad_edges_are_refused():
    with pytest.raises(M.MgError):
        M.schedule_graph([0, 0], [(0, 1), (1, 0)])
    with pytest.raises(M.MgError):
        M.schedule_graph([0, 0], [(0, 5)])


def test_a_64_song_console_graph_schedules_fast():
    t, e, off = [], [], 0
    for lay in W.layout_uneven_batch(64, seed=2):
        tt, ee = console_graph(list(lay.track_group))
        t += tt
        e += [(u + off, v + off) for u, v in ee]
        off += len(tt)
    t0 = time.perf_counter()
    s = M.schedule_graph(t, e, "greedy")
    assert time.perf_counter() - t0 < 5.0
    assert as_string(s["steps"]) == "iecnsgdrmecnsgdro" and len(t) > 10000

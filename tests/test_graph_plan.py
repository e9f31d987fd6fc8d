"""Host planning of graph consoles through the C ABI (mg_graph_plan; no GPU): the schedule of the console's own
graph is the console's type string (Sec. 4.2), the footprint covers the console's, and invalid graphs are refused."""
import pytest

import workloads as W
from tests.cases import console_graph, random_dag


def _M():
    M = pytest.importorskip("paper_2509_15948_gb300")
    try:
        M.load_library()
    except RuntimeError as e:
        pytest.skip(str(e))
    return M


def test_console_graph_schedule_and_footprint():
    M = _M()
    lay = W.SongLayout(4, 2, [1, 0, 1, -1], 30011)
    nt, tr, ed = console_graph(lay)
    plan = M.graph_plan(M.Graph(nt, tr, ed), M.Song(4, 0, [], lay.num_samples))
    assert plan["steps"] == [7] + list(range(7)) + [8] + list(range(7)) + [9]      # i e..r m e..r o
    ref = M.plan([M.Song(4, 2, [1, 0, 1, -1], lay.num_samples)])
    assert plan["n_processors"] == ref["n_processors"] == 42 and plan["n_params"] == ref["n_params"]
    assert plan["device_bytes"] >= ref["device_bytes"]       # plus a source per track and per-node adjoints
    beam = M.graph_plan(M.Graph(nt, tr, ed, schedule="beam"), M.Song(4, 0, [], lay.num_samples))
    assert len(beam["steps"]) <= len(plan["steps"])


def test_random_graph_plans():
    M = _M()
    nt, tr, ed = random_dag(3, 14, 2, 1)
    plan = M.graph_plan(M.Graph(nt, tr, ed), M.Song(3, 0, [], 10000))
    assert plan["n_processors"] == 14 and plan["steps"][0] == 7 and plan["steps"][-1] == 9


@pytest.mark.parametrize("types,tracks,edges,why", [
    ([7, 4, 9, 9], [0, -1, -1, -1], [(0, 1), (1, 2), (1, 3)], "exactly one output"),
    ([7, 4, 4, 9], [0, -1, -1, -1], [(0, 1), (1, 2), (2, 1), (2, 3)], "cycle"),
    ([7, 7, 9], [0, 0, -1], [(0, 1), (1, 2)], "input node with a predecessor"),
    ([7, 4, 9], [0, -1, -1], [(0, 2)], "without a predecessor"),
    ([7, 9, 4], [0, -1, -1], [(0, 1), (1, 2)], "output node with a successor"),
    ([7, 4, 9], [5, -1, -1], [(0, 1), (1, 2)], "valid track"),
    ([7, 4, 9], [0, -1, -1], [(0, 1), (1, 1), (1, 2)], "out of range"),
    ([7, 12, 9], [0, -1, -1], [(0, 1), (1, 2)], "type out of range"),
])
def test_invalid_graphs_are_refused(types, tracks, edges, why):
    M = _M()
    with pytest.raises(M.MgError) as e:
        M.graph_plan(M.Graph(types, tracks, edges), M.Song(1, 0, [], 1000))
    assert e.value.status == M.MG_ERR_INVALID and why in str(e.value)

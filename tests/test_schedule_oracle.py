"""Pins of the schedule oracle (Sec. 4): console graphs reach the type string the paper states as optimal,
a hand-built graph where the greedy choice is suboptimal, validity of every produced partition."""
import numpy as np

from oracle import schedule as OSch

CODES = {c: k for k, c in enumerate("iecnsgdrmo")}


def console_graph(track_group, types="ecnsgdr"):
    """Console DAG (Sec. 4.3): per track an input node and the chain; per subgroup a mix node and the chain;
    the output node sums subgroup chains and ungrouped tracks."""
    t, e = [], []

    def node(c):
        t.append(CODES[c])
        return len(t) - 1

    def chain(src):
        for c in types:
            v = node(c)
            e.append((src, v))
            src = v
        return src

    nsub = max(track_group) + 1 if any(g >= 0 for g in track_group) else 0
    mixes = [node("m") for _ in range(nsub)]
    out = node("o")
    for g in track_group:
        end = chain(node("i"))
        e.append((end, mixes[g] if g >= 0 else out))
    for m in mixes:
        e.append((chain(m), out))
    return t, e


def as_string(seq):
    inv = {v: k for k, v in CODES.items()}
    return "".join(inv[x] for x in seq)


def test_console_optimum_is_the_canonical_type_string():
    t, e = console_graph([0, 0, -1, -1])
    assert as_string(OSch.optimal_schedule(t, e)) == "iecnsgdrmecnsgdro"
    t, e = console_graph([-1, -1, -1])
    assert as_string(OSch.optimal_schedule(t, e)) == "iecnsgdro"
    t, e = console_graph([0, 1, 1, -1], types="egr")
    assert as_string(OSch.optimal_schedule(t, e)) == "iegrmegro"


def test_greedy_can_be_suboptimal():
    # types a = 0, b = 1: a chain a -> b -> a next to five independent b nodes
    t = [0, 1, 0, 1, 1, 1, 1, 1]
    e = [(0, 1), (1, 2)]
    assert OSch.optimal_schedule(t, e) == [0, 1, 0]
    assert OSch.greedy_schedule(t, e) == [1, 0, 1, 0]


def test_schedules_are_valid_partitions():
    rng = np.random.default_rng(0)
    for _ in range(20):
        n = int(rng.integers(4, 11))
        t = [int(x) for x in rng.integers(0, 3, n)]
        e = [(u, v) for v in range(n) for u in range(v) if rng.random() < 0.3]
        for seq in (OSch.optimal_schedule(t, e), OSch.greedy_schedule(t, e)):
            parts = OSch.subsets(t, e, seq)
            assert OSch.is_valid_partition(t, e, [sorted(p) for p in parts])
        assert len(OSch.optimal_schedule(t, e)) <= len(OSch.greedy_schedule(t, e))
    # a non-causal partition is rejected
    assert not OSch.is_valid_partition([0, 0], [(0, 1)], [[1], [0]])

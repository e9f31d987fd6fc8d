"""Node subset sequences for batched graph processing (Sec. 4, Alg. 1): the plain definitions (oracle; test
infrastructure).

A schedule is a sequence of types t_0 .. t_N; step n takes the maximal subset V_n of not yet computed nodes
of type t_n whose predecessors are all computed (Sec. 4.2: with the type fixed, the subset is made as large
as possible).  It is valid when the subsets partition V, are causal and homogeneous (Sec. 4.1).  The optimum
is the shortest such sequence, found here by breadth-first search over the sets of computed nodes (exact,
exponential: small graphs only).  Greedy: the type with the most computable nodes at every step (ties to the
smaller type code).
"""
from __future__ import annotations

from collections import deque
from typing import Dict, List, Sequence, Tuple


def preds_of(n: int, edges: Sequence[Tuple[int, int]]) -> List[List[int]]:
    preds = [[] for _ in range(n)]
    for u, v in edges:
        preds[v].append(u)
    return preds


def ready_subset(types: Sequence[int], preds: List[List[int]], done: frozenset, t: int) -> frozenset:
    """Maximal subset of type t computable after `done`."""
    return frozenset(v for v in range(len(types))
                     if v not in done and types[v] == t and all(u in done for u in preds[v]))


def optimal_schedule(types: Sequence[int], edges: Sequence[Tuple[int, int]]) -> List[int]:
    """Shortest type sequence covering every node (breadth-first over computed-node sets)."""
    n = len(types)
    preds = preds_of(n, edges)
    start = frozenset()
    parent: Dict[frozenset, Tuple[frozenset, int]] = {start: (None, -1)}
    q = deque([start])
    full = frozenset(range(n))
    while q:
        s = q.popleft()
        if s == full:
            seq = []
            while parent[s][0] is not None:
                s, t = parent[s][0], parent[s][1]
                seq.append(t)
            return seq[::-1]
        for t in sorted(set(types)):
            sub = ready_subset(types, preds, s, t)
            if sub:
                nxt = s | sub
                if nxt not in parent:
                    parent[nxt] = (s, t)
                    q.append(nxt)
    raise ValueError("graph has a cycle")


def greedy_schedule(types: Sequence[int], edges: Sequence[Tuple[int, int]]) -> List[int]:
    n = len(types)
    preds = preds_of(n, edges)
    done, seq = frozenset(), []
    while len(done) < n:
        best = max(sorted(set(types)), key=lambda t: (len(ready_subset(types, preds, done, t)), -t))
        sub = ready_subset(types, preds, done, best)
        if not sub:
            raise ValueError("graph has a cycle")
        done, seq = done | sub, seq + [best]
    return seq


def subsets(types: Sequence[int], edges: Sequence[Tuple[int, int]], seq: Sequence[int]) -> List[frozenset]:
    """The node subsets V_n a type sequence selects (raises if it does not cover the graph)."""
    preds = preds_of(len(types), edges)
    done, out = frozenset(), []
    for t in seq:
        sub = ready_subset(types, preds, done, t)
        out.append(sub)
        done = done | sub
    if len(done) != len(types):
        raise ValueError("sequence does not cover the graph")
    return out


def is_valid_partition(types, edges, parts: Sequence[Sequence[int]]) -> bool:
    """Sec. 4.1: a partition of V, causal (no path from a later or equal subset to an earlier one, checked on
    the edges), homogeneous (one type per subset)."""
    step = {}
    for k, p in enumerate(parts):
        for v in p:
            if v in step:
                return False
            step[v] = k
    if len(step) != len(types):
        return False
    if any(step[u] >= step[v] for u, v in edges):
        return False
    return all(len({types[v] for v in p}) == 1 for p in parts if p)

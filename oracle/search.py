"""Alg. 3: mixing graph search with dry/wet candidate sampling (Sec. 6.1-6.2), one pruning round
(oracle; test infrastructure).

Readings where the paper is silent (repeated in the design notes):
  * N_t is fixed at the start of the round; the candidate count is k = max(1, floor(N_t r_t + 0.5))
    capped at |V_t| (the paper's rounding can give 0, which would never terminate);
  * the least-weight nodes break ties by processor index;
  * SampleType draws from the remaining types, kept in chain order e c n s g d r, with the splitmix64
    generator (Steele, Lea, Flood 2014): index = next() mod |T_c|;
  * a type whose node set V_t has become empty leaves T_c;
  * failure with k > 1 halves r_t, failure with k = 1 removes the type (Alg. 3).
"""
from __future__ import annotations

from typing import Callable, List, Sequence, Tuple

import numpy as np

MASK64 = (1 << 64) - 1
TYPE_ORDER = "ecnsgdr"


class SplitMix64:
    """splitmix64 (Steele, Lea, Flood, OOPSLA 2014)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)


def dry_wet_round(w: Sequence[float], types: Sequence[str], present: Sequence[int], l_min: float, tau: float,
                  evaluate: Callable[[np.ndarray], float], rng: SplitMix64) -> Tuple[np.ndarray, float, List[tuple]]:
    """One pruning round of Alg. 3 over the processors with present[i] = 1.
    evaluate(mask) returns L_a of the graph with dry/wet weights w * mask.
    Returns (m, updated L_min, trace of (type, candidates, L_a, accepted))."""
    P = len(w)
    m = np.ones(P, np.uint8)
    tc = [t for t in TYPE_ORDER if any(present[i] and types[i] == t for i in range(P))]
    V = {t: [i for i in range(P) if present[i] and types[i] == t] for t in tc}
    N = {t: len(V[t]) for t in tc}
    r = {t: 0.1 for t in tc}
    trace = []
    while tc:
        t = tc[rng.next() % len(tc)]
        if not V[t]:
            tc.remove(t)
            continue
        k = min(max(1, int(np.floor(N[t] * r[t] + 0.5))), len(V[t]))
        order = sorted(V[t], key=lambda i: (w[i], i))
        cand = order[:k]
        mbar = np.ones(P, np.uint8)
        mbar[cand] = 0
        la = float(evaluate(m * mbar))
        ok = la < l_min + tau
        trace.append((t, tuple(cand), la, ok))
        if ok:
            l_min = min(l_min, la)
            m = m * mbar
            V[t] = [i for i in V[t] if i not in cand]
        else:
            if k > 1:
                r[t] = r[t] / 2.0
            else:
                tc.remove(t)
    return m, l_min, trace


def brute_force_round(present: Sequence[int], l_min: float, tau: float, evaluate: Callable[[np.ndarray], float],
                      rng: SplitMix64) -> Tuple[np.ndarray, float, List[tuple]]:
    """One pruning round with brute-force candidate sampling (Sec. 6.2, first method): every processor of
    the pool is tried alone, V_c = {v} with v drawn uniformly from the pool, until the pool is empty.
    Readings: the pool holds the present processors in ascending index order and v = pool[next() mod |pool|];
    a tried processor leaves the pool whether or not its trial succeeds (UpdatePool of Alg. 2).
    Returns (m, updated L_min, trace of (processor, L_a, accepted))."""
    P = len(present)
    m = np.ones(P, np.uint8)
    pool = [i for i in range(P) if present[i]]
    trace = []
    while pool:
        v = pool[rng.next() % len(pool)]
        cand = np.ones(P, np.uint8)
        cand[v] = 0
        la = float(evaluate(m * cand))
        ok = la < l_min + tau
        trace.append((v, la, ok))
        if ok:
            l_min = min(l_min, la)
            m = m * cand
        pool.remove(v)
    return m, l_min, trace


def uses_brute_force(iteration: int, every: int = 4) -> bool:
    """Hybrid sampling (Sec. 6.2): brute force on every 4th pruning iteration (1-based), dry/wet otherwise."""
    return iteration % every == 0


def node_deltas(la_full: float, evaluate: Callable[[np.ndarray], float], present: Sequence[int]) -> np.ndarray:
    """Delta_i = L_a(G minus v_i) - L_a(G) for every present processor (Sec. 7.2); NaN for absent ones."""
    P = len(present)
    out = np.full(P, np.nan)
    for i in range(P):
        if present[i]:
            m = np.ones(P, np.uint8)
            m[i] = 0
            out[i] = float(evaluate(m)) - la_full
    return out

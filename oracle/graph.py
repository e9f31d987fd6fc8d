"""General processing graphs (Sec. 2, Sec. 4), FP64 (oracle; test infrastructure).

A graph G = (V, E) has input nodes i (one dry source each, on both channels), processor nodes of the types
e c n s g d r (Sec. 3), mix nodes m and one output node o.  Every node's input is the sum of its predecessors'
outputs (Eq. 3's aggregation); an input node outputs its source, a mix node its input, a processor node the dry/wet
blend of Eq. (2b) of its processed input, and the output node's input is the rendered mix y_hat.  The nodes are
evaluated one at a time in a topological order (ascending index among the ready ones); the batched schedule of
Alg. 1 only reorders this work.  The objective is the console's: Eqs. (20)-(23), (26) for the one song.

Parameter layout: the processor nodes in ascending node index, each with its parameters, followed by one dry/wet
logit per processor node in the same order; reverb noises indexed by the rank of the reverb among the reverbs.
Absent processors (structural pruning) pass their input through and are left out of L_g and L_p.
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

import numpy as np
import torch

from . import processors as P
from .console import ConsoleDesc, PARAM_COUNT, TYPE_ORDER
from .loss import audio_loss, gain_staging

F64 = torch.float64
INPUT, MIX, OUTPUT = 7, 8, 9          # node type codes after the processor types 0..6 ("ecnsgdr")


def topo_order(n: int, edges: Sequence[Tuple[int, int]]) -> List[int]:
    """Kahn's algorithm taking the smallest ready index first; raises on a cycle."""
    indeg = [0] * n
    succ = [[] for _ in range(n)]
    for u, v in edges:
        succ[u].append(v)
        indeg[v] += 1
    ready = sorted(v for v in range(n) if indeg[v] == 0)
    order = []
    while ready:
        v = ready.pop(0)
        order.append(v)
        for w in succ[v]:
            indeg[w] -= 1
            if indeg[w] == 0:
                ready.append(w)
        ready.sort()
    if len(order) != n:
        raise ValueError("graph has a cycle")
    return order


class GraphOracle:
    def __init__(self, node_type: Sequence[int], input_index: Sequence[int], edges: Sequence[Tuple[int, int]],
                 sources: np.ndarray, target: Optional[np.ndarray], reverb_noise: Optional[np.ndarray],
                 num_samples: int, desc: ConsoleDesc = ConsoleDesc()):
        self.n = len(node_type)
        self.type = list(node_type)
        self.input_index = list(input_index)
        self.edges = [tuple(e) for e in edges]
        self.L = num_samples
        self.desc = desc
        self.preds = [[] for _ in range(self.n)]
        for u, v in self.edges:
            self.preds[v].append(u)
        self.order = topo_order(self.n, self.edges)
        outs = [v for v in range(self.n) if self.type[v] == OUTPUT]
        if len(outs) != 1:
            raise ValueError("exactly one output node")
        self.out = outs[0]
        # processors in node order, their parameter offsets and reverb ranks
        self.procs = [v for v in range(self.n) if self.type[v] < 7]
        self.offset, off, self.rev = {}, 0, {}
        for v in self.procs:
            self.offset[v] = off
            off += PARAM_COUNT[TYPE_ORDER[self.type[v]]]
            if TYPE_ORDER[self.type[v]] == "r":
                self.rev[v] = len(self.rev)
        self.n_proc_params = off
        self.n_params = off + len(self.procs)
        self.sources = torch.tensor(np.asarray(sources, np.float32), dtype=F64)
        self.target = torch.tensor(np.asarray(target, np.float32), dtype=F64) if target is not None else None
        self.fir_len = int(round(2 * desc.sample_rate))
        self.D = P.delay_slot(desc.sample_rate)
        self.noise_spec = [P.reverb_noise_stft(torch.tensor(np.asarray(reverb_noise[i], np.float32), dtype=F64))
                           for i in range(len(self.rev))] if self.rev else []

    def _process(self, v: int, u: torch.Tensor, pbar: torch.Tensor) -> torch.Tensor:
        t = TYPE_ORDER[self.type[v]]
        if t == "g":
            return P.gain_pan(u, pbar)
        if t == "s":
            return P.stereo_imager(u, pbar)
        if t == "e":
            return P.equalizer(u, pbar)
        if t == "r":
            return P.reverb(u, pbar, self.noise_spec[self.rev[v]], self.fir_len)
        if t == "c":
            return P.dynamics(u, pbar, gate=False)
        if t == "n":
            return P.dynamics(u, pbar, gate=True)
        return P.multitap_delay(u, pbar, self.D)

    def forward(self, params: torch.Tensor, mask=None, present=None, alpha_p: float = 0.0) -> dict:
        """Render and evaluate the objective.  mask / present: optional {0,1} per processor (in processor order)."""
        q = params[self.n_proc_params:]
        w = torch.sigmoid(q)
        if mask is not None:
            w = w * torch.as_tensor(np.asarray(mask, np.float64), dtype=F64)
        pidx = {v: i for i, v in enumerate(self.procs)}
        outs = {}
        lg = torch.zeros((), dtype=F64)
        lp = torch.zeros((), dtype=F64)
        mix = None
        for v in self.order:
            u = torch.zeros(2, self.L, dtype=F64)
            for p in self.preds[v]:
                u = u + outs[p]
            t = self.type[v]
            if t == INPUT:
                x = self.sources[self.input_index[v]]
                outs[v] = torch.stack([x, x])
            elif t == MIX:
                outs[v] = u
            elif t == OUTPUT:
                mix = u
            else:
                i = pidx[v]
                if present is not None and not present[i]:
                    outs[v] = u
                    continue
                off = self.offset[v]
                ybar = self._process(v, u, params[off: off + PARAM_COUNT[TYPE_ORDER[t]]])
                if TYPE_ORDER[t] in "erd":
                    lg = lg + gain_staging(ybar, u)
                outs[v] = P.dry_wet(u, ybar, w[i])
                lp = lp + w[i]
        if self.target is None:                      # rendering only
            return {"mix": mix}
        la = audio_loss(mix, self.target, self.desc.loss)
        total = la["a"] + self.desc.alpha_g * lg + alpha_p * lp
        return {"mix": mix, "La": la["a"], "Llr": la["lr"], "Lm": la["m"], "Ls": la["s"], "Lg": lg, "Lp": lp,
                "total": total}

    def loss_and_grad(self, params: np.ndarray, mask=None, present=None, alpha_p: float = 0.0):
        """Losses [1, 7] (La, Llr, Lm, Ls, Lg, Lp, total), d total / d params, and the mix."""
        x = torch.tensor(np.asarray(params, np.float64), dtype=F64, requires_grad=True)
        r = self.forward(x, mask, present, alpha_p)
        r["total"].backward()
        losses = np.array([[float(r[k].detach()) for k in ("La", "Llr", "Lm", "Ls", "Lg", "Lp", "total")]])
        return losses, x.grad.detach().numpy().copy(), r["mix"].detach().numpy()

    def render(self, params: np.ndarray, w: np.ndarray) -> np.ndarray:
        """Mix with explicit dry/wet weights w (ground-truth rendering), float32."""
        x = torch.tensor(np.asarray(params, np.float64), dtype=F64)
        x[self.n_proc_params:] = float("inf")
        target, self.target = self.target, None
        try:
            with torch.no_grad():
                mix = self.forward(x, mask=np.asarray(w, np.float64))["mix"]
        finally:
            self.target = target
        return mix.numpy().astype(np.float32)

"""FP64 CPU oracle of the differentiable mixing console (test infrastructure only).

This package is a plain, slow, obviously-correct restatement of the paper's
equations in double precision with PyTorch CPU ops.  Gradients come from
autograd (exact up to rounding), except for the multitap delay's angular
frequencies, whose gradient the paper defines by a straight-through rule with
sign normalisation and a radius regulariser (Sec. 3.7); that rule is written
out explicitly in `processors.DelayScatter`.

It is test infrastructure: only `tests/`, `__graft_entry__.smoke()` and the
CPU-baseline leg of `bench.py` may import it.  It shares no code with the CUDA
path and imports nothing from it.

Modules
-------
processors  Sec. 3 processors (g, s, e, r, c, n, d) and the dry/wet blend (Eq. 1)
loss        Sec. 5.1 multi-resolution STFT loss and the gain-staging regulariser
console     Sec. 1.2/4 mixing console (chains, subgroups, mix) and its objective (Sec. 6.3)
adam        Adam (Sec. 5.1)
search      Alg. 3 (dry/wet candidate sampling) driven by a scoring callback
"""
from . import processors, loss, console, adam, search  # noqa: F401

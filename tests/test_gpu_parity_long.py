"""CUDA path vs the FP64 oracle at the sizes the throughput benchmark runs (GPU).

* Single-track consoles of the multitap delay and the reverb (Sec. 3.4, 3.7) at lengths that reach each of the
  FFT size classes of the uneven 64-song batch (N = 3 2^17, 2^19, 5 2^17, 3 2^18, 2^20, 5 2^18, 3 2^19) and at
  the largest sizes of the factors 5 and 3 (57 s: N = 5 2^19, 60 s: N = 3 2^20, rows at the row kernels' limits
  of 2560 and 3072 points), with the row/column split the autotuner picks and with the default split.
* A batch of ten copies of a 4-track, 30 s song with every processor type, whose arena passes 4 GiB, so that
  the node buffers of the later songs sit at byte offsets beyond 2^32: every copy against the oracle's song.
* Sampled songs of the benchmark's own console (64 songs, 1,143 tracks, 1,053 s of audio, autotuned splits,
  retained spectra, one CUDA-graph replay of forward + loss + backward + Adam), each against the oracle run
  on that song alone; the targets of the sampled songs are rendered by the oracle.

Tolerances as in test_gpu_parity: relative L2 1e-5 on mixes and losses, 1e-3 on gradients."""
import gc
import importlib.util
import os

import numpy as np
import pytest

import workloads as W
from oracle import console as OC
from oracle import loss as OL
from tests.cases import Case, make_case, gpu_console, oracle_with_delay_taps, rel_l2
from tests.test_gpu_parity import check, check_results

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FS = 44100
# (seconds, f, log2 N / f): the size classes of the uneven batch's reverb and delay convolutions
# (N = f 2^k, f = 1, 3, 5, the smallest that holds the linear convolution)
SIZE_CLASSES = [(6.5, 3, 17), (9.5, 1, 19), (11.0, 5, 17), (15.0, 3, 18), (20.0, 1, 20), (25.0, 5, 18),
                (30.0, 3, 19)]
# the largest transforms of each factor: rows of 5 2^9 = 2560 and 3 2^10 = 3072 points (the row kernels' limits)
MAX_CLASSES = [(57.0, 5, 19), (60.0, 3, 20)]


def _free_device():
    import torch
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def _song_slices(con, s):
    """Processor indices and parameter indices (processor parameters, then dry/wet logits) of song s."""
    types, offs, song = con.layout()
    procs = np.nonzero(song == s)[0]
    pidx = np.concatenate([np.arange(offs[i], offs[i] + OC.PARAM_COUNT["ecnsgdr"[types[i]]]) for i in procs] +
                          [con.n_proc_params + procs])
    return procs, pidx


@pytest.mark.parametrize("seconds,f,logn", SIZE_CLASSES + MAX_CLASSES)
def test_reverb_and_delay_at_benchmark_fft_sizes(seconds, f, logn):
    _free_device()
    L = int(seconds * FS)
    case = make_case([W.SongLayout(1, 0, [-1], L)], types="dr", seed=40 + int(seconds))
    con, _, _ = check(case, autotune=1)
    sz = con.fft_sizes()
    assert all(int(r[0]) == f and int(r[1]) == logn for r in sz), sz
    con.close()


@pytest.mark.parametrize("seconds,f,logn", [c for c in SIZE_CLASSES if c[0] >= 20])
def test_reverb_and_delay_long_default_split(seconds, f, logn):
    _free_device()
    L = int(seconds * FS)
    case = make_case([W.SongLayout(1, 0, [-1], L)], types="dr", seed=50 + int(seconds))
    con, _, _ = check(case, autotune=0)
    assert all(int(r[0]) == f and int(r[1]) == logn for r in con.fft_sizes())
    con.close()


def test_batch_with_arena_past_4gib():
    """Ten copies of one 4-track, 30 s song (tracks 0-1 in a subgroup), every processor type.  The arena holds
    at least every processor's output, the three adjoint / input buffers of every chain, the equalizers' kept
    wet signals and the dynamics' dL/dg: more than 2^32 bytes, so the later songs' nodes sit past 4 GiB.  Every
    copy must match the oracle's song, and the copies must agree bitwise with each other."""
    import torch
    _free_device()
    copies, L = 10, 30 * FS
    single = make_case([W.layout_plain(L)], seed=61)
    ol, og, omix, taps = oracle_with_delay_taps(single, 1e-3)
    lay = single.layouts[0]
    P1 = len(single.ptypes)
    ld = -(-L // 64) * 64
    arena_lb = copies * (P1 * 2 * ld * 4 + 5 * 3 * 2 * ld * 4 + 5 * (2 * ld * 4 + 2 * ld * 4))
    assert arena_lb > 2 ** 32, arena_lb
    npp = single.oracle.n_proc_params
    params = np.concatenate([single.params[:npp]] * copies + [single.params[npp:]] * copies)
    songs = [OC.SongSpec(lay.num_tracks, lay.num_subgroups, lay.track_group, lay.num_samples)] * copies
    batch = Case([lay] * copies, single.types, single.sources * copies, single.targets * copies,
                 np.concatenate([single.noise] * copies), single.ptypes * copies, params, single.n_fft,
                 single.n_mels, OC.Console(songs, single.sources * copies, single.targets * copies,
                                           np.concatenate([single.noise] * copies),
                                           OC.ConsoleDesc(types=single.types, loss=OL.LossDesc())))
    con = gpu_console(batch)
    con.set_alpha_p(1e-3)
    con.set_params(params)
    losses, mixes = con.forward_loss(with_mix=True)
    con.backward()
    g = con.get_grads().cpu().numpy()
    gl = losses.cpu().numpy()
    gm = [m.cpu().numpy() for m in mixes]
    for s in range(copies):
        procs_s, pidx = _song_slices(con, s)
        check_results(single, (ol, og, omix, taps), (gl[s:s + 1], g[pidx], [gm[s]]), con, alpha_p=1e-3,
                      proc_map=procs_s)
        assert np.array_equal(gm[s], gm[0]) and np.array_equal(gl[s], gl[0]) and np.array_equal(g[pidx],
                                                                                                 g[_song_slices(con, 0)[1]])
    con.close()
    del con
    _free_device()


def _bench():
    spec = importlib.util.spec_from_file_location("bench_for_parity", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


# the smallest and the shortest songs of the batch, a mid-sized one, and the last one (31 tracks, 19.3 s),
# whose nodes are the last ones in the arena
SAMPLED_SONGS = (21, 62, 6, 63)


def test_benchmark_batch_sampled_songs():
    """The uneven 64-song batch built as the benchmark builds it (same sources, reverb noises, initial
    parameters, alpha_p, autotuned splits, retained spectra), stepped by the benchmark's CUDA graph: the losses
    and gradients of the sampled songs against the oracle, and their mixes from a forward of the same
    parameters.  The sampled songs' targets are ground-truth mixes rendered by the oracle; every other song's
    target is its plain sum of sources (on the host), which the sampled songs do not depend on."""
    import torch
    import paper_2509_15948_gb300 as M
    _free_device()
    b = _bench()
    layouts = W.layout_uneven_batch(64, seed=2)
    bank = b.source_bank(key=0)
    sources = [b.song_sources_from_bank(bank, l, s) for s, l in enumerate(layouts)]
    types = W.processor_types(layouts)
    noise = W.reverb_noise((0, 9), sum(t == "r" for t in types))
    gt, keep = W.ground_truth(types, (0, 77))
    p0 = W.init_params(types, (0, 5))
    alpha_p = 1e-4
    procs, npp, P = OC.layout([OC.SongSpec(l.num_tracks, l.num_subgroups, l.track_group, l.num_samples)
                               for l in layouts])
    targets = [np.stack([s.sum(0), s.sum(0)]).astype(np.float32) for s in sources]
    singles = {}
    for s in SAMPLED_SONGS:
        lay = layouts[s]
        sel = [p for p in procs if p.song == s]
        pidx = np.concatenate([np.arange(p.offset, p.offset + p.count) for p in sel] + [npp + np.array([p.index for p in sel])])
        revs = [p.rev for p in sel if p.type == "r"]
        spec = OC.SongSpec(lay.num_tracks, lay.num_subgroups, lay.track_group, lay.num_samples)
        nz = noise[revs]
        gts = gt[pidx].copy()
        tgt = OC.Console([spec], [sources[s]], None, nz).render_targets(gts, keep[[p.index for p in sel]])[0]
        targets[s] = tgt
        oc = OC.Console([spec], [sources[s]], [tgt], nz)
        single = Case([lay], "ecnsgdr", [sources[s]], [tgt], nz, [p.type for p in sel], p0[pidx].copy(),
                      (512, 2048, 8192), 96, oc)
        singles[s] = (single, oracle_with_delay_taps(single, alpha_p), pidx, [p.index for p in sel])
    con = M.Console([M.Song(l.num_tracks, l.num_subgroups, l.track_group, l.num_samples) for l in layouts], sources,
                    targets, noise, M.ConsoleConfig(autotune=1))
    assert con.get_info()["retains_spectra"] == 1
    con.set_params(p0)
    con.set_alpha_p(alpha_p)
    losses_g = con.train_step(lr=1e-2).clone()          # the benchmark's graph: losses and gradients at p0
    g = con.get_grads().cpu().numpy()
    gl = losses_g.cpu().numpy()
    con.set_params(p0)
    losses_f, mixes = con.forward_loss(with_mix=True)
    assert torch.equal(losses_f, losses_g)
    for s in SAMPLED_SONGS:
        single, ores, pidx, pmap = singles[s]
        check_results(single, ores, (gl[s:s + 1], g[pidx], [mixes[s].cpu().numpy()]), con, alpha_p=alpha_p,
                      proc_map=pmap)
    con.close()
    del con
    _free_device()

"""The allocation-free equalizer entry point (mg_eq_forward_noalloc) against the console's own equalizer.

This entry point exists for callers that cannot allocate device memory (code under another framework's
allocator, plug-in hosts that forbid device allocations on their processing threads, work being recorded on
a stream).  Its output must equal what the console computes for a one-track console whose only processor is
the equalizer, on two calls in a row (the second call reuses the shared scratch array left by the first).
The file is named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5   # relative L2, the bound the console's mixes are held to
MAX_L = 2 ** 17 - 2047 - 1023 - 1   # 128,001: the 2^17-point FFT holds the signal and the 2047-tap FIR


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_equalizer_matches_console_twice():
    """Two calls in a row with different lengths (the largest accepted L, a 2^17-point FFT, then a short one
    with a 2^12-point FFT), so that the second call reuses a scratch array left holding another size's data;
    each output is compared with the console's equalizer on the same input and parameters."""
    import torch
    import paper_2509_15948_gb300 as M
    lib = M.load_library()
    lib.mg_eq_forward_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                          ctypes.c_void_p]
    lib.mg_eq_forward_noalloc.restype = ctypes.c_int
    stream = torch.cuda.Stream()
    rng = np.random.default_rng(0)
    for call, L in enumerate((MAX_L, 3001)):
        src = W.song_sources(W.SongLayout(1, 0, [-1], L), (42, call))
        tgt = np.zeros((2, L), np.float32)
        con = M.Console([M.Song(1, 0, [-1], L)], [src], [tgt], None, M.ConsoleConfig(types="e"))
        u = torch.as_tensor(np.stack([src[0], src[0]])).cuda().contiguous()
        params = np.concatenate([rng.uniform(-1.0, 1.0, 1024), [rng.normal()]]).astype(np.float32)
        con.set_params(params)
        _, mixes = con.forward_loss(with_mix=True)
        ref = mixes[0].cpu().numpy()
        p = torch.as_tensor(params).cuda()
        y = torch.full_like(u, float("nan"))
        torch.cuda.synchronize()
        st = lib.mg_eq_forward_noalloc(u.data_ptr(), y.data_ptr(), L, p.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
        assert st == M.MG_OK
        stream.synchronize()
        assert _rel(y.cpu().numpy(), ref) <= TOL, (call, L, _rel(y.cpu().numpy(), ref))
        con.close()
    # one sample beyond the scratch bound is refused before any GPU work
    big = torch.zeros(2, MAX_L + 1, device="cuda")
    assert lib.mg_eq_forward_noalloc(big.data_ptr(), big.data_ptr(), MAX_L + 1, p.data_ptr(),
                                     ctypes.c_void_p(stream.cuda_stream)) == M.MG_ERR_UNSUPPORTED

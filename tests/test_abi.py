"""The C ABI library loads, exports every function include/mixgraph.h declares, and plans layouts on the
host (CPU only: no compute call needs a GPU here)."""
import ctypes
import os
import re

import pytest

import workloads as W
from oracle import console as OC

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2509_15948_gb300 import build as B
    B.build()
    import paper_2509_15948_gb300 as M
    return M.load_library()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "mixgraph.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mg_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 25
    for n in names:
        assert hasattr(lib, n), n


def test_plan_matches_oracle_layout():
    import paper_2509_15948_gb300 as M
    lays = W.layout_uneven_batch(5, seed=9)
    info = M.plan([M.Song(l.num_tracks, l.num_subgroups, l.track_group, l.num_samples) for l in lays])
    procs, npp, P = OC.layout([OC.SongSpec(l.num_tracks, l.num_subgroups, l.track_group, l.num_samples) for l in lays])
    assert info["n_processors"] == P and info["n_proc_params"] == npp and info["n_params"] == npp + P
    assert info["n_reverbs"] == sum(p.type == "r" for p in procs)
    assert abs(info["track_seconds"] - sum(l.num_tracks * l.num_samples for l in lays) / 44100.0) < 1e-9


def test_plan_type_mask_and_validation():
    import paper_2509_15948_gb300 as M
    s = [M.Song(4, 1, [0, 0, -1, -1], 10000)]
    info = M.plan(s, M.ConsoleConfig(types="gs"))
    assert info["n_processors"] == 10 and info["n_proc_params"] == 5 * 3
    with pytest.raises(M.MgError):
        M.plan([M.Song(2, 1, [0, 3], 1000)])            # subgroup index out of range
    with pytest.raises(M.MgError):
        M.plan(s, M.ConsoleConfig(n_fft=(500,)))         # FFT size not a power of two
    # the loss adjoint keeps bands x 4 channels of every frame of a work item (8192 samples) in shared
    # memory: 512 Mel bands over 128 frames of 64 points do not fit, 96 bands do
    with pytest.raises(M.MgError):
        M.plan(s, M.ConsoleConfig(n_fft=(64,), n_mels=512))
    assert M.plan(s, M.ConsoleConfig(n_fft=(512,), n_mels=96))["n_processors"] > 0


def test_console_needs_a_gpu_and_fails_loudly():
    import torch
    import paper_2509_15948_gb300 as M
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(RuntimeError):
        M.Console([M.Song(1, 0, [-1], 1000)], [W.song_sources(W.SongLayout(1, 0, [-1], 1000), (0,))], None)

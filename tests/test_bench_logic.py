"""Host logic of bench.py, no GPU: the byte model, the kernel-source fingerprint of the roofline traffic, and
the reference arm's JSON line (the FP64 oracle timed on the host cores)."""
import importlib.util
import json
import os
import subprocess
import sys

import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("K,S", [(4, 1), (16, 4), (32, 8)])
def test_model_bytes_closed_form_for_grouped_songs(K, S):
    # every track in a subgroup, all seven types: 5 streams x 7 types per chain (K + S chains), 2 per track input
    # and 2 per subgroup input of the sums, 2 per subgroup output, 2 for the master output, 2 for the loss:
    # 37 K + 39 S + 4 stereo FP32 streams per sample
    b = _bench()
    L = 1000
    groups = [k % S for k in range(K)]
    lay = W.SongLayout(K, S, groups, L)
    tot, per_type = b.model_bytes([lay])
    assert tot == (37 * K + 39 * S + 4) * L * 8
    assert all(v == 5 * (K + S) * L * 8 for v in per_type.values())


def test_model_bytes_ungrouped_tracks_and_type_subset():
    b = _bench()
    L = 500
    lay = W.SongLayout(3, 1, [0, 0, -1], L)   # two tracks in the subgroup, one straight to the master
    tot, per_type = b.model_bytes([lay], types="gs")
    chains = 4
    streams = 5 * 2 * chains + 2 * 2 + 2 * 1 + 2 * (1 + 1) + 2 + 2
    assert tot == streams * L * 8
    assert per_type["g"] == per_type["s"] == 5 * chains * L * 8 and per_type["e"] == 0


def test_kernel_source_fingerprint_is_stable_and_covers_existing_files():
    b = _bench()
    h1, h2 = b.kernel_src_sha1(), b.kernel_src_sha1()
    assert h1 == h2 and len(h1) == 40 and int(h1, 16) >= 0
    for name in b.KERNEL_SRCS:
        assert os.path.exists(os.path.join(ROOT, "paper_2509_15948_gb300", "csrc", name)), name
    assert b.KERNEL_BYTES_PER_POINT["row_bwd2"] == 40


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["warmup"] == 3                      # at least three warm-up steps, whatever was asked
    assert d["value"] > 0 and d["unit"] == "track-s/s" and d["higher_is_better"] is True
    assert d["dtype"] == "f64" and d["data"] == "synthetic" and "workload" in d["config"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]


def test_model_flops_counts_ffts_per_stage():
    """The flop model counts 2.5 n log2 n per real FFT of size n: 12 per reverb / delay node at the linear-
    convolution length, 8 per 6146-sample equalizer block plus 4 per node, 4 per loss frame and resolution."""
    import math
    b = _bench()
    L = 100_000
    lay = W.SongLayout(2, 1, [0, 0], L)
    f = b.model_flops([lay], fs=44100, n_fft=(512,), hop_div=4)
    rf = lambda n: 2.5 * n * math.log2(n)
    chains = 3
    assert f["r"] == pytest.approx(chains * (12 * rf(L + 88200 - 1) + 4 * 458 * rf(384)), rel=1e-12)
    assert f["d"] == pytest.approx(chains * 12 * rf(L + 20 * 4410 + 38 - 1), rel=1e-12)
    assert f["e"] == pytest.approx(chains * (8 * math.ceil(L / 6146) + 4) * rf(8192), rel=1e-12)
    frames = (L - 512) // 128 + 1
    assert f["loss"] == pytest.approx(4 * frames * rf(512), rel=1e-12)
    # warm-up drops the frames that start before it
    fw = b.model_flops([lay], fs=44100, n_fft=(512,), hop_div=4, warmup=1000)
    assert fw["loss"] == pytest.approx(4 * (frames - math.ceil(1000 / 128)) * rf(512), rel=1e-12)
    assert b.fp32_peak_tflops(2070.0) == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)

"""Python binding of the GB300 mixing-console library (include/mixgraph.h).

Argument marshalling only: every step of the forward pass, loss, backward pass, pruning scores and Adam
runs in the CUDA kernels of libmixgraph.so.  PyTorch supplies device memory and streams.  There is no CPU
fallback: importing works without a GPU (for layout planning), but every compute call needs the built
library and a CUDA device, and fails loudly otherwise.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libmixgraph.so")
TYPE_ORDER = "ecnsgdr"
LOSS_FIELDS = ("La", "Llr", "Lm", "Ls", "Lg", "Lp", "total")

MG_OK, MG_ERR_INVALID, MG_ERR_OOM, MG_ERR_CUDA, MG_ERR_STATE, MG_ERR_TIMEOUT, MG_ERR_UNSUPPORTED = range(7)
_STATUS = {0: "MG_OK", 1: "MG_ERR_INVALID", 2: "MG_ERR_OOM", 3: "MG_ERR_CUDA", 4: "MG_ERR_STATE",
           5: "MG_ERR_TIMEOUT", 6: "MG_ERR_UNSUPPORTED"}


class MgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class SongDesc(ctypes.Structure):
    _fields_ = [("num_tracks", ctypes.c_int32), ("num_subgroups", ctypes.c_int32),
                ("track_group", ctypes.POINTER(ctypes.c_int32)), ("num_samples", ctypes.c_int64),
                ("sources", ctypes.c_void_p), ("target", ctypes.c_void_p), ("on_device", ctypes.c_int32)]


class ConsoleDesc(ctypes.Structure):
    _fields_ = [("sample_rate", ctypes.c_double), ("type_mask", ctypes.c_uint32), ("n_resolutions", ctypes.c_int32),
                ("n_fft", ctypes.c_int32 * 3), ("hop_div", ctypes.c_int32), ("n_mels", ctypes.c_int32),
                ("a_weighting", ctypes.c_int32), ("warmup_samples", ctypes.c_int64), ("alpha_lr", ctypes.c_float),
                ("alpha_m", ctypes.c_float), ("alpha_s", ctypes.c_float), ("alpha_g", ctypes.c_float),
                ("reverb_noise", ctypes.c_void_p), ("noise_on_device", ctypes.c_int32),
                ("workspace_limit_bytes", ctypes.c_int64), ("retain_spectra", ctypes.c_int32),
                ("autotune", ctypes.c_int32)]


class GraphDesc(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int32), ("node_type", ctypes.POINTER(ctypes.c_int32)),
                ("input_track", ctypes.POINTER(ctypes.c_int32)), ("n_edges", ctypes.c_int32),
                ("edge_src", ctypes.POINTER(ctypes.c_int32)), ("edge_dst", ctypes.POINTER(ctypes.c_int32)),
                ("schedule", ctypes.c_int32), ("beam_width", ctypes.c_int32)]


NODE_INPUT, NODE_MIX, NODE_OUTPUT = 7, 8, 9


@dataclasses.dataclass
class Graph:
    """A processing graph of one song (Sec. 2): node types (0..6 processor types "ecnsgdr", NODE_INPUT, NODE_MIX,
    NODE_OUTPUT), the source track of every input node (-1 elsewhere), edges (src, dst), and the schedule of
    Alg. 1 ("greedy" or "beam")."""
    node_type: Sequence[int]
    input_track: Sequence[int]
    edges: Sequence[tuple]
    schedule: str = "greedy"
    beam_width: int = 8

    def desc(self):
        n, m = len(self.node_type), len(self.edges)
        keep = [(ctypes.c_int32 * max(1, n))(*[int(t) for t in self.node_type]),
                (ctypes.c_int32 * max(1, n))(*[int(t) for t in self.input_track]),
                (ctypes.c_int32 * max(1, m))(*[int(e[0]) for e in self.edges]),
                (ctypes.c_int32 * max(1, m))(*[int(e[1]) for e in self.edges])]
        d = GraphDesc(n, keep[0], keep[1], m, keep[2], keep[3], {"greedy": 0, "beam": 1}[self.schedule],
                      int(self.beam_width))
        return d, keep


class ConsoleInfo(ctypes.Structure):
    _fields_ = [("n_songs", ctypes.c_int32), ("n_processors", ctypes.c_int32), ("n_proc_params", ctypes.c_int64),
                ("n_params", ctypes.c_int64), ("n_reverbs", ctypes.c_int32), ("total_samples", ctypes.c_int64),
                ("track_seconds", ctypes.c_double), ("device_bytes", ctypes.c_int64),
                ("launches_per_step", ctypes.c_int32), ("retains_spectra", ctypes.c_int32)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Loads libmixgraph.so (built in-tree by build.py); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2509_15948_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, I32, I64, F32, U8P = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_void_p
    sig = {
        "mg_plan": [ctypes.POINTER(ConsoleDesc), ctypes.POINTER(SongDesc), I32, ctypes.POINTER(ConsoleInfo)],
        "mg_schedule_graph": [P, I32, P, P, I32, I32, I32, P, P, P, P],
        "mg_evaluate": [P, P],
        "mg_processor_fft": [P, P, P, P],
        "mg_schedule_io": [P, P, I32, I32, P, P, I32, P, P, P, P],
        "mg_console_create": [ctypes.POINTER(ConsoleDesc), ctypes.POINTER(SongDesc), I32, P, ctypes.POINTER(P)],
        "mg_console_destroy": [P],
        "mg_console_get_info": [P, ctypes.POINTER(ConsoleInfo)],
        "mg_processor_layout": [P, P, P, P],
        "mg_set_params": [P, P, I64, I32],
        "mg_get_params": [P, P, I64, I32],
        "mg_get_grads": [P, P, I64, I32],
        "mg_set_alpha_p": [P, F32],
        "mg_forward_loss": [P, U8P, P, P],
        "mg_backward": [P],
        "mg_prune_scores": [P, U8P, I32, P],
        "mg_adam_step": [P, F32, F32, F32, F32, F32],
        "mg_reset_optimizer": [P],
        "mg_train_step": [P, F32, F32, F32, F32, F32, P],
        "mg_prune": [P, U8P],
        "mg_get_present": [P, U8P],
        "mg_update_audio": [P, I32, P, P, I32],
        "mg_set_launch_mode": [P, I32],
        "mg_set_score_mode": [P, I32],
        "mg_debug_chain_hold": [P, I32],
        "mg_set_profiling": [P, I32],
        "mg_get_kernel_times": [P, P, P, I32],
        "mg_reset_kernel_times": [P],
        "mg_debug_read": [P, I32, I32, P, I64],
        "mg_get_stage_times": [P, P, P, I32],
        "mg_graph_plan": [ctypes.POINTER(ConsoleDesc), ctypes.POINTER(GraphDesc), ctypes.POINTER(SongDesc),
                          ctypes.POINTER(ConsoleInfo), P, P],
        "mg_graph_console_create": [ctypes.POINTER(ConsoleDesc), ctypes.POINTER(GraphDesc), ctypes.POINTER(SongDesc),
                                    P, ctypes.POINTER(P)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.mg_last_error.argtypes = [P]
    lib.mg_last_error.restype = ctypes.c_char_p
    lib.mg_num_kernel_families.argtypes = []
    lib.mg_num_kernel_families.restype = ctypes.c_int32
    lib.mg_kernel_family_name.argtypes = [I32]
    lib.mg_kernel_family_name.restype = ctypes.c_char_p
    _lib = lib
    return lib


@dataclasses.dataclass
class ConsoleConfig:
    sample_rate: float = 44100.0
    types: str = TYPE_ORDER
    n_fft: Sequence[int] = (512, 2048, 8192)
    hop_div: int = 4
    n_mels: int = 96
    a_weighting: bool = True
    warmup_samples: int = 0
    alpha_lr: float = 0.5
    alpha_m: float = 0.25
    alpha_s: float = 0.25
    alpha_g: float = 1e-3
    workspace_limit_bytes: int = 0
    retain_spectra: int = 0   # 1 keep, -1 recompute, 0 automatic (see mg_console_desc)
    autotune: int = 0         # 1: time the FFT convolution splits at creation and keep the fastest

    def type_mask(self) -> int:
        return sum(1 << i for i, t in enumerate(TYPE_ORDER) if t in self.types)


@dataclasses.dataclass
class Song:
    num_tracks: int
    num_subgroups: int
    track_group: List[int]
    num_samples: int


def _desc(cfg: ConsoleConfig, noise_ptr: int = 0, noise_on_device: int = 0) -> ConsoleDesc:
    d = ConsoleDesc()
    d.sample_rate = cfg.sample_rate
    d.type_mask = cfg.type_mask()
    d.n_resolutions = len(cfg.n_fft)
    for i, n in enumerate(cfg.n_fft):
        d.n_fft[i] = int(n)
    d.hop_div = cfg.hop_div
    d.n_mels = cfg.n_mels
    d.a_weighting = int(cfg.a_weighting)
    d.warmup_samples = cfg.warmup_samples
    d.alpha_lr, d.alpha_m, d.alpha_s, d.alpha_g = cfg.alpha_lr, cfg.alpha_m, cfg.alpha_s, cfg.alpha_g
    d.reverb_noise = noise_ptr
    d.noise_on_device = noise_on_device
    d.workspace_limit_bytes = cfg.workspace_limit_bytes
    d.retain_spectra = cfg.retain_spectra
    d.autotune = cfg.autotune
    return d


def _song_array(songs: Sequence[Song], src_ptrs=None, tgt_ptrs=None, on_device=0):
    arr = (SongDesc * len(songs))()
    keep = []
    for i, s in enumerate(songs):
        groups = list(s.track_group) if s.track_group else [-1] * s.num_tracks
        tg = (ctypes.c_int32 * s.num_tracks)(*[int(g) for g in groups])
        keep.append(tg)
        arr[i].num_tracks = s.num_tracks
        arr[i].num_subgroups = s.num_subgroups
        arr[i].track_group = tg
        arr[i].num_samples = s.num_samples
        arr[i].sources = src_ptrs[i] if src_ptrs else None
        arr[i].target = tgt_ptrs[i] if tgt_ptrs else None
        arr[i].on_device = on_device
    return arr, keep


def schedule_graph(types: Sequence[int], edges: Sequence[tuple], method: str = "greedy", beam_width: int = 8) -> dict:
    """Batched-processing schedule of a general graph (Sec. 4) through the C ABI (host only): the type sequence,
    each node's step, the node order with contiguous subsets, and the per-step store slices and gather lists."""
    lib = load_library()
    n, m = len(types), len(edges)
    t = np.ascontiguousarray(types, np.int32)
    es = np.ascontiguousarray([e[0] for e in edges], np.int32)
    ed = np.ascontiguousarray([e[1] for e in edges], np.int32)
    step_type = np.zeros(max(1, n), np.int32)
    node_step = np.zeros(max(1, n), np.int32)
    order = np.zeros(max(1, n), np.int32)
    nsteps = ctypes.c_int32()
    meth = {"greedy": 0, "beam": 1}[method]
    st = lib.mg_schedule_graph(t.ctypes.data, n, es.ctypes.data, ed.ctypes.data, m, meth, beam_width,
                               step_type.ctypes.data, ctypes.byref(nsteps), node_step.ctypes.data, order.ctypes.data)
    if st != MG_OK:
        raise MgError(st, "mg_schedule_graph failed (bad arguments or a cycle)")
    k = nsteps.value
    step_begin = np.zeros(k + 1, np.int32)
    gather_begin = np.zeros(k + 1, np.int32)
    gsrc = np.zeros(max(1, m), np.int32)
    gdst = np.zeros(max(1, m), np.int32)
    st = lib.mg_schedule_io(node_step.ctypes.data, order.ctypes.data, n, k, es.ctypes.data, ed.ctypes.data, m,
                            step_begin.ctypes.data, gather_begin.ctypes.data, gsrc.ctypes.data, gdst.ctypes.data)
    if st != MG_OK:
        raise MgError(st, "mg_schedule_io failed")
    return {"steps": step_type[:k].tolist(), "node_step": node_step[:n], "order": order[:n],
            "step_begin": step_begin, "gather_begin": gather_begin, "gather_src": gsrc[:m], "gather_dst": gdst[:m]}


def plan(songs: Sequence[Song], cfg: ConsoleConfig = ConsoleConfig()) -> dict:
    """Host-only layout planning through the C ABI (no GPU needed)."""
    lib = load_library()
    arr, _keep = _song_array(songs)
    info = ConsoleInfo()
    st = lib.mg_plan(ctypes.byref(_desc(cfg)), arr, len(songs), ctypes.byref(info))
    if st != MG_OK:
        raise MgError(st, lib.mg_last_error(None).decode())
    return {f: getattr(info, f) for f, _ in ConsoleInfo._fields_}


def graph_plan(graph: Graph, song: Song, cfg: ConsoleConfig = ConsoleConfig()) -> dict:
    """Host-only planning of a graph console (no GPU): sizes as plan() and the schedule's type sequence."""
    lib = load_library()
    arr, _keep = _song_array([song])
    gd, _gkeep = graph.desc()
    info = ConsoleInfo()
    steps = np.zeros(max(1, len(graph.node_type)), np.int32)
    n = ctypes.c_int32()
    st = lib.mg_graph_plan(ctypes.byref(_desc(cfg)), ctypes.byref(gd), arr, ctypes.byref(info), steps.ctypes.data,
                           ctypes.byref(n))
    if st != MG_OK:
        raise MgError(st, lib.mg_last_error(None).decode())
    out = {f: getattr(info, f) for f, _ in ConsoleInfo._fields_}
    out["steps"] = steps[:n.value].tolist()
    return out


class Console:
    """A batch of songs on one GPU.  sources: per song float32 [K][L] (numpy or torch); targets: [2][L];
    reverb_noise: float32 [n_reverbs][2][2 fs] (required when reverbs are enabled).  With graph (a Graph), the
    console is the general processing graph of one song (songs holds that one Song; its subgroups are ignored)."""

    def __init__(self, songs: Sequence[Song], sources, targets, reverb_noise=None, cfg: ConsoleConfig = ConsoleConfig(),
                 device: Optional[int] = None, stream=None, graph: Optional[Graph] = None):
        import torch
        self.torch = torch
        if not torch.cuda.is_available():
            raise RuntimeError("paper_2509_15948_gb300.Console needs a CUDA device (no CPU fallback)")
        self.lib = load_library()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        # a dedicated non-default stream: CUDA graphs cannot be captured on the legacy default stream
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        self.songs = list(songs)
        self.cfg = cfg
        dev = self.device
        src_t = [torch.as_tensor(np.asarray(s, np.float32) if not isinstance(s, torch.Tensor) else s,
                                 dtype=torch.float32).to(dev).contiguous() for s in sources]
        tgt_t = [torch.as_tensor(np.asarray(t, np.float32) if not isinstance(t, torch.Tensor) else t,
                                 dtype=torch.float32).to(dev).contiguous() for t in targets] if targets is not None else None
        for s, x in zip(self.songs, src_t):
            assert tuple(x.shape) == (s.num_tracks, s.num_samples), "sources must be [K][L]"
        noise_ptr = 0
        noise_t = None
        if reverb_noise is not None:
            noise_t = torch.as_tensor(np.asarray(reverb_noise, np.float32) if not isinstance(reverb_noise, torch.Tensor)
                                      else reverb_noise, dtype=torch.float32).to(dev).contiguous()
            noise_ptr = noise_t.data_ptr()
        arr, keep = _song_array(self.songs, [x.data_ptr() for x in src_t],
                                [x.data_ptr() for x in tgt_t] if tgt_t else None, on_device=1)
        # the copies above ran on the caller's stream; a stream (not device) synchronisation, so that a graph
        # being captured by another console on another thread is not disturbed
        torch.cuda.current_stream(dev).synchronize()
        h = ctypes.c_void_p()
        if graph is not None:
            assert len(self.songs) == 1, "a graph console holds one song"
            gd, self._graph_keep = graph.desc()
            st = self.lib.mg_graph_console_create(ctypes.byref(_desc(cfg, noise_ptr, 1)), ctypes.byref(gd), arr,
                                                  ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        else:
            st = self.lib.mg_console_create(ctypes.byref(_desc(cfg, noise_ptr, 1)), arr, len(self.songs),
                                            ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if st != MG_OK:
            raise MgError(st, self.lib.mg_last_error(None).decode())
        self.h = h
        info = ConsoleInfo()
        self.lib.mg_console_get_info(self.h, ctypes.byref(info))
        self.info = {f: getattr(info, f) for f, _ in ConsoleInfo._fields_}
        self.n_params = info.n_params
        self.n_processors = info.n_processors
        self.n_proc_params = info.n_proc_params
        self.n_songs = info.n_songs
        self._losses = torch.zeros(self.n_songs, 7, dtype=torch.float32, device=dev)

    # --------------------------------------------------------------------------------------------
    def _check(self, st):
        # the caller's stream waits for the console's stream, so tensors returned here are ready in order
        self.torch.cuda.current_stream(self.device).wait_stream(self.stream)
        if st != MG_OK:
            raise MgError(st, self.lib.mg_last_error(self.h).decode())

    def _enter(self):
        self.stream.wait_stream(self.torch.cuda.current_stream(self.device))

    def close(self):
        if getattr(self, "h", None):
            self.lib.mg_console_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_info(self) -> dict:
        info = ConsoleInfo()
        self._check(self.lib.mg_console_get_info(self.h, ctypes.byref(info)))
        return {f: getattr(info, f) for f, _ in ConsoleInfo._fields_}

    def layout(self):
        types = np.zeros(self.n_processors, np.int32)
        offs = np.zeros(self.n_processors, np.int64)
        song = np.zeros(self.n_processors, np.int32)
        self._check(self.lib.mg_processor_layout(self.h, types.ctypes.data, offs.ctypes.data, song.ctypes.data))
        return types, offs, song

    def fft_sizes(self) -> np.ndarray:
        """[P, 3]: f, log2 of N / f and log2 of N1 / f of every processor's FFT convolution (zeros elsewhere)."""
        out = np.zeros((3, self.n_processors), np.int32)
        self._check(self.lib.mg_processor_fft(self.h, out[0].ctypes.data, out[1].ctypes.data, out[2].ctypes.data))
        return out.T.copy()

    def processor_types(self) -> List[str]:
        return [TYPE_ORDER[t] for t in self.layout()[0]]

    def set_params(self, params):
        torch = self.torch
        self._enter()
        p = torch.as_tensor(np.asarray(params, np.float32) if not isinstance(params, torch.Tensor) else params,
                            dtype=torch.float32).to(self.device).contiguous()
        assert p.numel() == self.n_params
        self._keep_params = p
        self._check(self.lib.mg_set_params(self.h, p.data_ptr(), self.n_params, 1))

    def get_params(self):
        self._enter()
        out = self.torch.empty(self.n_params, dtype=self.torch.float32, device=self.device)
        self._check(self.lib.mg_get_params(self.h, out.data_ptr(), self.n_params, 1))
        return out

    def get_grads(self):
        self._enter()
        out = self.torch.empty(self.n_params, dtype=self.torch.float32, device=self.device)
        self._check(self.lib.mg_get_grads(self.h, out.data_ptr(), self.n_params, 1))
        return out

    def set_alpha_p(self, alpha_p: float):
        self._check(self.lib.mg_set_alpha_p(self.h, float(alpha_p)))

    def forward_loss(self, mask=None, with_mix: bool = False):
        """Losses [n_songs, 7] (La, Llr, Lm, Ls, Lg, Lp, total) on the device; optionally the mixes."""
        torch = self.torch
        mptr = None
        if mask is not None:
            m = torch.as_tensor(np.asarray(mask, np.uint8) if not isinstance(mask, torch.Tensor) else mask,
                                dtype=torch.uint8).to(self.device).contiguous()
            self._keep_mask = m
            mptr = m.data_ptr()
        mix = None
        if with_mix:
            mix = torch.empty(sum(2 * s.num_samples for s in self.songs), dtype=torch.float32, device=self.device)
        losses = torch.empty(self.n_songs, 7, dtype=torch.float32, device=self.device)
        self._enter()
        self._check(self.lib.mg_forward_loss(self.h, mptr, losses.data_ptr(), mix.data_ptr() if mix is not None else None))
        if with_mix:
            out, o = [], 0
            for s in self.songs:
                out.append(mix[o:o + 2 * s.num_samples].view(2, s.num_samples))
                o += 2 * s.num_samples
            return losses, out
        return losses

    def backward(self):
        self._enter()
        self._check(self.lib.mg_backward(self.h))

    def prune_scores(self, masks):
        torch = self.torch
        m = torch.as_tensor(np.asarray(masks, np.uint8) if not isinstance(masks, torch.Tensor) else masks,
                            dtype=torch.uint8).to(self.device).contiguous()
        assert m.dim() == 2 and m.shape[1] == self.n_processors
        out = torch.empty(m.shape[0], self.n_songs, dtype=torch.float32, device=self.device)
        self._enter()
        self._check(self.lib.mg_prune_scores(self.h, m.data_ptr(), m.shape[0], out.data_ptr()))
        return out

    def adam_step(self, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0):
        self._enter()
        self._check(self.lib.mg_adam_step(self.h, lr, beta1, beta2, eps, weight_decay))

    def reset_optimizer(self):
        self._check(self.lib.mg_reset_optimizer(self.h))

    def train_step(self, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0):
        """forward_loss + backward + adam_step replayed as one CUDA graph; returns the losses (device)."""
        self._enter()
        self._check(self.lib.mg_train_step(self.h, lr, beta1, beta2, eps, weight_decay, self._losses.data_ptr()))
        return self._losses

    def prune(self, keep):
        k = np.ascontiguousarray(np.asarray(keep, np.uint8))
        assert k.shape == (self.n_processors,)
        self._check(self.lib.mg_prune(self.h, k.ctypes.data))

    def present(self) -> np.ndarray:
        out = np.zeros(self.n_processors, np.uint8)
        self._check(self.lib.mg_get_present(self.h, out.ctypes.data))
        return out

    def update_audio(self, song: int, sources, target=None):
        torch = self.torch
        s = torch.as_tensor(sources, dtype=torch.float32).to(self.device).contiguous()
        t = torch.as_tensor(target, dtype=torch.float32).to(self.device).contiguous() if target is not None else None
        self._enter()
        self._check(self.lib.mg_update_audio(self.h, song, s.data_ptr(), t.data_ptr() if t is not None else None, 1))
        self.torch.cuda.current_stream(self.device).synchronize()

    def update_audio_host(self, song: int, sources: np.ndarray, target: Optional[np.ndarray] = None):
        """Same as update_audio from host buffers (pinned or pageable)."""
        s = sources if isinstance(sources, np.ndarray) else sources.numpy()
        t = target if (target is None or isinstance(target, np.ndarray)) else target.numpy()
        s = np.ascontiguousarray(s, np.float32)
        t = np.ascontiguousarray(t, np.float32) if t is not None else None
        self._check(self.lib.mg_update_audio(self.h, song, s.ctypes.data, t.ctypes.data if t is not None else None, 0))

    def evaluate(self):
        """[n_songs, 6] on the device: SI-SDR (dB) and the MIR feature distances d_rms, d_cf, d_sw, d_si, d_bs
        (Eq. 27) of the mix of the most recent forward against the target."""
        out = self.torch.empty(self.n_songs, 6, dtype=self.torch.float32, device=self.device)
        self._enter()
        self._check(self.lib.mg_evaluate(self.h, out.data_ptr()))
        return out

    def set_launch_mode(self, per_node: bool):
        self._check(self.lib.mg_set_launch_mode(self.h, int(per_node)))

    def debug_chain_hold(self, on: bool):
        """Test hook: the first chunk of every envelope-scan launch withholds its state (see mixgraph.h)."""
        self._check(self.lib.mg_debug_chain_hold(self.h, int(on)))

    def set_score_mode(self, full_renders: bool):
        """prune_scores: False batches the masks over one base render (default); True renders every mask in full."""
        self._check(self.lib.mg_set_score_mode(self.h, int(full_renders)))

    def set_profiling(self, on: bool):
        self._check(self.lib.mg_set_profiling(self.h, int(on)))

    def kernel_times(self) -> dict:
        n = self.lib.mg_num_kernel_families()
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int64 * n)()
        self._check(self.lib.mg_get_kernel_times(self.h, ms, cnt, n))
        return {self.lib.mg_kernel_family_name(i).decode(): (ms[i], cnt[i]) for i in range(n)}

    def debug_read(self, proc: int, what: int, shape) -> np.ndarray:
        """Host copy of one processor buffer: 0 y, 1 taps, 2 tap gradient, 3 du, 4 stats."""
        out = np.zeros(shape, np.float32)
        self._check(self.lib.mg_debug_read(self.h, proc, what, out.ctypes.data, out.size))
        return out

    STAGES = ("e", "c", "n", "s", "g", "d", "r", "loss", "sum", "other")

    def stage_times(self) -> dict:
        """Accumulated milliseconds and launches per console stage (processor types, loss, sums, other)."""
        ms = (ctypes.c_double * 10)()
        cnt = (ctypes.c_int64 * 10)()
        self._check(self.lib.mg_get_stage_times(self.h, ms, cnt, 10))
        return {name: (ms[i], cnt[i]) for i, name in enumerate(self.STAGES)}

    def reset_kernel_times(self):
        self._check(self.lib.mg_reset_kernel_times(self.h))


def _console_loss_function():
    import torch

    class ConsoleLoss(torch.autograd.Function):
        """torch.autograd.Function over the C ABI: forward = mg_forward_loss, backward = mg_backward.
        Input: parameter tensor [n_params] (CUDA); output: per-song total loss [n_songs]."""

        @staticmethod
        def forward(ctx, params, console: Console):
            console.set_params(params.detach())
            losses = console.forward_loss()
            ctx.console = console
            return losses[:, 6].clone()

        @staticmethod
        def backward(ctx, grad_out):
            con = ctx.console
            con.backward()
            g = con.get_grads()
            if not torch.all(grad_out == 1):
                types, offs, song = con.layout()
                cnt = np.diff(np.append(offs, con.n_proc_params))
                per_param_song = np.repeat(song, cnt)
                idx = torch.as_tensor(np.concatenate([per_param_song, song]), device=g.device, dtype=torch.long)
                scale = grad_out[idx]
                g = g * scale
            return g, None

    return ConsoleLoss


def console_loss(params, console: Console):
    """Differentiable per-song total loss of the console at `params` (see ConsoleLoss)."""
    return _console_loss_function().apply(params, console)

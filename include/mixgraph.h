/*
 * mixgraph.h - C ABI of the GB300 mixing-console hot path.
 *
 * Reverse engineering of a music mix (Sec. 1.1): given dry sources S = [s_1..s_K] and a target mix y,
 * find the graph G and parameters P with y_hat = G(S; P) close to y under the loss L_a.  This library
 * holds the hot path of that search: the batched forward and backward pass of the differentiable mixing
 * console G_c (Sec. 1.2, Sec. 3, Sec. 4), its multi-resolution STFT loss and regularisers (Sec. 5.1,
 * Sec. 6.3), Adam (Sec. 5.1), masked forwards that score pruning candidates (Alg. 2-3), and structural
 * pruning (Alg. 3, Prune).
 *
 * Conventions (all entry points):
 *  - Every call is stream-ordered on the stream given to mg_console_create and returns without waiting
 *    for the GPU unless stated.  Device pointers passed by the caller are borrowed for the duration of
 *    the enqueued work only when the call says "copied"; otherwise they must stay valid until the
 *    stream reaches the call.
 *  - The library owns all device memory it allocates; the caller owns what it passes in.
 *  - No C++ exception crosses the ABI.  Failures return a status; mg_last_error(console) gives a message
 *    (valid until the next call on that console); mg_last_error(NULL) is per host thread.
 *  - Threads: different consoles may be driven from different host threads at the same time (one thread
 *    per console at a time).  Console creation, destruction, pruning and the capture of a console's
 *    training-step graph are serialised inside the library; callers that share the device must not
 *    synchronise the whole device (cudaDeviceSynchronize) while other threads' consoles may be capturing.
 *  - Processor order P ("canonical"): song -> chain (tracks 0..K-1, then subgroups 0..S-1) -> type in
 *    chain order e c n s g d r (enabled types only).  The flat parameter vector holds every processor's
 *    parameters in that order (g 2, s 1, e 1024, r 768, c 4, n 4, d 880; Sec. 3), followed by one
 *    dry/wet logit q per processor in the same order; w = sigmoid(q) * mask (Sec. 5.1, Alg. 3).
 *  - Audio is FP32, sample rate as given; stereo buffers are planar [2][L] (left row, then right row).
 */
#ifndef MIXGRAPH_H
#define MIXGRAPH_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MG_OK = 0,
  MG_ERR_INVALID = 1,     /* bad argument (null pointer, size mismatch, out-of-range value) */
  MG_ERR_OOM = 2,         /* device allocation failed */
  MG_ERR_CUDA = 3,        /* a CUDA runtime call failed */
  MG_ERR_STATE = 4,       /* call out of order (e.g. backward without a preceding unmasked forward_loss) */
  MG_ERR_TIMEOUT = 5,     /* a bounded wait gave up */
  MG_ERR_UNSUPPORTED = 6  /* configuration outside the supported range */
} mg_status;

typedef struct mg_console mg_console;

/* One song (Sec. 1.1 problem statement): K mono dry sources, a subgroup assignment (given a priori,
 * Sec. 1.2) and the target stereo mix. */
typedef struct {
  int32_t num_tracks;          /* K >= 1 */
  int32_t num_subgroups;       /* S >= 0 */
  const int32_t* track_group;  /* host [K]: subgroup of each track in [0, S), or -1 = straight to the mix */
  int64_t num_samples;         /* L >= 1 */
  const float* sources;        /* [K][L] mono sources (input node i duplicates each to both channels); copied */
  const float* target;         /* [2][L] target mix y, or NULL (then the losses are not defined); copied */
  int32_t on_device;           /* 1: sources/target are device pointers, 0: host pointers */
} mg_song_desc;

/* Console and loss settings (Sec. 3, Sec. 5.1, Sec. 6.3). */
typedef struct {
  double sample_rate;          /* fs in Hz (e.g. 44100) */
  uint32_t type_mask;          /* bit i enables processor type "ecnsgdr"[i] in every chain (0x7F = all) */
  int32_t n_resolutions;       /* 1..3 STFT resolutions of Eq. (21) */
  int32_t n_fft[3];            /* FFT sizes, powers of two in [64, 8192] (e.g. 512, 2048, 8192) */
  int32_t hop_div;             /* hop = n_fft / hop_div (4 in Sec. 5.1) */
  int32_t n_mels;              /* Mel bands (96 in Sec. 5.1); 0 = linear-frequency bins.  Per resolution,
                                  bands (n_fft / 2 + 1 when linear) x 8192 / n_fft x 4 must be at most 40192
                                  (the loss adjoint's per-item buffer), else MG_ERR_INVALID */
  int32_t a_weighting;         /* 1 = A-weighting before the STFT (Sec. 5.1) */
  int64_t warmup_samples;      /* frames starting before this sample are left out of the loss */
  float alpha_lr, alpha_m, alpha_s;  /* Eq. (20) weights (0.5, 0.25, 0.25) */
  float alpha_g;               /* Eq. (23) gain-staging weight (1e-3) */
  const float* reverb_noise;   /* [n_reverbs][2][2*fs] fixed U(-1,1) noises of the reverbs in canonical order
                                  (Sec. 3.4); required when reverbs are enabled; copied */
  int32_t noise_on_device;     /* 1: reverb_noise is a device pointer */
  int64_t workspace_limit_bytes;  /* bound on FFT scratch for one launch group; 0 = no bound */
  int32_t retain_spectra;      /* reverb/delay FFT convolutions: 1 = every node keeps its filter spectrum, input
                                  spectrum and wet signal from the forward for the backward (3 N complex values per
                                  node, N the node's FFT size; the backward then runs 3 instead of 6 length-N FFTs);
                                  -1 = the backward recomputes them in a shared scratch; 0 = automatic: keep when
                                  the kept buffers fit in workspace_limit_bytes (if set) and in 80 % of the device
                                  memory free after the console's other buffers */
  int32_t autotune;            /* 1: at creation, time the reverb/delay FFT convolution passes of one node per FFT
                                  size under the candidate row/column splits (N = N1 N2) and keep the fastest for
                                  all nodes of that size (the split changes rounding, not the result beyond it);
                                  0: the default split */
} mg_console_desc;

/* Sizes of a console (layout only). */
typedef struct {
  int32_t n_songs;
  int32_t n_processors;        /* P */
  int64_t n_proc_params;       /* processor parameters; the dry/wet logits start here */
  int64_t n_params;            /* n_proc_params + P */
  int32_t n_reverbs;
  int64_t total_samples;       /* sum of L over songs */
  double track_seconds;        /* sum over songs of K * L / fs */
  int64_t device_bytes;        /* device memory held by the console; from mg_plan, the footprint a console with
                                  this descriptor would allocate (retained spectra only when retain_spectra = 1,
                                  else the shared scratch), used for admission by memory footprint */
  int32_t launches_per_step;   /* kernel launches of forward_loss + backward + adam_step (0 from mg_plan) */
  int32_t retains_spectra;     /* 1 when the reverb/delay spectra are kept between forward and backward */
} mg_console_info;

/* Host-only layout planning (no GPU needed): fills sizes for the given console. */
mg_status mg_plan(const mg_console_desc* desc, const mg_song_desc* songs, int32_t n_songs, mg_console_info* out);

/* Build a console over n_songs songs on the current CUDA device.  Allocates all device memory, uploads
 * sources and targets, precomputes the target spectrograms and the reverb noise STFTs.  Synchronises
 * the stream before returning.  Parameters start at zero; set them with mg_set_params. */
mg_status mg_console_create(const mg_console_desc* desc, const mg_song_desc* songs, int32_t n_songs,
                            cudaStream_t stream, mg_console** out);
mg_status mg_console_destroy(mg_console* c);
mg_status mg_console_get_info(const mg_console* c, mg_console_info* out);

/* FFT convolution size of every processor: N = f * 2^log_n, rows N1 = f * 2^log_n1 (0 for processors without
 * a four-step convolution); any pointer may be NULL. */
mg_status mg_processor_fft(const mg_console* c, int32_t* f, int32_t* log_n, int32_t* log_n1);

/* Canonical layout: types[P] (index into "ecnsgdr"), param_offset[P], song[P]; any pointer may be NULL. */
mg_status mg_processor_layout(const mg_console* c, int32_t* types, int64_t* param_offset, int32_t* song);

/* Parameter vector [n_params] in the canonical layout; copied (host or device). */
mg_status mg_set_params(mg_console* c, const float* params, int64_t n, int32_t on_device);
mg_status mg_get_params(const mg_console* c, float* out, int64_t n, int32_t on_device);
/* Gradient d(sum over songs of L)/d params of the last mg_backward, same layout.  The z entries of the
 * multitap delays hold the straight-through update direction of Eq. (19). */
mg_status mg_get_grads(const mg_console* c, float* out, int64_t n, int32_t on_device);
/* Sparsity weight alpha_p of Eq. (26) used by the next forward_loss / backward. */
mg_status mg_set_alpha_p(mg_console* c, float alpha_p);

/* Forward pass and objective (Alg. 1 schedule, Eqs. 2, 20-23, 26).
 * d_mask: device {0,1}[P] multiplied into the dry/wet weights, or NULL (all ones); copied.
 * d_losses: device [n_songs][7] = (L_a, L_lr, L_m, L_s, L_g, L_p, L) per song, or NULL.
 * d_mix: device [sum_songs 2*L] rendered mixes (song-major, planar stereo), or NULL.
 * A call with d_mask == NULL arms mg_backward. */
mg_status mg_forward_loss(mg_console* c, const uint8_t* d_mask, float* d_losses, float* d_mix);

/* Reverse pass of the last unmasked forward_loss: writes the parameter gradients.
 * MG_ERR_STATE if parameters, audio or structure changed since that forward, or a masked forward or
 * mg_prune_scores ran after it. */
mg_status mg_backward(mg_console* c);

/* Masked forwards that score pruning candidates (Alg. 2 Evaluate, Alg. 3; the per-node Delta_i of Sec. 7.2):
 * for every mask j in d_masks (device {0,1}[n_masks][P]) the audio loss L_a of every song with w * mask_j.
 * d_la: device [n_masks][n_songs].  Does not touch gradients or Adam state.
 * Batched (the default): the masks are read back to the host (the call synchronises the stream, so it cannot be
 * captured in a CUDA graph); the console is rendered once under the base mask (per processor, the value most
 * masks have); then, for all masks at once, only what a mask changes is computed again as forward-only copies
 * of the nodes (a track chain from its first processor whose mask differs from the base, a subgroup chain from
 * its first such processor or whole when one of its tracks changed, the mix and the loss of every changed
 * song), one launch per processor type and level over the copies of every mask, reading the base outputs of the
 * unchanged nodes.  Every score equals (bitwise) the score of a full render under its mask.  The copies live in
 * a workspace the console allocates on first use and keeps (grown as needed); masks are processed in chunks
 * whose copies fit workspace_limit_bytes when set, else 60 % of the free device memory (at most 64 GiB), and a
 * mask whose copies alone exceed it is scored by a full render.  MG_ERR_OOM if the workspace cannot be
 * allocated.  With mg_set_score_mode(c, 1), or in one-launch-per-node mode, every mask is a full render. */
mg_status mg_prune_scores(mg_console* c, const uint8_t* d_masks, int32_t n_masks, float* d_la);
/* 0: batched scoring (default); 1: one full masked render per mask (stream-ordered, no host synchronisation). */
mg_status mg_set_score_mode(mg_console* c, int32_t mode);

/* Test hook of the compressor / gate scans (the paper has no counterpart).  Their chunks pass the envelope state
 * from one CTA to the next; every wait for a neighbour's state is bounded (about half a second), after which the
 * kernel sets an error word and continues with a zero state, and the next mg_forward_loss, mg_backward,
 * mg_train_step or mg_prune_scores returns MG_ERR_TIMEOUT.  With on = 1 the first chunk of every such launch does
 * not publish its state, so that the wait of the second chunk runs out; on = 0 restores normal operation and
 * clears a reported timeout.  The console stays usable throughout. */
mg_status mg_debug_chain_hold(mg_console* c, int32_t on);

/* One Adam step (Sec. 5.1; Kingma-Ba bias correction, decoupled weight decay) on all parameters with the
 * gradients of the last mg_backward.  Moments start at zero after create / mg_reset_optimizer. */
mg_status mg_adam_step(mg_console* c, float lr, float beta1, float beta2, float eps, float weight_decay);
mg_status mg_reset_optimizer(mg_console* c);

/* forward_loss (unmasked) + backward + adam_step as one CUDA graph, captured on first use and replayed
 * after; d_losses as in mg_forward_loss (the pointer is part of the captured graph: pass the same one). */
mg_status mg_train_step(mg_console* c, float lr, float beta1, float beta2, float eps, float weight_decay,
                        float* d_losses);

/* Structural pruning (Alg. 3, Prune): processors with h_keep[i] == 0 are removed (bypassed, no work, left
 * out of L_g and L_p; their gradients read zero).  h_keep: host {0,1}[P]; removal is permanent. */
mg_status mg_prune(mg_console* c, const uint8_t* h_keep);
/* Host {0,1}[P]: 1 for processors not removed by mg_prune. */
mg_status mg_get_present(const mg_console* c, uint8_t* h_present);

/* Replace the audio of one song (same K and L): sources [K][L], target [2][L] (NULL keeps the old target);
 * recomputes the target spectrograms.  Copied (host or device), stream-ordered: device memory and page-locked
 * host memory (cudaHostAlloc / cudaHostRegister, mapped) are read by a kernel and must stay valid until the
 * console's stream reaches the call; pageable host memory is copied before the call returns. */
mg_status mg_update_audio(mg_console* c, int32_t song, const float* sources, const float* target,
                          int32_t on_device);

/* 0: one launch per processor type over all nodes of all songs (batched, default);
 * 1: the same kernels launched once per node (one-by-one processing, Sec. 4.1 / Fig. 2d). */
mg_status mg_set_launch_mode(mg_console* c, int32_t per_node);

/* Per-kernel timing with CUDA events around every launch (1 = on; off by default).  Times accumulate
 * until mg_reset_kernel_times.  Kernel families: see mg_kernel_family_name. */
mg_status mg_set_profiling(mg_console* c, int32_t on);
int32_t mg_num_kernel_families(void);
const char* mg_kernel_family_name(int32_t family);
/* Waits for the stream, then returns per family: total milliseconds and launch counts. */
mg_status mg_get_kernel_times(mg_console* c, double* ms, int64_t* launches, int32_t n_families);
mg_status mg_reset_kernel_times(mg_console* c);
/* Same timings grouped by stage of the console: [0..6] processor types e c n s g d r (forward and backward),
 * 7 loss (STFT, Mel, adjoint), 8 mix sums, 9 other (finalisation, optimiser).  n <= 10. */
mg_status mg_get_stage_times(mg_console* c, double* ms, int64_t* launches, int32_t n);

/* Diagnostic read-back of one processor's buffers (synchronises the stream), for per-node parity checks.
 * what: 0 output y [2][L], 1 FIR taps [2][Nh] (LTI processors), 2 FIR tap gradient [2][Nh], 3 input adjoint
 * du [2][L], 4 node statistics [16], 5 output adjoint dy [2][L].  host_out must hold exactly n = rows x columns floats. */
mg_status mg_debug_read(const mg_console* c, int32_t proc, int32_t what, float* host_out, int64_t n);

/* Equalizer forward that allocates nothing.  The paper has no counterpart: this entry point serves callers
 * that cannot allocate device memory (code running under another framework's allocator or memory pool,
 * plug-in hosts that forbid device allocations on their processing threads, work already being recorded on
 * a stream).  It computes one equalizer processor of the console, y = w y_bar + (1 - w) u with
 * y_bar = h_e * u (Eqs. 7-8) and w = sigmoid(q), using the same kernels as the console.
 *   d_u:      device [2][L] stereo input (left row, then right row), FP32
 *   d_y:      device [2][L] output (must not overlap d_u)
 *   L:        1 <= L <= 128,001 samples (the 2^17-point FFT must hold the signal and the 2047-tap FIR without
 *             wrap-around: L + 2047 + 1023 + 1 <= 2^17); larger L returns MG_ERR_UNSUPPORTED without touching the GPU
 *   d_params: device [1025]: the 1024 log-magnitudes of Eq. (7), then the dry/wet logit q
 * Scratch: one file-scope __device__ array of about 3.3 MB, held by every GPU that loads the library until the
 * process exits.  Every buffer in it is fully written before it is read within a call, so nothing needs
 * clearing; calls share the array, so calls that overlap on the GPU (on different streams, or on the same
 * device from several threads without ordering) race and must not be issued.
 * Every call looks up the array's device address on the current device (cudaGetSymbolAddress, which allocates
 * nothing).  The first call on a device, made with that device current, builds the lookup tables in the array
 * and synchronises the stream: make that first call before any stream capture.  If the address ever changes
 * (the module was reloaded after a device reset), the next call rebuilds the tables the same way.  Later calls
 * are asynchronous on `stream`.  Returns MG_ERR_INVALID for null pointers, and MG_ERR_CUDA if a CUDA call
 * fails or if a CUDA error from earlier work on this host thread is still pending on entry (then nothing is
 * launched and that error is left for its owner to read). */
mg_status mg_eq_forward_noalloc(const float* d_u, float* d_y, int64_t L, const float* d_params, cudaStream_t stream);

/* Evaluation metrics of every song's mix from the most recent forward (forward_loss, train_step or
 * prune_scores) against its target (Sec. 5.3): d_out (device) [n_songs][6] = SI-SDR in dB over the stereo
 * signal, then the MIR feature distances of Eq. (27), log10 of the mean squared feature difference over
 * disjoint 8 s segments (a shorter song is one segment) for RMS (per channel), crest factor (per channel),
 * stereo width ||l - r|| / ||l + r||, stereo imbalance (||l||^2 - ||r||^2) / (||l||^2 + ||r||^2) and the
 * 24-band Zwicker Bark spectrum of the mid signal (Hann-windowed 8192-sample frames, mean power, dB);
 * -inf where the features agree exactly.  FAD needs a pre-trained encoder and is not computed.  Stream-ordered. */
mg_status mg_evaluate(mg_console* c, float* d_out);

/* ---- Batched-processing schedule of a general processing graph (Sec. 4, Alg. 1 lines 1-4; host only) ----
 * A schedule is a sequence of node types; step n computes the maximal subset V_n of not yet computed nodes of
 * its type whose predecessors are all computed, so the subsets partition the graph, are causal and
 * homogeneous (Sec. 4.1).  Greedy: the type with the most computable nodes at each step, ties to the smaller
 * type code (Sec. 4.2).  Beam: a layered search keeping the beam_width states with the most computed nodes per
 * depth, stopping at the first depth that completes the graph (the shortest schedule when the beam holds
 * every state of a depth).  No GPU is used. */
enum { MG_SCHED_GREEDY = 0, MG_SCHED_BEAM = 1 };

/* node_type [n_nodes]: any non-negative type codes; edges edge_src[i] -> edge_dst[i], no self loops.
 * Outputs (caller-allocated, n_nodes entries each): step_type[0 .. *n_steps) the type sequence; node_step[v]
 * the step computing node v; order[i] the node placed at position i (ScheduleBatchedProcessing and
 * OptimizeNodeOrder: nodes sorted by step, then index, so every subset is one contiguous slice).
 * MG_ERR_INVALID for bad arguments or a graph with a cycle. */
mg_status mg_schedule_graph(const int32_t* node_type, int32_t n_nodes, const int32_t* edge_src,
                            const int32_t* edge_dst, int32_t n_edges, int32_t method, int32_t beam_width,
                            int32_t* step_type, int32_t* n_steps, int32_t* node_step, int32_t* order);

/* GetReadWriteIndex for a schedule in the new order: step_begin [n_steps + 1] the store slices (positions
 * step_begin[k] .. step_begin[k+1] are V_k); gather_begin [n_steps + 1] and gather_src / gather_dst [n_edges]
 * the gather lists of every step (producer position -> consumer position, grouped by the consumer's step,
 * then consumer, then producer; the aggregate of a consumer is the sum over its entries). */
mg_status mg_schedule_io(const int32_t* node_step, const int32_t* order, int32_t n_nodes, int32_t n_steps,
                         const int32_t* edge_src, const int32_t* edge_dst, int32_t n_edges, int32_t* step_begin,
                         int32_t* gather_begin, int32_t* gather_src, int32_t* gather_dst);

/* ---- General processing graphs on the GPU (Sec. 2, Sec. 4, Alg. 1) ----
 * A graph of one song: input nodes (one dry track each, duplicated to both channels), processor nodes of the types
 * 0..6 = "ecnsgdr" (Sec. 3, each followed by its dry/wet blend), mix nodes and exactly one output node.  Every node's
 * input is the sum of its predecessors' outputs (Eq. 3); the output node's input is the mix y_hat, scored by the
 * console's objective (Eqs. 20-23, 26).  The processors are the graph's processor nodes in ascending node index: the
 * canonical order of the parameters (each processor's parameters, then one dry/wet logit per processor) and of the
 * masks.  Execution follows the batched schedule of Alg. 1 (mg_schedule_graph): per step one aggregation launch
 * for the nodes with several predecessors (gather and aggregate) and one launch per kernel over the step's
 * processors (process and store); the backward pass walks the steps in reverse, summing the input adjoints of
 * nodes with several successors. */
enum { MG_NODE_INPUT = 7, MG_NODE_MIX = 8, MG_NODE_OUTPUT = 9 };

typedef struct {
  int32_t n_nodes;
  const int32_t* node_type;    /* host [n_nodes]: 0..6 processor types, MG_NODE_INPUT, MG_NODE_MIX, MG_NODE_OUTPUT */
  const int32_t* input_track;  /* host [n_nodes]: for input nodes the source track in [0, K); ignored otherwise */
  int32_t n_edges;
  const int32_t* edge_src;     /* host [n_edges]: edge_src[i] -> edge_dst[i] */
  const int32_t* edge_dst;
  int32_t schedule;            /* MG_SCHED_GREEDY or MG_SCHED_BEAM */
  int32_t beam_width;          /* beam search width (>= 1) */
} mg_graph_desc;

/* Host-only planning of a graph console (no GPU): sizes as mg_plan; step_type (host [n_nodes] or NULL) receives the
 * schedule's type sequence and n_steps (or NULL) its length.  MG_ERR_INVALID for a bad graph: node types out of
 * range, not exactly one output node, an input node with a predecessor or without a valid track, a processor, mix
 * or output node without a predecessor, an output node with a successor, an edge out of range or a self loop, a
 * cycle. */
mg_status mg_graph_plan(const mg_console_desc* desc, const mg_graph_desc* graph, const mg_song_desc* song,
                        mg_console_info* out, int32_t* step_type, int32_t* n_steps);

/* Console over one song whose structure is `graph` (song->num_subgroups and song->track_group are ignored; the
 * type_mask of desc is ignored: the processors are the graph's).  Every other entry point applies to it; candidate
 * scoring (mg_prune_scores) renders every mask in full.  Allocation and synchronisation as mg_console_create. */
mg_status mg_graph_console_create(const mg_console_desc* desc, const mg_graph_desc* graph, const mg_song_desc* song,
                                  cudaStream_t stream, mg_console** out);

/* Message of the last failed call: on console c (valid until the next call on c), or, with c = NULL, of the last
 * failed call of this host thread that had no console (creation, planning, scheduling).  Never NULL; the
 * empty string before any failure.  The library owns the string. */
const char* mg_last_error(const mg_console* c);

#ifdef __cplusplus
}
#endif
#endif /* MIXGRAPH_H */

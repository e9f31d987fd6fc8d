// Host engine and C ABI of the mixing-console hot path (see include/mixgraph.h).
//
// Layout (Sec. 4.3, re-designed for one GPU and many songs): every processor node of every song is one entry
// of a flattened node table (ProcDev).  The forward pass walks the console's type string
// i e c n s g d r m e c n s g d r o (Sec. 4.2) once: for each position one launch per kernel covers all nodes
// of that type in all songs (work items = (node, tile)), instead of the paper's per-graph gather /
// aggregate / store with index_select and scatter: node outputs are written once into their own slice of
// one device arena, and every node reads its input slice in place.  The backward pass walks the string in
// reverse.  Per-node reductions use fixed-order partial sums so results do not depend on batch composition.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <array>
#include <mutex>
#include <string>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "../../include/mixgraph.h"
#include "mg_internal.cuh"
#include "mg_fftp.cuh"

using namespace mg;

namespace {

constexpr const char* kTypeChars = "ecnsgdr";
constexpr int kParamCount[NTYPES] = {1024, 4, 4, 1, 2, 880, 768};

enum Family {
  F_GS_FWD, F_GS_BWD, F_SUM, F_DYN_FWD, F_DYN_BWD, F_EQ_FIR, F_DLY_FIR, F_REV_FIR, F_FIR_ADJ, F_COL_FWD, F_ROW_HZ,
  F_ROW_CONV, F_COL_OUT, F_COL_DYBAR, F_ROW_BWD2, F_COL_DU, F_COL_DH, F_LOSS_FWD, F_LOSS_BWD, F_LOSS_GATHER,
  F_FINALIZE, F_ADAM, F_MISC, F_EQ_OS_FWD, F_EQ_OS_BWD, F_EQ_OS_DU, F_SCALE, F_COUNT
};
const char* kFamilyNames[F_COUNT] = {
    "gs_fwd", "gs_bwd", "sum", "dyn_fwd", "dyn_bwd", "eq_fir", "dly_fir", "rev_fir", "fir_adj", "col_fwd", "row_hz",
    "row_conv", "col_out", "col_dybar", "row_bwd2", "col_du", "col_dh", "loss_fwd", "loss_bwd", "loss_gather",
    "finalize", "adam", "misc", "eq_os_fwd", "eq_os_bwd", "eq_os_du", "chan_scale"};

inline int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }
inline int ilog2_ceil(int64_t x) {
  int l = 0;
  while (((int64_t)1 << l) < x) ++l;
  return l;
}

struct HostProc {
  int type, song, chain, level, qidx, rev;
  int present = 1;
  int64_t poff;
  int L, ld;
  int logN = 0, logN1 = 0, logN2 = 0, f = 1, colG = 0, n0 = 0, Nh = 0, nchunks = 0, nframes = 0;
  int nfrows = 0, nbrows = 0;
  int nfcap = 0;                 // partial-sum rows allocated (the largest column-item count of the candidate splits)
  std::vector<int> splits;       // candidate row exponents logN1 of the FFT convolution (autotuner)
  // arena offsets (bytes)
  size_t o_cflag = 0;        // published states of the chained scans (c, n)
  size_t o_y = 0, o_stats = 0, o_fpart = 0, o_bpart = 0, o_taps = 0, o_dtaps = 0, o_aux = 0, o_carry = 0,
         o_cagg = 0, o_nspec = 0, o_hspec = 0, o_ybar = 0, o_dhspec = 0, o_eqg = 0;
  size_t scratch_bytes = 0;  // T1 + T2 + Hz
  size_t o_scratch = 0;      // offset inside the shared LTI scratch
};

struct HostChain {
  int song, level, index, L, ld;
  std::vector<int> procs;
  size_t o_in = 0;           // chain input: source (track) or mix-node output (subgroup)
  size_t o_dA = 0, o_dB = 0; // adjoint ping-pong
};

struct HostSong {
  int K, S, L, ld;
  std::vector<int> group;
  int nframes[3] = {0, 0, 0}, first[3] = {0, 0, 0}, litems[3] = {0, 0, 0}, lcap = 0;
  size_t o_mix = 0, o_dmix = 0, o_tgt = 0, o_Y[3] = {0, 0, 0}, o_Yh[3] = {0, 0, 0}, o_dF[3] = {0, 0, 0}, o_lpart = 0, o_coef = 0,
         o_ynorm = 0;
  std::vector<int> tracks_chain, groups_chain;
  int pbeg = 0, pend = 0;
  double track_seconds = 0;
};

template <class T>
struct DevVec {
  std::vector<T> h;
  T* d = nullptr;
};

// A launch list: items sorted by processor, with per-processor ranges for one-launch-per-node mode.
struct ItemList {
  std::vector<Item> h;
  std::vector<int> beg;  // ranges: [beg[i], beg[i+1]) for i-th proc
  Item* d = nullptr;
  int maxv = 0;          // kernel-specific size bound (max N2*G or N1)
};
struct ProcList {
  std::vector<int> h;
  int* d = nullptr;
};

struct LtiGroup {
  ProcList procs;
  ItemList col, rowpair, firtaps, dlyadj, revfir;
};

// A node of a general processing graph (Sec. 2): input, processor, mix or output, its edges, and the arena
// buffers its wiring needs: the sum of its inputs (more than one predecessor), the sum of its successors'
// input adjoints (more than one successor), and a processor's own input adjoint.
struct GNode {
  int type = 0, track = -1, proc = -1, step = 0;
  std::vector<int> preds, succs;
  size_t o_agg = 0, o_dsum = 0, o_du = 0;
};

struct Stage {
  int level, type;
  ProcList procs;
  ItemList elem;                 // g, s, c, n (tile / chunk items)
  ItemList elem_rev;             // c, n: chunk items in reverse order per node (the chained backward)
  ItemList chain_f, chain_b;     // c, n: the same chunks in rounds across nodes (batched launches)
  ItemList osf, osb;             // e: overlap-save blocks of the forward and backward kernels
  std::vector<LtiGroup> groups;  // e, r, d
};

}  // namespace

// Graph capture of one console must not overlap another thread's device allocation or release (cudaFree may
// synchronise the device, which invalidates a capture in progress): consoles driven from several host threads
// serialise those three operations on this lock.
std::mutex g_device_mutex;

struct mg_console {
  mg_console_desc desc{};
  std::vector<HostSong> songs;
  std::vector<HostProc> procs;
  std::vector<HostChain> chains;
  int P = 0, nrev = 0, nres = 0;
  int64_t npp = 0, nparams = 0;
  double track_seconds = 0;
  int64_t total_samples = 0;
  cudaStream_t stream = nullptr;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  char* scratch = nullptr;
  size_t scratch_bytes = 0;
  float* d_params = nullptr;
  float* d_grads = nullptr;
  float* d_m = nullptr;
  float* d_v = nullptr;
  int* d_step = nullptr;
  float* d_hyper = nullptr;
  float* d_alphas = nullptr;
  uint8_t* d_mask = nullptr;
  float* d_scratch_la = nullptr;   // [n_songs] L_a of every song under the base mask of a candidate scoring call
  std::vector<size_t> chain_out;   // arena offset of every chain's output (its last present processor, or its input)
  // candidate scoring: workspace of the forward-only node copies (grown on demand, kept), its byte budget, and
  // host staging of its tables and of the base mask
  char* score_ws = nullptr;
  size_t score_ws_bytes = 0;
  size_t score_budget = 0;
  std::vector<char> score_blob;
  std::vector<uint8_t> score_m0;
  // the last batched scoring call's surviving chunk: its base mask, the candidates' masks, per (candidate, song)
  // the node outputs a candidate recomputed (arena destination, workspace source) and its song copy, so that a
  // next call whose base mask equals, song by song, the old base or one of these candidates starts from them
  struct ScoreKeep {
    bool valid = false;
    std::vector<uint8_t> m0, masks;
    int nc = 0;
    std::vector<std::vector<std::pair<char*, const char*>>> promo;   // [cand * n_songs + song]
    std::vector<int> vsong;                                         // [cand * n_songs + song]
    const float* vla = nullptr;
  } score_keep;
  // general processing graph (Sec. 2, Sec. 4): nodes, the batched schedule (Alg. 1) as steps of one type each,
  // per step the aggregation sums of the forward and the adjoint sums of the backward, one source buffer per
  // track, and a zero buffer (the adjoint of an output nothing reads)
  bool is_graph = false;
  std::vector<GNode> gn;
  std::vector<int> gstep_type;
  std::vector<std::vector<int>> gstep_nodes;
  std::vector<int> gstep_stage;
  std::vector<ItemList> gstep_fsum, gstep_bsum;
  std::vector<size_t> o_src;
  size_t o_zero = 0;
  int score_mode = 0;              // 0: batched candidate scoring, 1: one full masked render per candidate
  int elem_tile = kElemTile;       // samples per work item of the elementwise kernels and sums (packing tuner)
  unsigned* d_chain = nullptr;     // launch generation and work ticket of the chained scans
  int* h_err = nullptr;            // host-mapped error word of the chained scans' bounded waits
  int* d_err = nullptr;
  int chain_hold = 0;              // test hook (mg_debug_chain_hold)
  int loss_per[3] = {0, 0, 0};     // frames per loss work item per resolution (packing tuner; 0: 8192 / n_fft)
  bool debug_sync = false;         // MG_DEBUG_SYNC=1 in the environment: synchronise and check after every launch
  bool dyn_tma = true;             // TMA staging of the compressor / gate forward (MG_DYN_TMA=0: plain loads)
  float** d_track_in = nullptr;    // input buffer of every track, song-major (mg_update_audio's one-launch ingest)
  std::vector<int> track_in_base;  // first entry of each song in d_track_in
  bool debug_reported = false;
  ProcDev* d_procs = nullptr;
  SongDev* d_songs = nullptr;
  LossRes* d_res = nullptr;
  int64_t* d_mixoff = nullptr;
  Tables tab{};
  std::vector<void*> table_allocs;
  std::vector<ProcDev> hpd;
  std::vector<SongDev> hsd;
  std::vector<LossRes> hres;
  int loss_max_dy = 0;            // floats of the loss adjoint's per-item band gradients (largest resolution)
  std::vector<Stage> stages;      // forward order
  // sums
  DevVec<float*> sum_out;
  DevVec<const float*> sum_in;
  DevVec<int> sum_beg, sum_L, sum_ld;
  ItemList sum_m_items, sum_o_items;
  int n_msum = 0;
  ProcList all_present;
  ProcList all_lti_present;
  DevVec<int4> loss_items[3];
  ItemList gather_items;
  // evaluation metrics (Sec. 5.3): (song, 8 s segment) items, per-song item ranges, Bark band bin ranges
  std::vector<int2> ev_items;
  std::vector<int> ev_begin, ev_lo, ev_hi;
  int2* d_ev_items = nullptr;
  int* d_ev_begin = nullptr;
  int* d_ev_lo = nullptr;
  int* d_ev_hi = nullptr;
  double* d_ev_out = nullptr;
  int ev_seg_len = 0;
  // state
  bool fwd_valid = false;
  bool per_node = false;
  bool profiling = false;
  float alpha_p = 0.f;
  std::string err;
  cudaGraphExec_t graph = nullptr;
  float* graph_losses = nullptr;
  bool graph_profiled = false;
  int launches = 0;
  int launches_step = 0;
  bool retain = false;           // reverb/delay nodes keep Hz, U and y_bar from the forward (own scratch each)
  // profiling
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_next = 0;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending, graph_pairs;
  double fam_ms[F_COUNT] = {0};
  int64_t fam_n[F_COUNT] = {0};
  // stages: 0..6 processor types e c n s g d r, 7 loss, 8 mix sums, 9 other (optimiser, finalisation)
  int cur_stage = 9;
  double stage_ms[10] = {0};
  int64_t stage_n[10] = {0};
  // loss items of one song (per resolution: first item, count) for per-song target refresh
  std::vector<std::array<int2, 3>> song_litems;
  bool capturing = false;
  std::vector<void*> small_allocs;
};

namespace {

thread_local std::string g_static_err;   // errors of calls without a console (per host thread)

mg_status fail(mg_console* c, mg_status s, const std::string& msg) {
  if (c) c->err = msg;
  else g_static_err = msg;
  return s;
}

#define CK(call)                                                                                  \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return fail(c, MG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// ------------------------------------------------------------------------------------------------
// planning (host only)
// ------------------------------------------------------------------------------------------------
// Four-step split of N = f 2^logN into rows N1 = f 2^logN1 and columns N2 = 2^logN2; a split is valid when the
// rows fit the row kernels (N1 <= 2048, 3072 with the factor 3, 2560 with the factor 5), a column tile holds at
// least one column (N2 <= 8192) and both factors are at least 8 (16 for the rows, one radix-16 pass).
bool split_ok(int f, int logN, int logN1) {
  const int logN2 = logN - logN1;
  const int max_a = f == 1 ? 11 : (f == 3 ? kPtw3MaxA : kPtw5MaxA);
  return logN1 >= 4 && logN2 >= 3 && logN2 <= 13 && logN1 <= max_a;
}
void apply_split(HostProc& p, int logN1) {
  p.logN1 = logN1;
  p.logN2 = p.logN - logN1;
  p.colG = std::min(8, std::min(8192 >> p.logN2, 1 << p.logN1));
  p.nfrows = (p.f << p.logN1) / p.colG;
  p.nbrows = p.nfrows;
}

mg_status validate(mg_console* c, const mg_console_desc* d, const mg_song_desc* s, int n, bool graph = false) {
  if (!d || !s || n <= 0) return fail(c, MG_ERR_INVALID, "null descriptor or no songs");
  if (!(d->sample_rate > 1000.0 && d->sample_rate < 1e6)) return fail(c, MG_ERR_INVALID, "sample_rate out of range");
  if (d->type_mask & ~0x7Fu) return fail(c, MG_ERR_INVALID, "type_mask has bits beyond the 7 processor types");
  if (d->n_resolutions < 1 || d->n_resolutions > 3) return fail(c, MG_ERR_INVALID, "n_resolutions must be 1..3");
  for (int r = 0; r < d->n_resolutions; ++r) {
    const int nf = d->n_fft[r];
    if (nf < 64 || nf > 8192 || (nf & (nf - 1))) return fail(c, MG_ERR_INVALID, "n_fft must be a power of two in [64, 8192]");
    if (d->hop_div < 1 || nf % d->hop_div) return fail(c, MG_ERR_INVALID, "hop_div must divide n_fft");
  }
  if (d->n_mels < 0 || d->n_mels > 512) return fail(c, MG_ERR_INVALID, "n_mels must be in [0, 512]");
  for (int r = 0; r < d->n_resolutions; ++r) {
    const int nf = d->n_fft[r], bands = d->n_mels > 0 ? d->n_mels : nf / 2 + 1;
    if ((8192 / nf) * bands * 4 > kLossMaxDy)
      return fail(c, MG_ERR_INVALID, "bands x frames per loss work item exceed shared memory (fewer n_mels or a larger n_fft)");
  }
  if (d->warmup_samples < 0) return fail(c, MG_ERR_INVALID, "negative warmup_samples");
  if (d->retain_spectra < -1 || d->retain_spectra > 1) return fail(c, MG_ERR_INVALID, "retain_spectra must be -1, 0 or 1");
  for (int i = 0; i < n; ++i) {
    if (s[i].num_tracks < 1 || s[i].num_subgroups < 0) return fail(c, MG_ERR_INVALID, "song needs >= 1 track");
    if (s[i].num_samples < 1 || s[i].num_samples > (1 << 22) - 200000)
      return fail(c, MG_ERR_UNSUPPORTED, "num_samples must be in [1, 3994304]");
    if (graph) continue;   // a graph's structure comes from its nodes and edges
    if (!s[i].track_group) return fail(c, MG_ERR_INVALID, "track_group is null");
    for (int k = 0; k < s[i].num_tracks; ++k)
      if (s[i].track_group[k] < -1 || s[i].track_group[k] >= s[i].num_subgroups)
        return fail(c, MG_ERR_INVALID, "track_group entry out of range");
  }
  return MG_OK;
}

// Work decomposition of one processor of L samples (p.type, p.L set): FIR span and FFT size of the LTI types
// (N = f 2^logN >= L + taps, the smaller of 2^k and 3 2^k'; rows N1 = f 2^logN1, columns N2 = 2^logN2; the
// autotuner's candidate splits), overlap-save blocks of the equalizer, scan chunks of the dynamics, tiles of
// the elementwise types.
void size_proc(HostProc& p, double fs) {
  const int t = p.type;
  const int D = (int)std::llround(0.1 * fs);
  const int revlen = (int)std::llround(2.0 * fs);
  if (t == T_E || t == T_R || t == T_D) {
    if (t == T_E) { p.n0 = -kEqHalf; p.Nh = kEqTaps; }
    if (t == T_D) { p.n0 = -kDlyHalf; p.Nh = kDlyTaps * D + kDlyFir - 1; }
    if (t == T_R) { p.n0 = 0; p.Nh = revlen; p.nframes = (revlen - kRevFft) / kRevHop + 1; }
    // N = f 2^logN >= L + taps: the smallest of 2^k, 3 2^k' and 5 2^k''; rows N1 = f 2^logN1, columns
    // N2 = 2^logN2
    const int64_t need = (int64_t)p.L + p.Nh + std::abs(p.n0) + 1;
    const int k2 = std::max(12, ilog2_ceil(need));
    const int k3 = std::max(11, ilog2_ceil((need + 2) / 3));
    const int k5 = std::max(10, ilog2_ceil((need + 4) / 5));
    const int64_t n2 = (int64_t)1 << k2, n3 = (int64_t)3 << k3, n5 = (int64_t)5 << k5;
    // 5 2^k'' when the rows fit (N1 = 5 2^logN1 <= 2560 with N2 <= 2^10)
    if (t != T_E && n5 < n3 && n5 < n2 && k5 - std::min(10, (k5 + 1) / 2) <= kPtw5MaxA) {
      p.f = 5;
      p.logN = k5;
      p.logN2 = std::min(10, (k5 + 1) / 2);
      p.logN1 = k5 - p.logN2;
    } else if (t != T_E && n3 < n2) {
      p.f = 3;
      p.logN = k3;
      p.logN2 = std::min(10, (k3 + 1) / 2);
      p.logN1 = k3 - p.logN2;
    } else {
      p.f = 1;
      p.logN = k2;
      p.logN1 = (k2 + 1) / 2;
      p.logN2 = k2 / 2;
    }
    p.colG = std::min(8, std::min(8192 >> p.logN2, 1 << p.logN1));
    if (t == T_E) {   // single-pass overlap-save in shared memory (no global FFT scratch)
      p.nfrows = (p.L + kEqOsFwdBlock - 1) / kEqOsFwdBlock;
      p.nbrows = (p.nfrows + kEqChunk - 1) / kEqChunk;   // backward items: chunks of forward blocks
    } else {
      p.nfrows = (p.f << p.logN1) / p.colG;
      p.nbrows = p.nfrows;
      p.scratch_bytes = (size_t)3 * ((size_t)p.f << p.logN) * sizeof(float2);
      // autotuner candidates: the default split and its neighbours; partial sums sized for all of them
      p.splits.clear();
      p.nfcap = p.nfrows;
      for (int dl = -2; dl <= 2; ++dl) {
        const int l1 = p.logN1 + dl;
        if (!split_ok(p.f, p.logN, l1)) continue;
        HostProc q = p;
        apply_split(q, l1);
        p.splits.push_back(l1);
        p.nfcap = std::max(p.nfcap, q.nfrows);
      }
    }
  } else if (t == T_C || t == T_N) {
    p.nchunks = (p.L + kDynChunk - 1) / kDynChunk;
    p.nbrows = p.nchunks;
  } else {
    p.nbrows = (p.L + kElemTile - 1) / kElemTile;
    p.nfcap = (p.L + kElemTileMin - 1) / kElemTileMin;   // partial-sum rows for every candidate tile
  }
}

// Graph planning (host): one song, its processors in node order (the canonical order of the parameters), each
// sized like a console processor, and the batched schedule of Alg. 1 (greedy or beam, schedule.cu) as steps.
mg_status plan_graph(mg_console* c, const mg_console_desc* d, const mg_graph_desc* g, const mg_song_desc* s) {
  c->is_graph = true;
  c->desc = *d;
  c->nres = d->n_resolutions;
  const double fs = d->sample_rate;
  c->songs.clear();
  c->procs.clear();
  c->chains.clear();
  c->nrev = 0;
  HostSong hs;
  hs.K = s->num_tracks;
  hs.S = 0;
  hs.L = (int)s->num_samples;
  hs.ld = (int)round_up(hs.L, 64);
  hs.group.assign(hs.K, -1);
  hs.pbeg = 0;
  hs.track_seconds = (double)hs.K * hs.L / fs;
  c->track_seconds = hs.track_seconds;
  c->total_samples = hs.L;
  const int n = g->n_nodes;
  c->gn.assign(n, GNode{});
  for (int v = 0; v < n; ++v) {
    c->gn[v].type = g->node_type[v];
    c->gn[v].track = g->node_type[v] == MG_NODE_INPUT ? g->input_track[v] : -1;
  }
  for (int e = 0; e < g->n_edges; ++e) {
    c->gn[g->edge_src[e]].succs.push_back(g->edge_dst[e]);
    c->gn[g->edge_dst[e]].preds.push_back(g->edge_src[e]);
  }
  std::vector<int> step_type(std::max(1, n)), node_step(std::max(1, n)), order(std::max(1, n));
  int nsteps = 0;
  if (mg_schedule_graph(g->node_type, n, g->edge_src, g->edge_dst, g->n_edges, g->schedule, g->beam_width,
                        step_type.data(), &nsteps, node_step.data(), order.data()) != MG_OK)
    return fail(c, MG_ERR_INVALID, "graph has a cycle or invalid edges");
  c->gstep_type.assign(step_type.begin(), step_type.begin() + nsteps);
  c->gstep_nodes.assign(nsteps, {});
  for (int v = 0; v < n; ++v) {
    c->gn[v].step = node_step[v];
    c->gstep_nodes[node_step[v]].push_back(v);
  }
  int64_t poff = 0;
  for (int v = 0; v < n; ++v) {
    const int t = c->gn[v].type;
    if (t >= NTYPES) continue;
    HostProc p;
    p.type = t;
    p.song = 0;
    p.chain = -1;
    p.level = c->gn[v].step;
    p.qidx = (int)c->procs.size();
    p.rev = t == T_R ? c->nrev++ : -1;
    p.poff = poff;
    poff += kParamCount[t];
    p.L = hs.L;
    p.ld = hs.ld;
    size_proc(p, fs);
    c->gn[v].proc = (int)c->procs.size();
    c->procs.push_back(p);
  }
  hs.pend = (int)c->procs.size();
  c->songs.push_back(hs);
  c->P = (int)c->procs.size();
  c->npp = poff;
  c->nparams = poff + c->P;
  return MG_OK;
}

// Checks of a graph description: node types, one output, edges in range and without self loops, inputs without
// predecessors and with a valid track, every processor, mix and the output with at least one predecessor, the
// output without successors.  Cycles are found by the scheduler.
mg_status validate_graph(mg_console* c, const mg_console_desc* d, const mg_graph_desc* g, const mg_song_desc* s) {
  if (!d || !g || !s) return fail(c, MG_ERR_INVALID, "null descriptor");
  if (g->n_nodes < 2 || !g->node_type || (g->n_edges > 0 && (!g->edge_src || !g->edge_dst)) || g->n_edges < 0)
    return fail(c, MG_ERR_INVALID, "graph needs nodes and edges");
  if (s->num_tracks < 1 || s->num_samples < 1 || s->num_samples > (1 << 22) - 200000)
    return fail(c, MG_ERR_INVALID, "song needs >= 1 track and 1..3994304 samples");
  std::vector<int> np(g->n_nodes, 0), ns(g->n_nodes, 0);
  int outputs = 0;
  for (int e = 0; e < g->n_edges; ++e) {
    const int a = g->edge_src[e], b = g->edge_dst[e];
    if (a < 0 || b < 0 || a >= g->n_nodes || b >= g->n_nodes || a == b) return fail(c, MG_ERR_INVALID, "edge out of range");
    ++ns[a];
    ++np[b];
  }
  for (int v = 0; v < g->n_nodes; ++v) {
    const int t = g->node_type[v];
    if (t < 0 || t > MG_NODE_OUTPUT) return fail(c, MG_ERR_INVALID, "node type out of range");
    if (t == MG_NODE_INPUT) {
      if (!g->input_track || g->input_track[v] < 0 || g->input_track[v] >= s->num_tracks)
        return fail(c, MG_ERR_INVALID, "input node without a valid track");
      if (np[v]) return fail(c, MG_ERR_INVALID, "input node with a predecessor");
    } else if (np[v] == 0) {
      return fail(c, MG_ERR_INVALID, "processor, mix or output node without a predecessor");
    }
    if (t == MG_NODE_OUTPUT) {
      ++outputs;
      if (ns[v]) return fail(c, MG_ERR_INVALID, "output node with a successor");
    }
  }
  if (outputs != 1) return fail(c, MG_ERR_INVALID, "a graph needs exactly one output node");
  return validate(c, d, s, 1, true);
}

void plan(mg_console* c, const mg_console_desc* d, const mg_song_desc* s, int n) {
  c->desc = *d;
  c->nres = d->n_resolutions;
  const double fs = d->sample_rate;
  const int D = (int)std::llround(0.1 * fs);
  const int revlen = (int)std::llround(2.0 * fs);
  std::vector<int> chain_types;
  for (int t = 0; t < NTYPES; ++t)
    if (d->type_mask & (1u << t)) chain_types.push_back(t);
  int64_t poff = 0;
  c->songs.clear();
  c->procs.clear();
  c->chains.clear();
  c->nrev = 0;
  c->track_seconds = 0;
  c->total_samples = 0;
  for (int si = 0; si < n; ++si) {
    HostSong hs;
    hs.K = s[si].num_tracks;
    hs.S = s[si].num_subgroups;
    hs.L = (int)s[si].num_samples;
    hs.ld = (int)round_up(hs.L, 64);
    hs.group.assign(s[si].track_group, s[si].track_group + hs.K);
    hs.pbeg = (int)c->procs.size();
    hs.track_seconds = (double)hs.K * hs.L / fs;
    c->track_seconds += hs.track_seconds;
    c->total_samples += hs.L;
    for (int ch = 0; ch < hs.K + hs.S; ++ch) {
      HostChain hc;
      hc.song = si;
      hc.level = ch < hs.K ? 0 : 1;
      hc.index = ch < hs.K ? ch : ch - hs.K;
      hc.L = hs.L;
      hc.ld = hs.ld;
      for (int t : chain_types) {
        HostProc p;
        p.type = t;
        p.song = si;
        p.chain = (int)c->chains.size();
        p.level = hc.level;
        p.qidx = (int)c->procs.size();
        p.rev = t == T_R ? c->nrev++ : -1;
        p.poff = poff;
        poff += kParamCount[t];
        p.L = hs.L;
        p.ld = hs.ld;
        size_proc(p, fs);
        hc.procs.push_back((int)c->procs.size());
        c->procs.push_back(p);
      }
      if (hc.level == 0) hs.tracks_chain.push_back((int)c->chains.size());
      else hs.groups_chain.push_back((int)c->chains.size());
      c->chains.push_back(hc);
    }
    hs.pend = (int)c->procs.size();
    c->songs.push_back(hs);
  }
  c->P = (int)c->procs.size();
  c->npp = poff;
  c->nparams = poff + c->P;
}

// ------------------------------------------------------------------------------------------------
// host tables (double precision, rounded once to fp32)
// ------------------------------------------------------------------------------------------------
double a_weight(double f) {
  auto ra = [](double x) {
    const double f2 = x * x;
    return (12194.0 * 12194.0 * f2 * f2) /
           ((f2 + 20.6 * 20.6) * std::sqrt((f2 + 107.7 * 107.7) * (f2 + 737.9 * 737.9)) * (f2 + 12194.0 * 12194.0));
  };
  return ra(f) / ra(1000.0);
}

void mel_bank(int nfft, int nmels, double fs, std::vector<std::vector<double>>& W) {
  const int nb = nfft / 2 + 1;
  auto hz2mel = [](double f) { return 2595.0 * std::log10(1.0 + f / 700.0); };
  auto mel2hz = [](double m) { return 700.0 * (std::pow(10.0, m / 2595.0) - 1.0); };
  std::vector<double> edges(nmels + 2);
  const double top = hz2mel(fs / 2.0);
  for (int i = 0; i < nmels + 2; ++i) edges[i] = mel2hz(top * i / (nmels + 1));
  W.assign(nmels, std::vector<double>(nb, 0.0));
  for (int b = 0; b < nmels; ++b)
    for (int k = 0; k < nb; ++k) {
      const double f = (double)k * fs / nfft;
      const double lo = edges[b], ce = edges[b + 1], hi = edges[b + 2];
      W[b][k] = std::max(0.0, std::min((f - lo) / (ce - lo), (hi - f) / (hi - ce)));
    }
}

// ------------------------------------------------------------------------------------------------
// launching
// ------------------------------------------------------------------------------------------------
void accumulate_pair(mg_console* c, int code, cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  const int fam = code % F_COUNT, st = code / F_COUNT;
  c->fam_ms[fam] += ms;
  c->fam_n[fam] += 1;
  c->stage_ms[st] += ms;
  c->stage_n[st] += 1;
}

// RAII: launches inside belong to one stage of the per-stage timing.
struct StageScope {
  mg_console* c;
  int prev;
  StageScope(mg_console* cc, int st) : c(cc), prev(cc->cur_stage) { c->cur_stage = st; }
  ~StageScope() { c->cur_stage = prev; }
};

template <class F>
void run(mg_console* c, int fam, F&& f) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->profiling) {
    if (c->ev_next + 2 > c->ev_pool.size()) {
      for (int i = 0; i < 256; ++i) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        c->ev_pool.push_back(e);
      }
    }
    e0 = c->ev_pool[c->ev_next++];
    e1 = c->ev_pool[c->ev_next++];
    cudaEventRecordWithFlags(e0, c->stream, c->capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
  }
  f();
  ++c->launches;
  if (c->debug_sync && !c->capturing) {
    // diagnostic mode: wait for every launch and report the first one that fails
    const cudaError_t e = cudaStreamSynchronize(c->stream);
    const cudaError_t l = cudaPeekAtLastError();
    if ((e != cudaSuccess || l != cudaSuccess) && !c->debug_reported) {
      c->debug_reported = true;
      std::fprintf(stderr, "mixgraph: launch %d (family %s, stage %d) failed: %s\n", c->launches, kFamilyNames[fam],
                   c->cur_stage, cudaGetErrorString(e != cudaSuccess ? e : l));
    }
  }
  if (c->profiling) {
    cudaEventRecordWithFlags(e1, c->stream, c->capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
    auto pr = std::make_pair(fam + F_COUNT * c->cur_stage, std::make_pair(e0, e1));
    if (c->capturing) c->graph_pairs.push_back(pr);
    else c->pending.push_back(pr);
  }
}

// Launch an item list: once over all items (batched) or once per processor (one-by-one).
template <class F>
void run_items(mg_console* c, int fam, const ItemList& L, F&& f) {
  if (L.h.empty()) return;
  if (!c->per_node) {
    run(c, fam, [&] { f(L.d, (int)L.h.size()); });
    return;
  }
  for (size_t i = 0; i + 1 < L.beg.size(); ++i) {
    const int b = L.beg[i], e = L.beg[i + 1];
    if (e > b) run(c, fam, [&] { f(L.d + b, e - b); });
  }
}
template <class F>
void run_procs(mg_console* c, int fam, const ProcList& L, F&& f) {
  if (L.h.empty()) return;
  if (!c->per_node) {
    run(c, fam, [&] { f(L.d, (int)L.h.size()); });
    return;
  }
  for (size_t i = 0; i < L.h.size(); ++i) run(c, fam, [&] { f(L.d + i, 1); });
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

LaunchCtx make_ctx(mg_console* c, const uint8_t* mask) {
  LaunchCtx x{};
  x.stream = c->stream;
  x.procs = c->d_procs;
  x.q = c->d_params + c->npp;
  x.mask = mask;
  x.hyper = c->d_hyper;
  x.alpha_g = c->desc.alpha_g;
  x.fs = c->desc.sample_rate;
  x.elem_tile = c->elem_tile;
  x.chain = c->d_chain;
  x.err = c->d_err;
  x.chain_hold = c->chain_hold;
  x.dyn_tma = c->dyn_tma && tensor_map_encoder() != nullptr;
  x.tab = c->tab;
  return x;
}

void lti_forward(mg_console* c, const LaunchCtx& x, int type, LtiGroup& g) {
  if (type == T_E) run_procs(c, F_EQ_FIR, g.procs, [&](const int* p, int n) { launch_eq_fir(x, p, n); });
  if (type == T_D) {
    run_procs(c, F_DLY_FIR, g.procs, [&](const int* p, int n) { launch_dly_prep(x, p, n); });
    run_items(c, F_DLY_FIR, g.firtaps, [&](const Item* it, int n) { launch_dly_fir(x, it, n); });
  }
  if (type == T_R) run_items(c, F_REV_FIR, g.revfir, [&](const Item* it, int n) { launch_rev_fir(x, it, n); });
  run_procs(c, F_SCALE, g.procs, [&](const int* p, int n) { launch_chan_scale(x, p, n, 0); });
  run_items(c, F_COL_FWD, g.col, [&](const Item* it, int n) { launch_col_fwd_taps(x, it, n, g.col.maxv); });
  run_items(c, F_ROW_HZ, g.rowpair, [&](const Item* it, int n) { launch_row_fwd_hz(x, it, n, g.rowpair.maxv); });
  run_items(c, F_COL_FWD, g.col, [&](const Item* it, int n) { launch_col_fwd_audio(x, it, n, g.col.maxv); });
  if (c->retain) {   // U stays in T1, y_bar in T2 (natural order) for the backward
    run_items(c, F_ROW_CONV, g.rowpair, [&](const Item* it, int n) { launch_row_conv_fwd(x, it, n, g.rowpair.maxv, true); });
    run_items(c, F_COL_OUT, g.col, [&](const Item* it, int n) { launch_col_inv_out_keep(x, it, n, g.col.maxv); });
    return;
  }
  run_items(c, F_ROW_CONV, g.rowpair, [&](const Item* it, int n) { launch_row_conv_fwd(x, it, n, g.rowpair.maxv, false); });
  run_items(c, F_COL_OUT, g.col, [&](const Item* it, int n) { launch_col_inv_out(x, it, n, g.col.maxv); });
}

void lti_backward(mg_console* c, const LaunchCtx& x, int type, LtiGroup& g) {
  run_procs(c, F_SCALE, g.procs, [&](const int* p, int n) { launch_chan_scale(x, p, n, 1); });
  if (c->retain) {
    run_items(c, F_COL_DYBAR, g.col, [&](const Item* it, int n) { launch_col_dybar_keep(x, it, n, g.col.maxv); });
  } else {
    run_items(c, F_COL_FWD, g.col, [&](const Item* it, int n) { launch_col_fwd_taps(x, it, n, g.col.maxv); });
    run_items(c, F_ROW_HZ, g.rowpair, [&](const Item* it, int n) { launch_row_fwd_hz(x, it, n, g.rowpair.maxv); });
    run_items(c, F_COL_FWD, g.col, [&](const Item* it, int n) { launch_col_fwd_audio(x, it, n, g.col.maxv); });
    run_items(c, F_ROW_CONV, g.rowpair, [&](const Item* it, int n) { launch_row_conv_fwd(x, it, n, g.rowpair.maxv, true); });
    run_items(c, F_COL_DYBAR, g.col, [&](const Item* it, int n) { launch_col_dybar(x, it, n, g.col.maxv); });
  }
  run_items(c, F_ROW_BWD2, g.rowpair, [&](const Item* it, int n) { launch_row_bwd2(x, it, n, g.rowpair.maxv); });
  run_items(c, F_COL_DU, g.col, [&](const Item* it, int n) { launch_col_du(x, it, n, g.col.maxv); });
  run_items(c, F_COL_DH, g.col, [&](const Item* it, int n) { launch_col_dh(x, it, n, g.col.maxv); });
  if (type == T_E) run_procs(c, F_FIR_ADJ, g.procs, [&](const int* p, int n) { launch_eq_fir_adj(x, p, n); });
  if (type == T_D) run_items(c, F_FIR_ADJ, g.dlyadj, [&](const Item* it, int n) { launch_dly_adj(x, it, n); });
  if (type == T_R) {
    run_items(c, F_FIR_ADJ, g.revfir, [&](const Item* it, int n) { launch_rev_adj(x, it, n); });
    run_procs(c, F_FIR_ADJ, g.procs, [&](const int* p, int n) { launch_rev_adj_fin(x, p, n); });
  }
}

void stage_forward(mg_console* c, const LaunchCtx& x, Stage& s) {
  StageScope scope(c, s.type);
  switch (s.type) {
    case T_G:
    case T_S:
      run_items(c, F_GS_FWD, s.elem, [&](const Item* it, int n) { launch_gs_fwd(x, it, n); });
      break;
    case T_C:
    case T_N:
      run_items(c, F_DYN_FWD, c->per_node ? s.elem : s.chain_f, [&](const Item* it, int n) { launch_dyn_fwd(x, it, n); });
      break;
    case T_E:
      run_procs(c, F_EQ_FIR, s.procs, [&](const int* p, int n) { launch_eq_fir(x, p, n); });
      run_procs(c, F_EQ_FIR, s.procs, [&](const int* p, int n) { launch_eq_spec(x, p, n); });
      run_items(c, F_EQ_OS_FWD, s.osf, [&](const Item* it, int n) { launch_eq_os_fwd(x, it, n); });
      break;
    default:
      for (auto& g : s.groups) lti_forward(c, x, s.type, g);
  }
}

void stage_backward(mg_console* c, const LaunchCtx& x, Stage& s) {
  StageScope scope(c, s.type);
  switch (s.type) {
    case T_G:
    case T_S:
      run_items(c, F_GS_BWD, s.elem, [&](const Item* it, int n) { launch_gs_bwd(x, it, n); });
      break;
    case T_C:
    case T_N:
      run_items(c, F_DYN_BWD, c->per_node ? s.elem_rev : s.chain_b, [&](const Item* it, int n) { launch_dyn_bwd(x, it, n); });
      break;
    case T_E:
      run_items(c, F_EQ_OS_BWD, s.osb, [&](const Item* it, int n) { launch_eq_os_bwd(x, it, n); });
      run_items(c, F_EQ_OS_DU, s.osf, [&](const Item* it, int n) { launch_eq_os_du(x, it, n); });
      run_procs(c, F_FIR_ADJ, s.procs, [&](const int* p, int n) { launch_eq_dh_reduce(x, p, n); });
      run_procs(c, F_FIR_ADJ, s.procs, [&](const int* p, int n) { launch_eq_fir_adj(x, p, n); });
      break;
    default:
      for (auto& g : s.groups) lti_backward(c, x, s.type, g);
  }
}

void run_sums(mg_console* c, const ItemList& items) {
  run_items(c, F_SUM, items, [&](const Item* it, int n) {
    launch_sum(c->stream, c->sum_out.d, c->sum_in.d, c->sum_beg.d, c->sum_L.d, c->sum_ld.d, it, n, c->elem_tile);
  });
}

// Forward of a graph: per schedule step the aggregation sums, then the step's processors (Alg. 1).
void render_graph(mg_console* c, const LaunchCtx& x) {
  for (size_t k = 0; k < c->gstep_type.size(); ++k) {
    {
      StageScope scope(c, 8);
      run_sums(c, c->gstep_fsum[k]);
    }
    if (c->gstep_stage[k] >= 0) stage_forward(c, x, c->stages[c->gstep_stage[k]]);
  }
}

void render(mg_console* c, const LaunchCtx& x) {
  if (c->is_graph) {
    render_graph(c, x);
    return;
  }
  for (int level = 0; level < 2; ++level) {
    if (level == 1 && !c->sum_m_items.h.empty()) {
      StageScope scope(c, 8);
      run_items(c, F_SUM, c->sum_m_items, [&](const Item* it, int n) {
        launch_sum(c->stream, c->sum_out.d, c->sum_in.d, c->sum_beg.d, c->sum_L.d, c->sum_ld.d, it, n, c->elem_tile);
      });
    }
    for (auto& s : c->stages)
      if (s.level == level) stage_forward(c, x, s);
  }
  StageScope scope(c, 8);
  run_items(c, F_SUM, c->sum_o_items, [&](const Item* it, int n) {
    launch_sum(c->stream, c->sum_out.d, c->sum_in.d, c->sum_beg.d, c->sum_L.d, c->sum_ld.d, it, n, c->elem_tile);
  });
}

void loss_forward(mg_console* c, const LaunchCtx& x, int mode, float* out_losses, float* out_la, int la_stride) {
  StageScope scope(c, 7);
  for (int r = 0; r < c->nres; ++r) {
    auto& L = c->loss_items[r];
    if (!L.h.empty())
      run(c, F_LOSS_FWD, [&] {   // frame kernel: 0 target spectrogram, 1 loss partials (losses and trials)
        launch_loss_frames(x, c->d_songs, c->d_res, L.d, (int)L.h.size(), mode == 0 ? 0 : (mode == 1 ? 3 : 1), c->loss_max_dy);
      });
  }
  if (mode != 0) run_procs(c, F_FINALIZE, c->all_lti_present, [&](const int* p, int n) { launch_node_stats(x, p, n, 1); });
  run(c, F_FINALIZE, [&] {
    launch_loss_finalize_mode(x, c->d_songs, (int)c->songs.size(), c->d_res, c->nres, c->d_alphas, mode, out_losses,
                              out_la, la_stride);
  });
}

void backward_pass(mg_console* c, const LaunchCtx& x) {
  {
    StageScope scope(c, 7);
    for (int r = 0; r < c->nres; ++r) {
      auto& L = c->loss_items[r];
      if (!L.h.empty())
        run(c, F_LOSS_BWD, [&] { launch_loss_frames(x, c->d_songs, c->d_res, L.d, (int)L.h.size(), 2, c->loss_max_dy); });
    }
    run_items(c, F_LOSS_GATHER, c->gather_items,
              [&](const Item* it, int n) { launch_loss_gather(x, c->d_songs, c->d_res, c->nres, it, n); });
  }
  run(c, F_MISC, [&] { cudaMemsetAsync(c->d_grads, 0, sizeof(float) * c->nparams, c->stream); });
  if (c->is_graph) {
    // per schedule step in reverse: the adjoint sums, then the step's processors
    for (int k = (int)c->gstep_type.size() - 1; k >= 0; --k) {
      {
        StageScope scope(c, 8);
        run_sums(c, c->gstep_bsum[k]);
      }
      if (c->gstep_stage[k] >= 0) stage_backward(c, x, c->stages[c->gstep_stage[k]]);
    }
  } else {
    for (int level = 1; level >= 0; --level)
      for (int i = (int)c->stages.size() - 1; i >= 0; --i)
        if (c->stages[i].level == level) stage_backward(c, x, c->stages[i]);
  }
  run_procs(c, F_FINALIZE, c->all_present, [&](const int* p, int n) { launch_node_stats(x, p, n, 0); });
  run_procs(c, F_FINALIZE, c->all_present,
            [&](const int* p, int n) { launch_grad_finalize2(x, p, n, c->d_grads + c->npp); });
}

// ------------------------------------------------------------------------------------------------
// device layout
// ------------------------------------------------------------------------------------------------
struct Bump {
  size_t off = 0;
  size_t take(size_t bytes) {
    off = (size_t)round_up((int64_t)off, 256);
    const size_t o = off;
    off += bytes;
    return o;
  }
};

// cuTensorMapEncodeTiled through the runtime's driver entry point (nothing links the driver library); nullptr when
// the driver does not offer it.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// Tensor map of a compressor / gate input u ([2][ld] floats) as 2 ld / 32 rows of 128 bytes, copied in boxes of
// 128 rows (one channel of a 4096-sample chunk) with the 128-byte swizzle; rows past the buffer read as zeros.
bool encode_dyn_map(CUtensorMap* m, const float* u, int ld) {
  const auto enc = tensor_map_encoder();
  if (!enc || !u || ld % 64 || (reinterpret_cast<uintptr_t>(u) & 255)) return false;
  const cuuint64_t dims[2] = {32, (cuuint64_t)(2 * (int64_t)ld / 32)};
  const cuuint64_t strides[1] = {128};
  const cuuint32_t box[2] = {32, (cuuint32_t)(kDynChunk / 32)};
  const cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(u), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Device copy of a host table.  Earlier copies stay allocated until the console is destroyed (tables are
// rebuilt only by mg_prune), so no pointer captured in a graph or kernel argument ever dangles.
template <class T>
mg_status upload(mg_console* c, std::vector<T>& h, T** d) {
  *d = nullptr;
  if (h.empty()) return MG_OK;
  CK(cudaMalloc(d, h.size() * sizeof(T)));
  CK(cudaMemcpyAsync(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream));
  c->small_allocs.push_back(*d);
  return MG_OK;
}
mg_status upload_items(mg_console* c, ItemList& L) { return upload(c, L.h, &L.d); }

// Tensor maps of the present compressors' and gates' input u and output adjoint dL/dy (from the node table),
// uploaded to a fresh table; a node whose maps cannot be encoded keeps nullptr and reads global memory directly.
mg_status attach_dyn_maps(mg_console* c) {
  std::vector<CUtensorMap> maps;
  std::vector<std::pair<int, int>> owner;   // (processor, 0 u / 1 dL/dy)
  for (int pi = 0; pi < c->P; ++pi) {
    ProcDev& d = c->hpd[pi];
    d.umap = nullptr;
    d.dymap = nullptr;
    const HostProc& p = c->procs[pi];
    if (!c->dyn_tma || !p.present || (p.type != T_C && p.type != T_N)) continue;
    CUtensorMap m;
    if (encode_dyn_map(&m, d.u, p.ld)) {
      maps.push_back(m);
      owner.push_back({pi, 0});
    }
    if (encode_dyn_map(&m, d.dy, p.ld)) {
      maps.push_back(m);
      owner.push_back({pi, 1});
    }
  }
  CUtensorMap* dm = nullptr;
  if (upload(c, maps, &dm) != MG_OK) return MG_ERR_CUDA;
  for (size_t k = 0; k < owner.size(); ++k) {
    if (owner[k].second == 0) c->hpd[owner[k].first].umap = dm + k;
    else c->hpd[owner[k].first].dymap = dm + k;
  }
  return MG_OK;
}
mg_status upload_procs(mg_console* c, ProcList& L) { return upload(c, L.h, &L.d); }

mg_status build_graph_tables(mg_console* c);

// Node-table entry of processor pi: everything but its wiring (u, y, dy, du, present), from the arena layout.
void fill_procdev(mg_console* c, int pi) {
  auto A = [&](size_t off) { return c->arena + off; };
  HostProc& p = c->procs[pi];
  ProcDev& d = c->hpd[pi];
  d.type = p.type;
  d.song = p.song;
  d.qidx = p.qidx;
  d.rev = p.rev;
  d.L = p.L;
  d.ld = p.ld;
  d.p = c->d_params + p.poff;
  d.gp = c->d_grads + p.poff;
  d.stats = (float*)A(p.o_stats);
  d.fpart = p.nfrows ? (float*)A(p.o_fpart) : nullptr;
  d.bpart = p.nbrows ? (float*)A(p.o_bpart) : nullptr;
  d.nfpart = p.nfrows;
  d.nbpart = p.nbrows;
  d.logN = p.logN;
  d.logN1 = p.logN1;
  d.logN2 = p.logN2;
  d.f = p.f;
  for (int r = 0; r < 5; ++r) {   // exp(-2 pi i r / N), N = f 2^logN, r < f (used when f = 3, 5)
    const double ang = -2.0 * 3.14159265358979323846 * r / ((double)std::max(1, p.f) * std::ldexp(1.0, p.logN));
    d.cfn[r] = r < p.f ? make_float2((float)std::cos(ang), (float)std::sin(ang)) : make_float2(1.f, 0.f);
  }
  d.colG = p.colG;
  d.n0 = p.n0;
  d.Nh = p.Nh;
  if (p.scratch_bytes) {
    const size_t N = (size_t)p.f << p.logN;
    d.T1 = (float2*)(c->scratch + p.o_scratch);
    d.T2 = d.T1 + N;
    d.Hz = d.T2 + N;
  }
  if (p.type == T_E || p.type == T_R || p.type == T_D) {
    d.taps = (float*)A(p.o_taps);
    d.dtaps = (float*)A(p.o_dtaps);
  }
  if (p.type == T_E) {
    d.hspec = (float*)A(p.o_hspec);
    d.ybar = (float*)A(p.o_ybar);
    d.dhspec = (float2*)A(p.o_dhspec);
    d.eqg = (float2*)A(p.o_eqg);
  }
  d.aux = p.o_aux ? (float*)A(p.o_aux) : nullptr;
  d.carry = p.nchunks ? (float*)A(p.o_carry) : nullptr;
  d.chunkagg = p.nchunks ? (float*)A(p.o_cagg) : nullptr;
  d.cflag = p.nchunks ? (unsigned long long*)A(p.o_cflag) : nullptr;
  d.nchunks = p.nchunks;
  d.nspec = p.type == T_R ? (const float2*)A(p.o_nspec) : nullptr;
  d.nframes = p.nframes;
}

// Chunk items of the chained envelope scans in rounds: round r holds chunk r (forward) or chunk n - 1 - r
// (backward) of every node with more than r chunks.  Consecutive tickets then belong to different nodes, and the
// chunk whose state a CTA waits for was drawn a round earlier; in node-major order the resident CTAs would all
// be consecutive chunks of one node and wait on each other in turn.
template <class F>
void chain_rounds(const std::vector<int>& procs, F&& nchunks, ItemList& fwd, ItemList* rev) {
  int rounds = 0;
  for (int p : procs) rounds = std::max(rounds, nchunks(p));
  for (int r = 0; r < rounds; ++r)
    for (int p : procs) {
      const int n = nchunks(p);
      if (r >= n) continue;
      fwd.h.push_back(Item{p, r});
      if (rev) rev->h.push_back(Item{p, n - 1 - r});
    }
  fwd.beg = {0, (int)fwd.h.size()};
  if (rev) rev->beg = {0, (int)rev->h.size()};
}

// Work lists of one stage (st.level, st.type, st.procs.h set): tiles or scan chunks, overlap-save blocks, or LTI
// groups with their FFT scratch offsets (groups under the workspace limit when the spectra are not kept).
mg_status make_stage(mg_console* c, Stage& st) {
  const int t = st.type;
  const int64_t limit = c->desc.workspace_limit_bytes > 0 ? c->desc.workspace_limit_bytes : INT64_MAX;
  if (t == T_G || t == T_S || t == T_C || t == T_N) {
    for (int pi : st.procs.h) {
      st.elem.beg.push_back((int)st.elem.h.size());
      st.elem_rev.beg.push_back((int)st.elem_rev.h.size());
      const int nt = (t == T_C || t == T_N) ? c->procs[pi].nchunks : c->procs[pi].nbrows;
      for (int i = 0; i < nt; ++i) st.elem.h.push_back(Item{pi, i});
      if (t == T_C || t == T_N)
        for (int i = nt - 1; i >= 0; --i) st.elem_rev.h.push_back(Item{pi, i});
    }
    st.elem.beg.push_back((int)st.elem.h.size());
    st.elem_rev.beg.push_back((int)st.elem_rev.h.size());
    if (t == T_C || t == T_N)
      chain_rounds(st.procs.h, [&](int pi) { return c->procs[pi].nchunks; }, st.chain_f, &st.chain_b);
    if (upload_items(c, st.elem) || upload_items(c, st.elem_rev) || upload_items(c, st.chain_f) ||
        upload_items(c, st.chain_b) || upload_procs(c, st.procs))
      return MG_ERR_CUDA;
  } else if (t == T_E) {
    // equalizer: overlap-save blocks (forward and backward blockings differ)
    for (int pi : st.procs.h) {
      st.osf.beg.push_back((int)st.osf.h.size());
      st.osb.beg.push_back((int)st.osb.h.size());
      for (int i = 0; i < c->procs[pi].nfrows; ++i) st.osf.h.push_back(Item{pi, i});
      for (int i = 0; i < c->procs[pi].nbrows; ++i) st.osb.h.push_back(Item{pi, i});
    }
    st.osf.beg.push_back((int)st.osf.h.size());
    st.osb.beg.push_back((int)st.osb.h.size());
    if (upload_items(c, st.osf) || upload_items(c, st.osb) || upload_procs(c, st.procs)) return MG_ERR_CUDA;
  } else {
    // LTI: groups under the workspace limit, each with its own scratch offsets
    size_t used = 0;
    LtiGroup g;
    auto close = [&]() -> mg_status {
      if (g.procs.h.empty()) return MG_OK;
      for (ItemList* L : {&g.col, &g.rowpair, &g.firtaps, &g.dlyadj, &g.revfir})
        L->beg.push_back((int)L->h.size());
      if (upload_procs(c, g.procs) || upload_items(c, g.col) ||
          upload_items(c, g.rowpair) || upload_items(c, g.firtaps) || upload_items(c, g.dlyadj) ||
          upload_items(c, g.revfir))
        return MG_ERR_CUDA;
      st.groups.push_back(g);
      g = LtiGroup{};
      used = 0;
      return MG_OK;
    };
    for (int pi : st.procs.h) {
      HostProc& p = c->procs[pi];
      if (!c->retain) {   // retained spectra: the offsets fixed at creation, one group per stage
        if (used > 0 && (int64_t)(used + p.scratch_bytes) > limit)
          if (close() != MG_OK) return MG_ERR_CUDA;
        p.o_scratch = used;
        used += p.scratch_bytes;
      }
      ProcDev& d = c->hpd[pi];
      const size_t N = (size_t)p.f << p.logN;
      d.T1 = (float2*)(c->scratch + p.o_scratch);
      d.T2 = d.T1 + N;
      d.Hz = d.T2 + N;
      g.procs.h.push_back(pi);
      const int N1 = p.f << p.logN1, N2 = 1 << p.logN2;
      for (ItemList* L : {&g.col, &g.rowpair, &g.firtaps, &g.dlyadj, &g.revfir})
        L->beg.push_back((int)L->h.size());
      for (int i = 0; i < N1 / p.colG; ++i) g.col.h.push_back(Item{pi, i});
      g.col.maxv = std::max(g.col.maxv, N2 * p.colG);
      for (int i = 0; i <= N2 / 2; ++i) g.rowpair.h.push_back(Item{pi, i});
      g.rowpair.maxv = std::max(g.rowpair.maxv, N1);
      if (t == T_D) {
        for (int i = 0; i < (p.Nh + 255) / 256; ++i) g.firtaps.h.push_back(Item{pi, i});
        for (int i = 0; i < 2 * kDlyTaps; ++i) g.dlyadj.h.push_back(Item{pi, i});
      }
      if (t == T_R) {
        const int ng = (p.nframes + kRevFG - 1) / kRevFG;
        for (int i = 0; i < ng; ++i) g.revfir.h.push_back(Item{pi, i});
      }
    }
    if (close() != MG_OK) return MG_ERR_CUDA;
  }
  return MG_OK;
}

// Pointers of the node table for the current structure (present processors), stage lists and launch lists.
mg_status build_tables(mg_console* c) {
  if (c->is_graph) return build_graph_tables(c);
  auto A = [&](size_t off) { return c->arena + off; };
  c->hpd.assign(c->P, ProcDev{});
  // forward / backward wiring per chain
  std::vector<size_t> chain_out(c->chains.size());
  for (size_t ci = 0; ci < c->chains.size(); ++ci) {
    const HostChain& ch = c->chains[ci];
    size_t cur = ch.o_in;
    for (int pi : ch.procs) {
      HostProc& p = c->procs[pi];
      ProcDev& d = c->hpd[pi];
      d.present = p.present;
      if (!p.present) continue;
      d.u = (const float*)A(cur);
      d.y = (float*)A(p.o_y);
      cur = p.o_y;
    }
    chain_out[ci] = cur;
  }
  c->chain_out = chain_out;
  // adjoints: chain output adjoint
  std::vector<size_t> chain_dout(c->chains.size()), chain_din(c->chains.size());
  for (int level = 1; level >= 0; --level) {
    for (size_t ci = 0; ci < c->chains.size(); ++ci) {
      const HostChain& ch = c->chains[ci];
      if (ch.level != level) continue;
      const HostSong& s = c->songs[ch.song];
      size_t dout = s.o_dmix;
      if (level == 0 && s.group[ch.index] >= 0) dout = chain_din[s.groups_chain[s.group[ch.index]]];
      chain_dout[ci] = dout;
      size_t cur = dout;
      bool useA = true;
      for (int k = (int)ch.procs.size() - 1; k >= 0; --k) {
        const int pi = ch.procs[k];
        if (!c->procs[pi].present) continue;
        ProcDev& d = c->hpd[pi];
        d.dy = (const float*)A(cur);
        const size_t nxt = useA ? ch.o_dA : ch.o_dB;
        d.du = (float*)A(nxt);
        cur = nxt;
        useA = !useA;
      }
      chain_din[ci] = cur;
    }
  }
  for (int pi = 0; pi < c->P; ++pi) fill_procdev(c, pi);
  if (attach_dyn_maps(c) != MG_OK || upload(c, c->hpd, &c->d_procs) != MG_OK) return MG_ERR_CUDA;

  // sums: m per subgroup (level 1 inputs), o per song
  c->sum_out.h.clear(); c->sum_in.h.clear(); c->sum_beg.h.clear(); c->sum_L.h.clear(); c->sum_ld.h.clear();
  c->sum_m_items = ItemList{}; c->sum_o_items = ItemList{};
  int sid = 0;
  auto add_sum = [&](size_t out, const std::vector<size_t>& ins, int L, int ld, ItemList& items) {
    c->sum_beg.h.push_back((int)c->sum_in.h.size());
    c->sum_out.h.push_back((float*)A(out));
    for (size_t o : ins) c->sum_in.h.push_back((const float*)A(o));
    c->sum_L.h.push_back(L);
    c->sum_ld.h.push_back(ld);
    items.beg.push_back((int)items.h.size());
    for (int t = 0; t < (L + c->elem_tile - 1) / c->elem_tile; ++t) items.h.push_back(Item{sid, t});
    ++sid;
  };
  for (auto& s : c->songs)
    for (int g = 0; g < s.S; ++g) {
      std::vector<size_t> ins;
      for (int k = 0; k < s.K; ++k)
        if (s.group[k] == g) ins.push_back(chain_out[s.tracks_chain[k]]);
      add_sum(c->chains[s.groups_chain[g]].o_in, ins, s.L, s.ld, c->sum_m_items);
    }
  c->sum_m_items.beg.push_back((int)c->sum_m_items.h.size());
  for (auto& s : c->songs) {
    std::vector<size_t> ins;
    for (int g = 0; g < s.S; ++g) ins.push_back(chain_out[s.groups_chain[g]]);
    for (int k = 0; k < s.K; ++k)
      if (s.group[k] < 0) ins.push_back(chain_out[s.tracks_chain[k]]);
    add_sum(s.o_mix, ins, s.L, s.ld, c->sum_o_items);
  }
  c->sum_o_items.beg.push_back((int)c->sum_o_items.h.size());
  c->sum_beg.h.push_back((int)c->sum_in.h.size());
  if (upload(c, c->sum_out.h, &c->sum_out.d) || upload(c, c->sum_in.h, &c->sum_in.d) ||
      upload(c, c->sum_beg.h, &c->sum_beg.d) || upload(c, c->sum_L.h, &c->sum_L.d) ||
      upload(c, c->sum_ld.h, &c->sum_ld.d) || upload_items(c, c->sum_m_items) || upload_items(c, c->sum_o_items))
    return MG_ERR_CUDA;

  // stages in console order: level 0 types e..r, level 1 types e..r
  c->stages.clear();
  c->all_present = ProcList{};
  c->all_lti_present = ProcList{};
  const int64_t limit = c->desc.workspace_limit_bytes > 0 ? c->desc.workspace_limit_bytes : INT64_MAX;
  for (int level = 0; level < 2; ++level)
    for (int t = 0; t < NTYPES; ++t) {
      Stage st;
      st.level = level;
      st.type = t;
      for (int pi = 0; pi < c->P; ++pi) {
        const HostProc& p = c->procs[pi];
        if (p.level != level || p.type != t || !p.present) continue;
        st.procs.h.push_back(pi);
        c->all_present.h.push_back(pi);
        if (t == T_E || t == T_R || t == T_D) c->all_lti_present.h.push_back(pi);
      }
      if (st.procs.h.empty()) continue;
      if (make_stage(c, st) != MG_OK) return MG_ERR_CUDA;
      c->stages.push_back(st);
    }
  // scratch pointers changed with grouping: re-upload the node table
  if (attach_dyn_maps(c) != MG_OK || upload(c, c->hpd, &c->d_procs) != MG_OK) return MG_ERR_CUDA;
  if (upload_procs(c, c->all_present) || upload_procs(c, c->all_lti_present)) return MG_ERR_CUDA;
  return MG_OK;
}

// Graph wiring (Alg. 1: gather, aggregate, process, store).  A node's input is its one predecessor's output in
// place, or the sum of its predecessors' outputs (an aggregation sum in the node's step); an input node's output
// is its track's source, a mix node's its input, a processor's its own buffer (its input when removed by
// pruning), and the output node's sum is the song's mix.  In the backward pass the adjoint of a node's output is
// its one successor's input adjoint in place, or the sum of its successors' input adjoints (an adjoint sum in
// the node's step), or zero when nothing reads it; a processor writes its own input adjoint, a mix node passes
// its output adjoint through, the output node's input adjoint is the mix adjoint.  Sums read their inputs in
// edge order.  Stages are the schedule's processor steps.
mg_status build_graph_tables(mg_console* c) {
  auto A = [&](size_t off) { return c->arena + off; };
  const HostSong& hs = c->songs[0];
  const int n = (int)c->gn.size();
  c->hpd.assign(c->P, ProcDev{});
  for (int pi = 0; pi < c->P; ++pi) fill_procdev(c, pi);
  c->sum_out.h.clear(); c->sum_in.h.clear(); c->sum_beg.h.clear(); c->sum_L.h.clear(); c->sum_ld.h.clear();
  const int nsteps = (int)c->gstep_type.size();
  c->gstep_fsum.assign(nsteps, ItemList{});
  c->gstep_bsum.assign(nsteps, ItemList{});
  c->gstep_stage.assign(nsteps, -1);
  int sid = 0;
  auto add_sum = [&](size_t out, const std::vector<size_t>& ins, ItemList& items) {
    c->sum_beg.h.push_back((int)c->sum_in.h.size());
    c->sum_out.h.push_back((float*)A(out));
    for (size_t o : ins) c->sum_in.h.push_back((const float*)A(o));
    c->sum_L.h.push_back(hs.L);
    c->sum_ld.h.push_back(hs.ld);
    items.beg.push_back((int)items.h.size());
    for (int t = 0; t < (hs.L + c->elem_tile - 1) / c->elem_tile; ++t) items.h.push_back(Item{sid, t});
    ++sid;
  };
  // forward: outputs in schedule order
  std::vector<size_t> out(n, 0), in(n, 0);
  for (int k = 0; k < nsteps; ++k)
    for (int v : c->gstep_nodes[k]) {
      GNode& g = c->gn[v];
      if (g.type == MG_NODE_INPUT) {
        out[v] = c->o_src[g.track];
        continue;
      }
      std::vector<size_t> ins;
      for (int u : g.preds) ins.push_back(out[u]);
      if (g.type == MG_NODE_OUTPUT) {
        add_sum(hs.o_mix, ins, c->gstep_fsum[k]);
        continue;
      }
      in[v] = g.preds.size() == 1 ? out[g.preds[0]] : g.o_agg;
      if (g.preds.size() > 1) add_sum(g.o_agg, ins, c->gstep_fsum[k]);
      if (g.type == MG_NODE_MIX) {
        out[v] = in[v];
        continue;
      }
      HostProc& p = c->procs[g.proc];
      ProcDev& d = c->hpd[g.proc];
      d.present = p.present;
      out[v] = p.present ? p.o_y : in[v];
      d.u = (const float*)A(in[v]);
      d.y = (float*)A(p.o_y);
    }
  // backward: input adjoints in reverse schedule order
  std::vector<size_t> din(n, 0), dout(n, 0);
  for (int k = nsteps - 1; k >= 0; --k)
    for (int v : c->gstep_nodes[k]) {
      GNode& g = c->gn[v];
      if (g.type == MG_NODE_OUTPUT) {
        din[v] = hs.o_dmix;
        continue;
      }
      if (g.type == MG_NODE_INPUT) continue;
      if (g.succs.empty()) {
        dout[v] = c->o_zero;
      } else if (g.succs.size() == 1) {
        dout[v] = din[g.succs[0]];
      } else {
        std::vector<size_t> ins;
        for (int w : g.succs) ins.push_back(din[w]);
        add_sum(g.o_dsum, ins, c->gstep_bsum[k]);
        dout[v] = g.o_dsum;
      }
      if (g.type == MG_NODE_MIX) {
        din[v] = dout[v];
        continue;
      }
      const HostProc& p = c->procs[g.proc];
      ProcDev& d = c->hpd[g.proc];
      din[v] = p.present ? g.o_du : dout[v];
      d.dy = (const float*)A(dout[v]);
      d.du = (float*)A(g.o_du);
    }
  c->sum_beg.h.push_back((int)c->sum_in.h.size());
  if (upload(c, c->sum_out.h, &c->sum_out.d) || upload(c, c->sum_in.h, &c->sum_in.d) ||
      upload(c, c->sum_beg.h, &c->sum_beg.d) || upload(c, c->sum_L.h, &c->sum_L.d) ||
      upload(c, c->sum_ld.h, &c->sum_ld.d))
    return MG_ERR_CUDA;
  for (int k = 0; k < nsteps; ++k) {
    c->gstep_fsum[k].beg.push_back((int)c->gstep_fsum[k].h.size());
    c->gstep_bsum[k].beg.push_back((int)c->gstep_bsum[k].h.size());
    if (upload_items(c, c->gstep_fsum[k]) || upload_items(c, c->gstep_bsum[k])) return MG_ERR_CUDA;
  }
  // stages: the present processors of every processor step
  c->stages.clear();
  c->all_present = ProcList{};
  c->all_lti_present = ProcList{};
  for (int pi = 0; pi < c->P; ++pi)
    if (c->procs[pi].present) {
      c->all_present.h.push_back(pi);
      const int t = c->procs[pi].type;
      if (t == T_E || t == T_R || t == T_D) c->all_lti_present.h.push_back(pi);
    }
  for (int k = 0; k < nsteps; ++k) {
    if (c->gstep_type[k] >= NTYPES) continue;
    Stage st;
    st.level = k;
    st.type = c->gstep_type[k];
    for (int v : c->gstep_nodes[k])
      if (c->procs[c->gn[v].proc].present) st.procs.h.push_back(c->gn[v].proc);
    if (st.procs.h.empty()) continue;
    if (make_stage(c, st) != MG_OK) return MG_ERR_CUDA;
    c->gstep_stage[k] = (int)c->stages.size();
    c->stages.push_back(st);
  }
  if (attach_dyn_maps(c) != MG_OK || upload(c, c->hpd, &c->d_procs) != MG_OK) return MG_ERR_CUDA;
  if (upload_procs(c, c->all_present) || upload_procs(c, c->all_lti_present)) return MG_ERR_CUDA;
  return MG_OK;
}

// Host-only sizing: arena offsets of every song, chain and processor buffer, and the two LTI scratch sizes
// (one group's shared scratch, and the retained per-node spectra).  Returns the arena size in bytes.
size_t layout_arena(mg_console* c, const mg_console_desc* d, size_t* shared_scratch, size_t* keep_scratch) {
  Bump b;
  for (auto& hs : c->songs) {
    const size_t st = (size_t)2 * hs.ld * sizeof(float);
    hs.o_mix = b.take(st);
    hs.o_dmix = b.take(st);
    hs.o_tgt = b.take(st);
    for (int r = 0; r < c->nres; ++r) {
      const int nf = d->n_fft[r], hop = nf / d->hop_div;
      hs.nframes[r] = hs.L >= nf ? (hs.L - nf) / hop + 1 : 0;
      hs.first[r] = std::min(hs.nframes[r], (int)((d->warmup_samples + hop - 1) / hop));
      if (c->loss_per[r] <= 0) c->loss_per[r] = 8192 / nf;
      const int per = c->loss_per[r], per_min = std::max(1, 8192 / nf / kLossPerDiv);
      hs.litems[r] = (hs.nframes[r] - hs.first[r] + per - 1) / per;
      hs.lcap = std::max(hs.lcap, (hs.nframes[r] - hs.first[r] + per_min - 1) / per_min);   // every candidate
      const int nbands = d->n_mels > 0 ? d->n_mels : nf / 2 + 1;
      hs.o_Y[r] = b.take((size_t)std::max(1, hs.nframes[r]) * nbands * 4 * sizeof(float));
      hs.o_Yh[r] = b.take((size_t)std::max(1, hs.nframes[r]) * nbands * 4 * sizeof(float));
      hs.o_dF[r] = b.take((size_t)std::max(1, hs.nframes[r]) * nf * sizeof(float2));
    }
    hs.o_lpart = b.take((size_t)3 * std::max(1, hs.lcap) * 6 * sizeof(float));
    hs.o_coef = b.take(18 * sizeof(float));
    hs.o_ynorm = b.take(9 * sizeof(double));
  }
  for (auto& ch : c->chains) {
    const size_t st = (size_t)2 * ch.ld * sizeof(float);
    ch.o_in = b.take(st);
    ch.o_dA = b.take(st);
    ch.o_dB = b.take(st);
  }
  size_t scratch_need = 0;
  for (auto& p : c->procs) {
    p.o_y = b.take((size_t)2 * p.ld * sizeof(float));
    p.o_stats = b.take(kStatsFloats * sizeof(float));
    if (p.nfrows) p.o_fpart = b.take((size_t)std::max(p.nfrows, p.nfcap) * kNPart * sizeof(float));
    if (p.nbrows) p.o_bpart = b.take((size_t)std::max(p.nbrows, p.nfcap) * kNPart * sizeof(float));
    if (p.type == T_E || p.type == T_R || p.type == T_D) {
      p.o_taps = b.take((size_t)2 * p.Nh * sizeof(float));
      p.o_dtaps = b.take((size_t)2 * p.Nh * sizeof(float));
      scratch_need = std::max(scratch_need, p.scratch_bytes);
    }
    if (p.type == T_E) {
      p.o_hspec = b.take((size_t)kEqOsM * sizeof(float));
      p.o_ybar = b.take((size_t)2 * p.ld * sizeof(float));
      p.o_dhspec = b.take((size_t)p.nbrows * kEqOsM * sizeof(float2));
      p.o_eqg = b.take((size_t)p.nfrows * kEqOsM * sizeof(float2));
    }
    if (p.type == T_D) p.o_aux = b.take((2 * kDlyTaps * kDlyFir + 2 * kDlyTaps) * sizeof(float));
    if (p.type == T_C || p.type == T_N) p.o_aux = b.take((size_t)p.ld * sizeof(float));   // dL/dg per sample
    if (p.type == T_R) {
      const int ng = (p.nframes + kRevFG - 1) / kRevFG;
      p.o_aux = b.take((size_t)2 * ng * kRevBins * 2 * sizeof(float));
      p.o_nspec = b.take((size_t)2 * p.nframes * kRevBins * sizeof(float2));
    }
    if (p.nchunks) {
      p.o_cflag = b.take(p.nchunks * sizeof(unsigned long long));
      p.o_carry = b.take(p.nchunks * sizeof(float));
      p.o_cagg = b.take(p.nchunks * sizeof(float));
    }
  }
  if (c->is_graph) {
    const size_t st = (size_t)2 * c->songs[0].ld * sizeof(float);
    c->o_src.assign(c->songs[0].K, 0);
    for (auto& o : c->o_src) o = b.take(st);
    c->o_zero = b.take(st);
    for (auto& v : c->gn) {
      const bool proc = v.type < NTYPES;
      if ((proc || v.type == MG_NODE_MIX) && v.preds.size() > 1) v.o_agg = b.take(st);
      if (v.type != MG_NODE_INPUT && v.type != MG_NODE_OUTPUT && v.succs.size() > 1) v.o_dsum = b.take(st);
      if (proc) v.o_du = b.take(st);
    }
  }
  const int64_t limit = d->workspace_limit_bytes > 0 ? d->workspace_limit_bytes : INT64_MAX;
  size_t worst = 0;
  int levels = 2;
  for (auto& p : c->procs) levels = std::max(levels, p.level + 1);
  for (int level = 0; level < levels; ++level)
    for (int t : {T_R, T_D}) {
      size_t used = 0;
      for (auto& p : c->procs) {
        if (p.level != level || p.type != t) continue;
        if (used > 0 && (int64_t)(used + p.scratch_bytes) > limit) used = 0;
        used += p.scratch_bytes;
        worst = std::max(worst, used);
      }
    }
  size_t keep = 0;
  for (auto& p : c->procs)
    if (p.type == T_R || p.type == T_D) keep += p.scratch_bytes;
  *shared_scratch = std::max(worst, scratch_need);
  *keep_scratch = std::max(keep, scratch_need);
  return b.off;
}

// Device bytes of a console with the given scratch choice: arena, LTI scratch, parameters, gradients and the
// two Adam moments.
size_t console_device_bytes(const mg_console* c, size_t arena, size_t scratch) {
  return arena + scratch + 4 * sizeof(float) * (size_t)c->nparams;
}

// Autotuner of the FFT convolution split: for every size class (f, logN) of the reverb / delay nodes, one node
// of the class runs its forward and backward passes (filter spectrum, input spectrum, product, inverse, dL/dy_bar,
// backward rows, du, dL/dh) under each candidate split; the fastest (minimum of three timed repetitions after
// one warm-up) is applied to the whole class.  The buffers hold whatever the console holds at that point; the
// passes do the same work for any values.
mg_status autotune_splits(mg_console* c) {
  std::vector<std::pair<int, int>> classes;
  std::vector<int> rep_of;
  for (int pi = 0; pi < c->P; ++pi) {
    const HostProc& p = c->procs[pi];
    if ((p.type != T_R && p.type != T_D) || p.splits.size() < 2) continue;
    const auto key = std::make_pair(p.f, p.logN);
    if (std::find(classes.begin(), classes.end(), key) == classes.end()) {
      classes.push_back(key);
      rep_of.push_back(pi);
    }
  }
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  LaunchCtx x = make_ctx(c, nullptr);
  // With retained spectra every node owns its FFT buffers, so up to kTuneNodes nodes of a size class are timed
  // together: launches of many nodes run at the throughput of the real stage launches, where one node's
  // launches (a wave or two of CTAs) would be dominated by their tails.  Without retained spectra the nodes
  // share one scratch, so one node is timed.
  constexpr int kTuneNodes = 16;
  for (size_t k = 0; k < classes.size(); ++k) {
    const int pi = rep_of[k];
    HostProc& p = c->procs[pi];
    const HostProc saved = p;
    std::vector<int> members{pi};
    for (int qi = 0; c->retain && qi < c->P && (int)members.size() < kTuneNodes; ++qi) {
      const HostProc& q = c->procs[qi];
      if (qi != pi && (q.type == T_R || q.type == T_D) && q.f == p.f && q.logN == p.logN) members.push_back(qi);
    }
    int best = p.logN1;
    float best_ms = 1e30f;
    for (int l1 : saved.splits) {
      ItemList col, pair;
      for (int mi : members) {
        HostProc& m = c->procs[mi];
        apply_split(m, l1);
        ProcDev& dv = c->hpd[mi];
        dv.logN1 = m.logN1;
        dv.logN2 = m.logN2;
        dv.colG = m.colG;
        dv.nfpart = m.nfrows;
        dv.nbpart = m.nbrows;
        CK(cudaMemcpyAsync(c->d_procs + mi, &dv, sizeof(ProcDev), cudaMemcpyHostToDevice, c->stream));
        for (int i = 0; i < m.nfrows; ++i) col.h.push_back(Item{mi, i});
        for (int i = 0; i <= (1 << m.logN2) / 2; ++i) pair.h.push_back(Item{mi, i});
      }
      if (upload_items(c, col) || upload_items(c, pair)) return MG_ERR_CUDA;
      const int n2g = (1 << p.logN2) * p.colG, n1 = p.f << p.logN1, nc = (int)col.h.size(), np_ = (int)pair.h.size();
      auto passes = [&] {
        launch_col_fwd_taps(x, col.d, nc, n2g);
        launch_row_fwd_hz(x, pair.d, np_, n1);
        launch_col_fwd_audio(x, col.d, nc, n2g);
        launch_row_conv_fwd(x, pair.d, np_, n1, c->retain);
        if (c->retain) launch_col_inv_out_keep(x, col.d, nc, n2g);
        else launch_col_inv_out(x, col.d, nc, n2g);
        if (c->retain) {
          launch_col_dybar_keep(x, col.d, nc, n2g);
        } else {
          launch_col_fwd_taps(x, col.d, nc, n2g);
          launch_row_fwd_hz(x, pair.d, np_, n1);
          launch_col_fwd_audio(x, col.d, nc, n2g);
          launch_row_conv_fwd(x, pair.d, np_, n1, true);
          launch_col_dybar(x, col.d, nc, n2g);
        }
        launch_row_bwd2(x, pair.d, np_, n1);
        launch_col_du(x, col.d, nc, n2g);
        launch_col_dh(x, col.d, nc, n2g);
      };
      passes();
      float ms = 1e30f;
      for (int r = 0; r < 3; ++r) {
        CK(cudaEventRecord(e0, c->stream));
        passes();
        CK(cudaEventRecord(e1, c->stream));
        CK(cudaEventSynchronize(e1));
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, e0, e1));
        ms = std::min(ms, t);
      }
      CK(cudaGetLastError());
      if (ms < best_ms) {
        best_ms = ms;
        best = l1;
      }
    }
    p = saved;
    for (HostProc& q : c->procs)
      if ((q.type == T_R || q.type == T_D) && q.f == classes[k].first && q.logN == classes[k].second) apply_split(q, best);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // the arena is untouched (partial sums sized for every candidate); the node table and work lists follow the
  // chosen splits
  for (int pi = 0; pi < c->P; ++pi) {
    const HostProc& p = c->procs[pi];
    if (p.type != T_R && p.type != T_D) continue;
    ProcDev& dv = c->hpd[pi];
    dv.logN1 = p.logN1;
    dv.logN2 = p.logN2;
    dv.colG = p.colG;
    dv.nfpart = p.nfrows;
    dv.nbpart = p.nbrows;
  }
  if (build_tables(c) != MG_OK) return MG_ERR_CUDA;
  CK(cudaStreamSynchronize(c->stream));
  return MG_OK;
}

// Loss work items for the current frames per item (song-major within each resolution, so one song's items are
// one contiguous range), with the per-song item counts and the resolutions' item length on the device.
mg_status build_loss_items(mg_console* c) {
  c->song_litems.assign(c->songs.size(), std::array<int2, 3>{});
  for (int r = 0; r < c->nres; ++r) {
    auto& L = c->loss_items[r];
    L.h.clear();
    const int per = c->loss_per[r];
    c->hres[r].per = per;
    for (size_t si = 0; si < c->songs.size(); ++si) {
      HostSong& hs = c->songs[si];
      const int first = (int)L.h.size();
      for (int t = hs.first[r]; t < hs.nframes[r]; t += per)
        L.h.push_back(make_int4((int)si, r, t, std::min(per, hs.nframes[r] - t)));
      c->song_litems[si][r] = make_int2(first, (int)L.h.size() - first);
      hs.litems[r] = (int)L.h.size() - first;
      c->hsd[si].litems[r] = hs.litems[r];
    }
    if (upload(c, L.h, &L.d) != MG_OK) return MG_ERR_CUDA;
  }
  if (upload(c, c->hsd, &c->d_songs) != MG_OK || upload(c, c->hres, &c->d_res) != MG_OK) return MG_ERR_CUDA;
  return MG_OK;
}

// Packing tuner: the samples per work item (one CTA) of the gain/pan and imager kernels and of the sums, which
// decides how the nodes of those stages are cut into CTAs.  Every candidate from kElemTileMin to 16384 samples runs
// the forward and backward launches of those stages and the sums over all nodes (the minimum of three timed
// repetitions after one warm-up) on the console's own buffers; the fastest is kept.  The arena holds the partial
// sums of the smallest tile, so every candidate fits.
mg_status autotune_packing(mg_console* c) {
  bool any = false;
  for (const auto& p : c->procs) any = any || p.type == T_G || p.type == T_S;
  if (!any) return MG_OK;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int best = c->elem_tile;
  float best_ms = 1e30f;
  auto set_tile = [&](int tile) -> mg_status {
    c->elem_tile = tile;
    for (auto& p : c->procs)
      if (p.type == T_G || p.type == T_S) p.nbrows = (p.L + tile - 1) / tile;
    return build_tables(c);
  };
  for (int tile = kElemTileMin; tile <= 16384; tile *= 2) {
    if (set_tile(tile) != MG_OK) return MG_ERR_CUDA;
    LaunchCtx x = make_ctx(c, nullptr);
    auto pass = [&] {
      for (auto& st : c->stages)
        if (st.type == T_G || st.type == T_S) {
          stage_forward(c, x, st);
          stage_backward(c, x, st);
        }
      if (c->is_graph) {
        for (size_t k = 0; k < c->gstep_fsum.size(); ++k) {
          run_sums(c, c->gstep_fsum[k]);
          run_sums(c, c->gstep_bsum[k]);
        }
      } else {
        run_sums(c, c->sum_m_items);
        run_sums(c, c->sum_o_items);
      }
    };
    pass();
    float ms = 1e30f;
    for (int r = 0; r < 3; ++r) {
      CK(cudaEventRecord(e0, c->stream));
      pass();
      CK(cudaEventRecord(e1, c->stream));
      CK(cudaEventSynchronize(e1));
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, e0, e1));
      ms = std::min(ms, t);
    }
    CK(cudaGetLastError());
    if (ms < best_ms) {
      best_ms = ms;
      best = tile;
    }
  }
  if (set_tile(best) != MG_OK) return MG_ERR_CUDA;
  // frames per loss work item: 8192 / n_fft (one 8192-point buffer per CTA), half or a quarter of it; the loss
  // forward and its adjoint over all songs
  int best_div = 1;
  best_ms = 1e30f;
  auto set_div = [&](int div) -> mg_status {
    for (int r = 0; r < c->nres; ++r) c->loss_per[r] = std::max(1, 8192 / c->hres[r].nfft / div);
    return build_loss_items(c);
  };
  for (int div = 1; div <= kLossPerDiv; div *= 2) {
    if (set_div(div) != MG_OK) return MG_ERR_CUDA;
    LaunchCtx x = make_ctx(c, nullptr);
    auto pass = [&] {
      for (int r = 0; r < c->nres; ++r) {
        auto& L = c->loss_items[r];
        if (L.h.empty()) continue;
        launch_loss_frames(x, c->d_songs, c->d_res, L.d, (int)L.h.size(), 1, c->loss_max_dy);
        launch_loss_frames(x, c->d_songs, c->d_res, L.d, (int)L.h.size(), 2, c->loss_max_dy);
      }
    };
    pass();
    float ms = 1e30f;
    for (int r = 0; r < 3; ++r) {
      CK(cudaEventRecord(e0, c->stream));
      pass();
      CK(cudaEventRecord(e1, c->stream));
      CK(cudaEventSynchronize(e1));
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, e0, e1));
      ms = std::min(ms, t);
    }
    CK(cudaGetLastError());
    if (ms < best_ms) {
      best_ms = ms;
      best_div = div;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (set_div(best_div) != MG_OK) return MG_ERR_CUDA;
  CK(cudaStreamSynchronize(c->stream));
  return MG_OK;
}

mg_status create_impl(mg_console* c, const mg_console_desc* d, const mg_song_desc* s, int n) {
  if (!c->is_graph) plan(c, d, s, n);
  init_kernel_attributes();
  init_loss_attributes();
  init_fir_attributes();
  init_eqos_attributes();
  init_eval_attributes();
  const double fs = d->sample_rate;
  // ---- arena layout and LTI scratch ----
  size_t shared_scratch = 0, keep_scratch = 0;
  const size_t arena = layout_arena(c, d, &shared_scratch, &keep_scratch);
  {
    // retained spectra: every reverb/delay node gets its own T1 / T2 / Hz for the whole step
    const int64_t limit = d->workspace_limit_bytes > 0 ? d->workspace_limit_bytes : INT64_MAX;
    bool retain = d->retain_spectra == 1;
    if (d->retain_spectra == 0 && (int64_t)keep_scratch <= limit) {
      retain = keep_scratch <= shared_scratch;   // costs no memory beyond the shared scratch
      if (!retain) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return MG_ERR_CUDA;
        const size_t others = console_device_bytes(c, arena, 0) + ((size_t)256 << 20);
        retain = free_b > others && (double)keep_scratch <= 0.8 * (double)(free_b - others);
      }
    }
    c->retain = retain;
    c->scratch_bytes = shared_scratch;
    if (retain) {
      size_t off = 0;
      for (auto& p : c->procs)
        if (p.type == T_R || p.type == T_D) {
          p.o_scratch = off;
          off += p.scratch_bytes;
        }
      c->scratch_bytes = keep_scratch;
    }
  }
  c->arena_bytes = arena;
  // ---- allocations ----
  CK(cudaMalloc(&c->arena, c->arena_bytes));
  CK(cudaMemsetAsync(c->arena, 0, c->arena_bytes, c->stream));
  if (c->scratch_bytes) CK(cudaMalloc(&c->scratch, c->scratch_bytes));
  CK(cudaMalloc(&c->d_params, sizeof(float) * c->nparams));
  CK(cudaMalloc(&c->d_grads, sizeof(float) * c->nparams));
  CK(cudaMalloc(&c->d_m, sizeof(float) * c->nparams));
  CK(cudaMalloc(&c->d_v, sizeof(float) * c->nparams));
  CK(cudaMalloc(&c->d_step, sizeof(int)));
  CK(cudaMalloc(&c->d_hyper, 8 * sizeof(float)));
  CK(cudaMalloc(&c->d_alphas, 4 * sizeof(float)));
  CK(cudaMalloc(&c->d_mask, std::max(1, c->P)));
  CK(cudaMalloc(&c->d_scratch_la, sizeof(float) * std::max<size_t>(1, c->songs.size())));
  CK(cudaMalloc(&c->d_chain, 2 * sizeof(unsigned)));
  CK(cudaMemsetAsync(c->d_chain, 0, 2 * sizeof(unsigned), c->stream));
  CK(cudaHostAlloc(&c->h_err, sizeof(int), cudaHostAllocMapped));
  *c->h_err = 0;
  CK(cudaHostGetDevicePointer(&c->d_err, c->h_err, 0));
  CK(cudaMemsetAsync(c->d_params, 0, sizeof(float) * c->nparams, c->stream));
  CK(cudaMemsetAsync(c->d_grads, 0, sizeof(float) * c->nparams, c->stream));
  CK(cudaMemsetAsync(c->d_m, 0, sizeof(float) * c->nparams, c->stream));
  CK(cudaMemsetAsync(c->d_v, 0, sizeof(float) * c->nparams, c->stream));
  CK(cudaMemsetAsync(c->d_step, 0, sizeof(int), c->stream));
  CK(cudaMemsetAsync(c->d_hyper, 0, 8 * sizeof(float), c->stream));
  {
    const float al[4] = {d->alpha_lr, d->alpha_m, d->alpha_s, 0.f};
    CK(cudaMemcpy(c->d_alphas, al, sizeof(al), cudaMemcpyHostToDevice));
  }
  // ---- tables ----
  auto up_table = [&](const void* h, size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
    cudaMemcpy(p, h, bytes, cudaMemcpyHostToDevice);
    c->table_allocs.push_back(p);
    return p;
  };
  {
    const double PI = 3.14159265358979323846;
    std::vector<float2> tw(kTwN);
    for (int j = 0; j < kTwN; ++j) tw[j] = make_float2((float)std::cos(2 * PI * j / kTwN), (float)-std::sin(2 * PI * j / kTwN));
    std::vector<float> ceq(kEqTaps), cdl(kDlyFir), hwin(kRevFft), heq(kEqTaps), hdl(kDlyFir);
    for (int m = 0; m < kEqTaps; ++m) ceq[m] = (float)std::cos(2 * PI * m / kEqTaps);
    for (int m = 0; m < kDlyFir; ++m) cdl[m] = (float)std::cos(2 * PI * m / kDlyFir);
    for (int j = 0; j < kRevFft; ++j) hwin[j] = (float)(0.5 * (1.0 - std::cos(2 * PI * j / kRevFft)));
    std::vector<float2> rcs(kRevFft);
    for (int m = 0; m < kRevFft; ++m) rcs[m] = make_float2((float)std::cos(2 * PI * m / kRevFft), (float)std::sin(2 * PI * m / kRevFft));
    for (int j = 0; j < kEqTaps; ++j) heq[j] = (float)(0.5 * (1.0 + std::cos(2 * PI * (j - kEqHalf) / (kEqTaps - 1))));
    for (int j = 0; j < kDlyFir; ++j) hdl[j] = (float)(0.5 * (1.0 + std::cos(2 * PI * (j - kDlyHalf) / (kDlyFir - 1))));
    const int D = (int)std::llround(0.1 * fs);
    std::vector<float2> dw(D);
    for (int q = 0; q < D; ++q) dw[q] = make_float2((float)std::cos(2 * PI * q / D), (float)std::sin(2 * PI * q / D));
    c->tab.tw = (const float2*)up_table(tw.data(), tw.size() * sizeof(float2));
    std::vector<float2> twf(kTwN);
    for (int j = 0; j < kTwN; ++j) {
      const double a = 2 * PI * j / (double)(1 << kTwFineLog);
      twf[j] = make_float2((float)std::cos(a), (float)-std::sin(a));
    }
    c->tab.twf = (const float2*)up_table(twf.data(), twf.size() * sizeof(float2));
    std::vector<float2> c3((kTwLog + 1) * 3);
    for (int a = 0; a <= kTwLog; ++a)
      for (int r = 0; r < 3; ++r) {
        const double ang = -2.0 * PI * r / (3.0 * std::ldexp(1.0, a));
        c3[a * 3 + r] = make_float2((float)std::cos(ang), (float)std::sin(ang));
      }
    c->tab.c3 = (const float2*)up_table(c3.data(), c3.size() * sizeof(float2));
    std::vector<float2> ptw(kPtwCount), ptw3(kPtw3Count), ptw5(kPtw5Count);
    for (int e = 0; e < kPtwCount; ++e) ptw[e] = tw[ptw_source(e)];
    // pass twiddles of the F 2^a-point transforms (layout of ptwf_base), in double then rounded
    auto fill_ptwf = [&](std::vector<float2>& t, int f, int max_a) {
      for (int a = 1; a <= max_a; ++a)
        for (int lp2 = 0; lp2 < a; lp2 += 4) {
          const int logr = std::min(4, a - lp2), p = f << lp2;
          for (int r = 0; r < logr; ++r)
            for (int k = 0; k < p; ++k) {
              const int64_t m = ((int64_t)k << r) << (a - lp2 - logr);
              const double ang = -2.0 * PI * (double)m / ((double)f * std::ldexp(1.0, a));
              t[ptwf_base(f, a, lp2) + r * p + k] = make_float2((float)std::cos(ang), (float)std::sin(ang));
            }
        }
    };
    fill_ptwf(ptw3, 3, kPtw3MaxA);
    fill_ptwf(ptw5, 5, kPtw5MaxA);
    c->tab.ptw = (const float2*)up_table(ptw.data(), ptw.size() * sizeof(float2));
    c->tab.ptw3 = (const float2*)up_table(ptw3.data(), ptw3.size() * sizeof(float2));
    c->tab.ptw5 = (const float2*)up_table(ptw5.data(), ptw5.size() * sizeof(float2));
    c->tab.cos_eq = (const float*)up_table(ceq.data(), ceq.size() * sizeof(float));
    c->tab.cos_dl = (const float*)up_table(cdl.data(), cdl.size() * sizeof(float));
    c->tab.rev_win = (const float*)up_table(hwin.data(), hwin.size() * sizeof(float));
    c->tab.rev_cs = (const float2*)up_table(rcs.data(), rcs.size() * sizeof(float2));
    c->tab.hann_eq = (const float*)up_table(heq.data(), heq.size() * sizeof(float));
    c->tab.hann_dl = (const float*)up_table(hdl.data(), hdl.size() * sizeof(float));
    c->tab.dly_w = (const float2*)up_table(dw.data(), dw.size() * sizeof(float2));
    if (!c->tab.tw || !c->tab.twf || !c->tab.c3 || !c->tab.ptw || !c->tab.ptw3 || !c->tab.ptw5 || !c->tab.dly_w)
      return fail(c, MG_ERR_OOM, "table allocation failed");
  }
  // loss resolutions
  c->hres.assign(c->nres, LossRes{});
  for (int r = 0; r < c->nres; ++r) {
    const int nf = d->n_fft[r], nb = nf / 2 + 1;
    LossRes& R = c->hres[r];
    R.nfft = nf;
    R.log_nfft = ilog2_ceil(nf);
    R.hop = nf / d->hop_div;
    R.per = c->loss_per[r];
    std::vector<float> win(nf), aw2(nb);
    const double PI = 3.14159265358979323846;
    for (int j = 0; j < nf; ++j) win[j] = (float)(0.5 * (1.0 - std::cos(2 * PI * j / nf)));
    for (int k = 0; k < nb; ++k) {
      const double a = d->a_weighting ? a_weight((double)k * fs / nf) : 1.0;
      aw2[k] = (float)(a * a);
    }
    std::vector<int> bb, bbin, kb, kband;
    std::vector<float> bw, kw;
    if (d->n_mels > 0) {
      std::vector<std::vector<double>> W;
      mel_bank(nf, d->n_mels, fs, W);
      R.nbands = d->n_mels;
      for (int b2 = 0; b2 < d->n_mels; ++b2) {
        bb.push_back((int)bbin.size());
        for (int k = 0; k < nb; ++k)
          if (W[b2][k] > 0) { bbin.push_back(k); bw.push_back((float)W[b2][k]); }
      }
      bb.push_back((int)bbin.size());
      for (int k = 0; k < nb; ++k) {
        kb.push_back((int)kband.size());
        for (int b2 = 0; b2 < d->n_mels; ++b2)
          if (W[b2][k] > 0) { kband.push_back(b2); kw.push_back((float)W[b2][k]); }
      }
      kb.push_back((int)kband.size());
    } else {
      R.nbands = nb;
      for (int k = 0; k < nb; ++k) { bb.push_back(k); bbin.push_back(k); bw.push_back(1.f); kb.push_back(k); kband.push_back(k); kw.push_back(1.f); }
      bb.push_back(nb);
      kb.push_back(nb);
    }
    if (bbin.empty()) { bbin.push_back(0); bw.push_back(0.f); }
    if (kband.empty()) { kband.push_back(0); kw.push_back(0.f); }
    R.win = (const float*)up_table(win.data(), win.size() * sizeof(float));
    R.aw2 = (const float*)up_table(aw2.data(), aw2.size() * sizeof(float));
    R.band_beg = (const int*)up_table(bb.data(), bb.size() * sizeof(int));
    R.band_bin = (const int*)up_table(bbin.data(), bbin.size() * sizeof(int));
    R.band_w = (const float*)up_table(bw.data(), bw.size() * sizeof(float));
    R.bin_beg = (const int*)up_table(kb.data(), kb.size() * sizeof(int));
    R.bin_band = (const int*)up_table(kband.data(), kband.size() * sizeof(int));
    R.bin_w = (const float*)up_table(kw.data(), kw.size() * sizeof(float));
  }
  c->loss_max_dy = 0;   // at most kLossMaxDy (validated with the description)
  for (const LossRes& R : c->hres) c->loss_max_dy = std::max(c->loss_max_dy, (8192 / R.nfft) * R.nbands * 4);
  if (upload(c, c->hres, &c->d_res) != MG_OK) return MG_ERR_CUDA;
  // songs on device
  c->hsd.assign(c->songs.size(), SongDev{});
  std::vector<int64_t> mixoff;
  int64_t moff = 0;
  for (size_t si = 0; si < c->songs.size(); ++si) {
    HostSong& hs = c->songs[si];
    SongDev& sd = c->hsd[si];
    sd.L = hs.L;
    sd.ld = hs.ld;
    for (int r = 0; r < 3; ++r) {
      sd.nframes[r] = hs.nframes[r];
      sd.first_frame[r] = hs.first[r];
      sd.litems[r] = r < c->nres ? hs.litems[r] : 0;
      sd.Y[r] = r < c->nres ? (float*)(c->arena + hs.o_Y[r]) : nullptr;
      sd.Yh[r] = r < c->nres ? (float*)(c->arena + hs.o_Yh[r]) : nullptr;
      sd.dF[r] = r < c->nres ? (float*)(c->arena + hs.o_dF[r]) : nullptr;
    }
    sd.lcap = std::max(1, hs.lcap);
    sd.mix = (const float*)(c->arena + hs.o_mix);
    sd.dmix = (float*)(c->arena + hs.o_dmix);
    sd.target = (const float*)(c->arena + hs.o_tgt);
    sd.lpart = (float*)(c->arena + hs.o_lpart);
    sd.coef = (float*)(c->arena + hs.o_coef);
    sd.ynorm2 = (double*)(c->arena + hs.o_ynorm);
    sd.pbeg = hs.pbeg;
    sd.pend = hs.pend;
    mixoff.push_back(moff);
    moff += 2 * (int64_t)hs.L;
  }
  if (upload(c, c->hsd, &c->d_songs) || upload(c, mixoff, &c->d_mixoff)) return MG_ERR_CUDA;
  if (build_loss_items(c) != MG_OK) return MG_ERR_CUDA;
  c->gather_items = ItemList{};
  for (size_t si = 0; si < c->songs.size(); ++si) {
    c->gather_items.beg.push_back((int)c->gather_items.h.size());
    for (int t = 0; t < (c->songs[si].L + kElemTile - 1) / kElemTile; ++t) c->gather_items.h.push_back(Item{(int)si, t});
  }
  c->gather_items.beg.push_back((int)c->gather_items.h.size());
  if (upload_items(c, c->gather_items) != MG_OK) return MG_ERR_CUDA;
  // evaluation items: disjoint full 8 s segments (a shorter song is one segment); Zwicker band bin ranges of
  // the 8192-point Bark frames
  {
    static const double edges[25] = {0, 100, 200, 300, 400, 510, 630, 770, 920, 1080, 1270, 1480, 1720, 2000, 2320,
                                     2700, 3150, 3700, 4400, 5300, 6400, 7700, 9500, 12000, 15500};
    c->ev_seg_len = (int)std::llround(8.0 * fs);
    c->ev_items.clear();
    c->ev_begin.clear();
    for (size_t si = 0; si < c->songs.size(); ++si) {
      c->ev_begin.push_back((int)c->ev_items.size());
      const int L = c->songs[si].L;
      const int nseg = L < c->ev_seg_len ? 1 : L / c->ev_seg_len;
      for (int k = 0; k < nseg; ++k) c->ev_items.push_back(make_int2((int)si, k));
    }
    c->ev_begin.push_back((int)c->ev_items.size());
    c->ev_lo.assign(24, 0);
    c->ev_hi.assign(24, 0);
    for (int b = 0; b < 24; ++b) {
      // bins k = 0 .. 4096 with edges[b] <= k fs / 8192 < edges[b + 1]
      int lo = 4097, hi = 0;
      for (int k = 0; k <= 4096; ++k) {
        const double f = k * fs / 8192.0;
        if (f >= edges[b] && f < edges[b + 1]) {
          lo = std::min(lo, k);
          hi = std::max(hi, k + 1);
        }
      }
      c->ev_lo[b] = lo > 4096 ? 0 : lo;
      c->ev_hi[b] = hi;
    }
    if (upload(c, c->ev_items, &c->d_ev_items) || upload(c, c->ev_begin, &c->d_ev_begin) ||
        upload(c, c->ev_lo, &c->d_ev_lo) || upload(c, c->ev_hi, &c->d_ev_hi))
      return MG_ERR_CUDA;
    CK(cudaMalloc(&c->d_ev_out, std::max<size_t>(1, c->ev_items.size()) * 66 * sizeof(double)));
    c->small_allocs.push_back(c->d_ev_out);
  }
  // ---- audio ----
  {
    float* tmp = nullptr;
    size_t tmpn = 0;
    for (size_t si = 0; si < c->songs.size(); ++si) {
      const HostSong& hs = c->songs[si];
      const size_t need = (size_t)hs.K * hs.L;
      if (need > tmpn) {
        if (tmp) cudaFree(tmp);
        CK(cudaMalloc(&tmp, need * sizeof(float)));
        tmpn = need;
      }
      if (!s[si].sources) return fail(c, MG_ERR_INVALID, "sources is null");
      CK(cudaMemcpyAsync(tmp, s[si].sources, need * sizeof(float),
                         s[si].on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
      for (int k = 0; k < hs.K; ++k)
        launch_ingest(c->stream, tmp + (size_t)k * hs.L,
                      (float*)(c->arena + (c->is_graph ? c->o_src[k] : c->chains[hs.tracks_chain[k]].o_in)), hs.L, hs.ld);
      if (s[si].target) {
        CK(cudaMemcpy2DAsync(c->arena + hs.o_tgt, (size_t)hs.ld * sizeof(float), s[si].target, (size_t)hs.L * sizeof(float),
                             (size_t)hs.L * sizeof(float), 2,
                             s[si].on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
      }
      CK(cudaStreamSynchronize(c->stream));
    }
    if (tmp) cudaFree(tmp);
  }
  {
    std::vector<float*> ins;
    for (size_t si = 0; si < c->songs.size(); ++si) {
      const HostSong& hs = c->songs[si];
      c->track_in_base.push_back((int)ins.size());
      for (int k = 0; k < hs.K; ++k)
        ins.push_back((float*)(c->arena + (c->is_graph ? c->o_src[k] : c->chains[hs.tracks_chain[k]].o_in)));
    }
    if (upload(c, ins, &c->d_track_in) != MG_OK) return MG_ERR_CUDA;
  }
  // ---- tables of the node structure ----
  if (build_tables(c) != MG_OK) return MG_ERR_CUDA;
  // ---- reverb noise spectra ----
  if (c->nrev > 0) {
    if (!d->reverb_noise) return fail(c, MG_ERR_INVALID, "reverb_noise is required when reverbs are enabled");
    const int rl = (int)std::llround(2.0 * fs);
    float* nz = nullptr;
    const size_t bytes = (size_t)c->nrev * 2 * rl * sizeof(float);
    CK(cudaMalloc(&nz, bytes));
    CK(cudaMemcpyAsync(nz, d->reverb_noise, bytes, d->noise_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       c->stream));
    ItemList it;
    for (int pi = 0; pi < c->P; ++pi)
      if (c->procs[pi].type == T_R)
        for (int i = 0; i < (c->procs[pi].nframes + kRevFG - 1) / kRevFG; ++i) it.h.push_back(Item{pi, i});
    if (upload_items(c, it) != MG_OK) return MG_ERR_CUDA;
    LaunchCtx x = make_ctx(c, nullptr);
    launch_rev_noise_stft(x, it.d, (int)it.h.size(), nz, rl);
    CK(cudaStreamSynchronize(c->stream));
    cudaFree(nz);
  }
  // ---- FFT split autotuner ----
  if (d->autotune && autotune_splits(c) != MG_OK) return MG_ERR_CUDA;
  if (d->autotune && autotune_packing(c) != MG_OK) return MG_ERR_CUDA;
  // ---- target spectrograms ----
  {
    LaunchCtx x = make_ctx(c, nullptr);
    const bool prof = c->profiling;
    c->profiling = false;
    loss_forward(c, x, 0, nullptr, nullptr, 0);
    c->profiling = prof;
  }
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaGetLastError());
  return MG_OK;
}

void destroy_impl(mg_console* c) {
  if (c->graph) cudaGraphExecDestroy(c->graph);
  for (void* p : c->small_allocs) cudaFree(p);
  for (void* p : c->table_allocs) cudaFree(p);
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  cudaFree(c->arena);
  cudaFree(c->scratch);
  cudaFree(c->d_params);
  cudaFree(c->d_grads);
  cudaFree(c->d_m);
  cudaFree(c->d_v);
  cudaFree(c->d_step);
  cudaFree(c->d_hyper);
  cudaFree(c->d_alphas);
  cudaFree(c->d_mask);
  cudaFree(c->d_scratch_la);
  cudaFree(c->score_ws);
  cudaFree(c->d_chain);
  if (c->h_err) cudaFreeHost(c->h_err);
}

void fill_info(const mg_console* c, mg_console_info* o) {
  o->n_songs = (int32_t)c->songs.size();
  o->n_processors = c->P;
  o->n_proc_params = c->npp;
  o->n_params = c->nparams;
  o->n_reverbs = c->nrev;
  o->total_samples = c->total_samples;
  o->track_seconds = c->track_seconds;
  o->device_bytes = (int64_t)(c->arena_bytes + c->scratch_bytes + 4 * sizeof(float) * c->nparams);
  o->launches_per_step = c->launches_step;
  o->retains_spectra = c->retain ? 1 : 0;
}

// ------------------------------------------------------------------------------------------------
// batched candidate scoring (Alg. 2-3 Evaluate, Sec. 7.2 Delta_i)
// ------------------------------------------------------------------------------------------------
// The candidate masks of one call differ from a base mask (the per-processor majority of the candidates) in a
// few processors.  The base is rendered once.  Under candidate j a node's output equals the base output unless
// the node, or a node upstream of it, has a different mask value; only those nodes are computed again, as
// forward-only copies ("virtual nodes") with their own output and FFT scratch that read the base outputs where
// their input did not change:
//   - a track chain from its first differing processor to its end,
//   - a subgroup chain from its first differing processor, or all of it when one of its tracks changed (its
//     mix node m is then summed again),
//   - the output node o and the loss of every song that changed.
// The copies of every candidate run in one launch per processor type and level, in console order, with the
// same kernels, parameters, splits and work items as a full render, so every score is bitwise the score of a
// full render under that candidate's mask.

// Which parts of the console one candidate changes.
struct CandPlan {
  std::vector<std::pair<int, int>> chains;   // (chain, position of its first changed processor)
  std::vector<int> songs;                    // songs whose mix changes
  size_t bytes = 0;                          // workspace bytes of its copies, sums, songs and tables
};

// One chunk of candidates, built on the host: node copies and their work lists, sums, song copies, loss items.
struct ScoreChunk {
  std::vector<ProcDev> vp;
  std::vector<int> vsrc;                     // processor copied by every node copy
  std::vector<uint8_t> vmask;                // mask value of every node copy
  std::vector<Stage> stages;                 // level 0 then level 1, types in chain order
  std::vector<float*> sum_out;
  std::vector<const float*> sum_in;
  std::vector<int> sum_beg, sum_L, sum_ld;
  ItemList m_items, o_items;
  std::vector<SongDev> vs;
  std::vector<int4> litems[3];
  std::vector<int> map;                      // [candidate][song]: song copy, or -1 (unchanged)
  std::vector<std::vector<std::pair<char*, const char*>>> promo;   // [candidate][song]: (arena, copy) buffers
  size_t table_begin = 0;                    // workspace offset of the tables (copied from the host blob)
  size_t end = 0;                            // workspace bytes the chunk uses
  unsigned long long* flags = nullptr;       // published states of the chained scans of the node copies
  std::vector<CUtensorMap> umaps;            // tensor maps of the compressor / gate copies' inputs
  std::vector<std::pair<int, int>> umap_of;  // (node copy, map)
  size_t flags_bytes = 0;
  float* vq = nullptr;
  float* vla = nullptr;
  int* d_vsrc = nullptr;
  int* d_map = nullptr;
  ProcDev* d_vp = nullptr;
  uint8_t* d_vmask = nullptr;
  SongDev* d_vs = nullptr;
  int4* d_litems[3] = {nullptr, nullptr, nullptr};
  float** d_sum_out = nullptr;
  const float** d_sum_in = nullptr;
  int *d_sum_beg = nullptr, *d_sum_L = nullptr, *d_sum_ld = nullptr;
};

// Bytes of the workspace a node copy of processor pi needs (forward-only buffers) and its work items.
size_t copy_bytes(const mg_console* c, int pi, size_t* items) {
  const HostProc& p = c->procs[pi];
  auto al = [](size_t b) { return (size_t)round_up((int64_t)b, 256); };
  size_t b = al((size_t)2 * p.ld * sizeof(float)) + al(kStatsFloats * sizeof(float));
  size_t it = 0;
  if (p.nfrows) b += al((size_t)std::max(p.nfrows, p.nfcap) * kNPart * sizeof(float));
  if (p.type == T_C || p.type == T_N) {
    b += 2 * al((size_t)p.nchunks * sizeof(float)) + (size_t)p.nchunks * sizeof(unsigned long long) +
         sizeof(CUtensorMap);   // + states, + tensor map
    it = p.nchunks + 1;
  } else if (p.type == T_G || p.type == T_S) {
    it = p.nbrows;
  } else if (p.type == T_E) {
    b += al((size_t)2 * p.ld * sizeof(float));   // the wet signal the equalizer forward stores
    it = p.nfrows;
  } else {
    const size_t N = (size_t)p.f << p.logN;
    b += al(N * sizeof(float2)) * (c->retain ? 1 : 2);   // T1, and Hz when the base does not keep it
    it = ((size_t)p.f << p.logN1) / p.colG + ((size_t)1 << p.logN2) / 2 + 1 + 1;
  }
  *items = it;
  return b;
}

// The changed chains and songs of candidate mask mj against the base mask m0, and its workspace bytes.
CandPlan plan_candidate(const mg_console* c, const uint8_t* mj, const uint8_t* m0) {
  CandPlan cp;
  auto al = [](size_t b) { return (size_t)round_up((int64_t)b, 256); };
  auto first_changed = [&](int ci) {
    const HostChain& ch = c->chains[ci];
    for (size_t k = 0; k < ch.procs.size(); ++k) {
      const int pi = ch.procs[k];
      if (c->procs[pi].present && mj[pi] != m0[pi]) return (int)k;
    }
    return -1;
  };
  size_t nodes = 0, items = 0;
  auto add_chain = [&](int ci, int from) {
    cp.chains.push_back({ci, from});
    const HostChain& ch = c->chains[ci];
    for (size_t k = from; k < ch.procs.size(); ++k) {
      if (!c->procs[ch.procs[k]].present) continue;
      size_t it = 0;
      cp.bytes += copy_bytes(c, ch.procs[k], &it);
      items += it;
      ++nodes;
    }
  };
  for (size_t si = 0; si < c->songs.size(); ++si) {
    const HostSong& hs = c->songs[si];
    bool song_changed = false;
    std::vector<char> group_in(hs.S, 0);
    for (int k = 0; k < hs.K; ++k) {
      const int f = first_changed(hs.tracks_chain[k]);
      if (f < 0) continue;
      add_chain(hs.tracks_chain[k], f);
      song_changed = true;
      if (hs.group[k] >= 0) group_in[hs.group[k]] = 1;
    }
    const size_t st = al((size_t)2 * hs.ld * sizeof(float));
    const size_t tiles = (hs.L + kElemTileMin - 1) / kElemTileMin;
    for (int g = 0; g < hs.S; ++g) {
      const int f = group_in[g] ? 0 : first_changed(hs.groups_chain[g]);
      if (f < 0) continue;
      add_chain(hs.groups_chain[g], f);
      song_changed = true;
      if (group_in[g]) cp.bytes += st + al(sizeof(void*) * (hs.K + 1)) + al(tiles * sizeof(Item)) + al(64);
    }
    if (song_changed) {
      cp.songs.push_back((int)si);
      cp.bytes += st + al((size_t)3 * std::max(1, hs.lcap) * 6 * sizeof(float)) + al(18 * sizeof(float)) +
                  al(sizeof(SongDev)) + al(sizeof(void*) * (hs.K + hs.S + 1)) + al(tiles * sizeof(Item)) + al(64);
      for (int r = 0; r < c->nres; ++r) cp.bytes += al((size_t)hs.litems[r] * sizeof(int4));
    }
  }
  // tables of the node copies: the node table, sources, masks, logits, work items and lists, per-candidate map
  cp.bytes += al(nodes * sizeof(ProcDev)) + 4 * al(nodes * sizeof(int)) + al(nodes) + al(items * sizeof(Item)) +
              al(c->songs.size() * sizeof(int)) + al(sizeof(float) * (cp.songs.size() + 1));
  return cp;
}

// Bump allocation in the workspace: buffers first, then the tables, whose contents go to a host blob that is
// copied to the device once per chunk.
struct WsBuilder {
  char* base;
  Bump b;
  size_t table_begin = 0;
  std::vector<char>* blob;
  char* buffer(size_t bytes) { return base + b.take(bytes); }
  void start_tables() {
    b.off = (size_t)round_up((int64_t)b.off, 256);
    table_begin = b.off;
    blob->clear();
  }
  template <class T>
  T* table(const std::vector<T>& v) {
    if (v.empty()) return nullptr;
    const size_t o = b.take(v.size() * sizeof(T));
    if (blob->size() < o - table_begin + v.size() * sizeof(T)) blob->resize(o - table_begin + v.size() * sizeof(T));
    std::memcpy(blob->data() + (o - table_begin), v.data(), v.size() * sizeof(T));
    return reinterpret_cast<T*>(base + o);
  }
};

mg_status ensure_score_ws(mg_console* c, size_t bytes) {
  if (bytes <= c->score_ws_bytes) return MG_OK;
  CK(cudaStreamSynchronize(c->stream));
  std::lock_guard<std::mutex> lock(g_device_mutex);
  if (c->score_ws) cudaFree(c->score_ws);
  c->score_ws = nullptr;
  c->score_ws_bytes = 0;
  const size_t want = (size_t)round_up((int64_t)bytes + ((int64_t)bytes >> 3), 1 << 20);   // 1/8 headroom
  if (cudaMalloc(&c->score_ws, want) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, MG_ERR_OOM, "candidate scoring workspace allocation failed");
  }
  c->score_ws_bytes = want;
  CK(cudaMemsetAsync(c->score_ws, 0, want, c->stream));
  return MG_OK;
}

// Builds the node copies, sums, song copies and loss items of candidates [j0, j1) in the workspace.
void build_chunk(mg_console* c, const std::vector<CandPlan>& plans, const uint8_t* hm, int j0, int j1, ScoreChunk& k) {
  WsBuilder w{c->score_ws, Bump{}, 0, &c->score_blob};
  auto A = [&](size_t off) { return c->arena + off; };
  const int ns = (int)c->songs.size();
  k.map.assign((size_t)(j1 - j0) * ns, -1);
  k.promo.assign((size_t)(j1 - j0) * ns, {});
  // node copies per (level, type), in candidate order
  std::vector<int> by_lt[2][NTYPES];
  std::vector<std::pair<int, int>> flag_nodes;   // (node copy, chunks) of the chained scans
  for (int j = j0; j < j1; ++j) {
    const uint8_t* mj = hm + (size_t)j * c->P;
    const CandPlan& cp = plans[j];
    std::vector<const float*> chain_y(c->chains.size(), nullptr);   // output of the chain's copy, if any
    std::vector<const float*> group_in(c->chains.size(), nullptr);   // recomputed input of a subgroup chain
    auto copy_chain = [&](int ci, int from) {
      const HostChain& ch = c->chains[ci];
      const float* cur = group_in[ci] ? group_in[ci] : (const float*)A(ch.o_in);
      for (int kk = 0; kk < from; ++kk)
        if (c->procs[ch.procs[kk]].present) cur = c->hpd[ch.procs[kk]].y;
      for (size_t kk = from; kk < ch.procs.size(); ++kk) {
        const int pi = ch.procs[kk];
        const HostProc& p = c->procs[pi];
        if (!p.present) continue;
        ProcDev d = c->hpd[pi];
        const int v = (int)k.vp.size();
        d.qidx = v;
        d.u = cur;
        d.y = (float*)w.buffer((size_t)2 * p.ld * sizeof(float));
        d.stats = (float*)w.buffer(kStatsFloats * sizeof(float));
        d.fpart = p.nfrows ? (float*)w.buffer((size_t)std::max(p.nfrows, p.nfcap) * kNPart * sizeof(float)) : nullptr;
        d.dy = nullptr;
        d.du = nullptr;
        d.gp = nullptr;
        d.bpart = nullptr;
        d.dtaps = nullptr;
        d.dhspec = nullptr;
        d.eqg = nullptr;
        d.ybar = p.type == T_E ? (float*)w.buffer((size_t)2 * p.ld * sizeof(float)) : nullptr;
        if (p.type == T_C || p.type == T_N) {
          d.carry = (float*)w.buffer((size_t)p.nchunks * sizeof(float));
          d.chunkagg = (float*)w.buffer((size_t)p.nchunks * sizeof(float));
          d.aux = nullptr;
          flag_nodes.push_back({(int)k.vp.size(), p.nchunks});
          d.umap = nullptr;
          d.dymap = nullptr;
          CUtensorMap m;
          if (c->dyn_tma && encode_dyn_map(&m, d.u, p.ld)) {
            k.umap_of.push_back({(int)k.vp.size(), (int)k.umaps.size()});
            k.umaps.push_back(m);
          }
        }
        if (p.type == T_R || p.type == T_D) {
          const size_t N = (size_t)p.f << p.logN;
          d.T1 = (float2*)w.buffer(N * sizeof(float2));
          d.T2 = nullptr;
          if (!c->retain) d.Hz = (float2*)w.buffer(N * sizeof(float2));   // else the base node's kept spectrum
        }
        k.vp.push_back(d);
        k.vsrc.push_back(pi);
        k.vmask.push_back(mj[pi]);
        by_lt[p.level][p.type].push_back(v);
        k.promo[(size_t)(j - j0) * ns + p.song].push_back({A(p.o_y), (const char*)d.y});
        cur = d.y;
      }
      chain_y[ci] = cur;
    };
    auto out_of = [&](int ci) { return chain_y[ci] ? chain_y[ci] : (const float*)A(c->chain_out[ci]); };
    // track chains, then subgroup inputs and chains, then the mix, song by song
    size_t ci_next = 0;
    for (int si : cp.songs) {
      const HostSong& hs = c->songs[si];
      for (; ci_next < cp.chains.size() && c->chains[cp.chains[ci_next].first].song == si &&
             c->chains[cp.chains[ci_next].first].level == 0; ++ci_next)
        copy_chain(cp.chains[ci_next].first, cp.chains[ci_next].second);
      for (int g = 0; g < hs.S; ++g) {
        bool changed = false;
        for (int kk = 0; kk < hs.K; ++kk)
          if (hs.group[kk] == g && chain_y[hs.tracks_chain[kk]]) changed = true;
        if (!changed) continue;
        float* out = (float*)w.buffer((size_t)2 * hs.ld * sizeof(float));
        const int sid = (int)k.sum_out.size();
        k.sum_beg.push_back((int)k.sum_in.size());
        k.sum_out.push_back(out);
        for (int kk = 0; kk < hs.K; ++kk)
          if (hs.group[kk] == g) k.sum_in.push_back(out_of(hs.tracks_chain[kk]));
        k.sum_L.push_back(hs.L);
        k.sum_ld.push_back(hs.ld);
        k.m_items.beg.push_back((int)k.m_items.h.size());
        for (int t = 0; t < (hs.L + c->elem_tile - 1) / c->elem_tile; ++t) k.m_items.h.push_back(Item{sid, t});
        group_in[hs.groups_chain[g]] = out;
        k.promo[(size_t)(j - j0) * ns + si].push_back({A(c->chains[hs.groups_chain[g]].o_in), (const char*)out});
      }
      for (; ci_next < cp.chains.size() && c->chains[cp.chains[ci_next].first].song == si; ++ci_next)
        copy_chain(cp.chains[ci_next].first, cp.chains[ci_next].second);
      // the mix and the song copy
      float* mix = (float*)w.buffer((size_t)2 * hs.ld * sizeof(float));
      const int sid = (int)k.sum_out.size();
      k.sum_beg.push_back((int)k.sum_in.size());
      k.sum_out.push_back(mix);
      for (int g = 0; g < hs.S; ++g) k.sum_in.push_back(out_of(hs.groups_chain[g]));
      for (int kk = 0; kk < hs.K; ++kk)
        if (hs.group[kk] < 0) k.sum_in.push_back(out_of(hs.tracks_chain[kk]));
      k.sum_L.push_back(hs.L);
      k.sum_ld.push_back(hs.ld);
      k.o_items.beg.push_back((int)k.o_items.h.size());
      for (int t = 0; t < (hs.L + c->elem_tile - 1) / c->elem_tile; ++t) k.o_items.h.push_back(Item{sid, t});
      SongDev sd = c->hsd[si];
      const int vsi = (int)k.vs.size();
      sd.mix = mix;
      sd.dmix = nullptr;
      for (int r = 0; r < 3; ++r) sd.Yh[r] = nullptr;
      sd.lpart = (float*)w.buffer((size_t)3 * sd.lcap * 6 * sizeof(float));
      sd.coef = (float*)w.buffer(18 * sizeof(float));
      k.vs.push_back(sd);
      for (int r = 0; r < c->nres; ++r) {
        const int per = c->loss_per[r];
        for (int t = hs.first[r]; t < hs.nframes[r]; t += per)
          k.litems[r].push_back(make_int4(vsi, r, t, std::min(per, hs.nframes[r] - t)));
      }
      k.map[(size_t)(j - j0) * ns + si] = vsi;
      k.promo[(size_t)(j - j0) * ns + si].push_back({A(hs.o_mix), (const char*)mix});
    }
  }
  k.sum_beg.push_back((int)k.sum_in.size());
  k.m_items.beg.push_back((int)k.m_items.h.size());
  k.o_items.beg.push_back((int)k.o_items.h.size());
  const int V = (int)k.vp.size();
  // one contiguous region of publication flags, cleared before the chunk runs
  size_t nflags = 0;
  for (const auto& fn : flag_nodes) nflags += fn.second;
  k.flags = (unsigned long long*)w.buffer(sizeof(unsigned long long) * std::max<size_t>(1, nflags));
  k.flags_bytes = sizeof(unsigned long long) * std::max<size_t>(1, nflags);
  for (size_t f = 0, off = 0; f < flag_nodes.size(); off += flag_nodes[f].second, ++f)
    k.vp[flag_nodes[f].first].cflag = k.flags + off;
  k.vq = (float*)w.buffer(sizeof(float) * std::max(1, V));
  k.vla = (float*)w.buffer(sizeof(float) * std::max<size_t>(1, k.vs.size()));
  // work lists per (level, type)
  k.stages.clear();
  for (int level = 0; level < 2; ++level)
    for (int t = 0; t < NTYPES; ++t) {
      if (by_lt[level][t].empty()) continue;
      Stage st;
      st.level = level;
      st.type = t;
      st.procs.h = by_lt[level][t];
      if (t == T_R || t == T_D) st.groups.push_back(LtiGroup{});
      for (int v : by_lt[level][t]) {
        const ProcDev& d = k.vp[v];
        if ((t == T_C || t == T_N) && !c->per_node) {
          continue;   // in rounds below
        } else if (t == T_G || t == T_S || t == T_C || t == T_N) {
          st.elem.beg.push_back((int)st.elem.h.size());
          const int nt = (t == T_C || t == T_N) ? d.nchunks : (d.L + c->elem_tile - 1) / c->elem_tile;
          for (int i = 0; i < nt; ++i) st.elem.h.push_back(Item{v, i});
        } else if (t == T_E) {
          st.osf.beg.push_back((int)st.osf.h.size());
          for (int i = 0; i < d.nfpart; ++i) st.osf.h.push_back(Item{v, i});
        } else {
          LtiGroup& g = st.groups[0];
          g.procs.h.push_back(v);
          g.col.beg.push_back((int)g.col.h.size());
          g.rowpair.beg.push_back((int)g.rowpair.h.size());
          const int N1 = d.f << d.logN1, N2 = 1 << d.logN2;
          for (int i = 0; i < N1 / d.colG; ++i) g.col.h.push_back(Item{v, i});
          for (int i = 0; i <= N2 / 2; ++i) g.rowpair.h.push_back(Item{v, i});
          g.col.maxv = std::max(g.col.maxv, N2 * d.colG);
          g.rowpair.maxv = std::max(g.rowpair.maxv, N1);
        }
      }
      st.elem.beg.push_back((int)st.elem.h.size());
      if ((t == T_C || t == T_N) && !c->per_node)
        chain_rounds(st.procs.h, [&](int v) { return k.vp[v].nchunks; }, st.elem, nullptr);
      st.osf.beg.push_back((int)st.osf.h.size());
      for (auto& g : st.groups) {
        g.col.beg.push_back((int)g.col.h.size());
        g.rowpair.beg.push_back((int)g.rowpair.h.size());
      }
      k.stages.push_back(std::move(st));
    }
  // tables
  w.start_tables();
  k.table_begin = w.table_begin;
  {
    CUtensorMap* dm = w.table(k.umaps);
    for (const auto& um : k.umap_of) k.vp[um.first].umap = dm + um.second;
  }
  k.d_vp = w.table(k.vp);
  k.d_vsrc = w.table(k.vsrc);
  k.d_vmask = w.table(k.vmask);
  k.d_map = w.table(k.map);
  k.d_vs = w.table(k.vs);
  for (int r = 0; r < 3; ++r) k.d_litems[r] = w.table(k.litems[r]);
  k.d_sum_out = w.table(k.sum_out);
  k.d_sum_in = w.table(k.sum_in);
  k.d_sum_beg = w.table(k.sum_beg);
  k.d_sum_L = w.table(k.sum_L);
  k.d_sum_ld = w.table(k.sum_ld);
  k.m_items.d = w.table(k.m_items.h);
  k.o_items.d = w.table(k.o_items.h);
  for (auto& st : k.stages) {
    st.procs.d = w.table(st.procs.h);
    st.elem.d = w.table(st.elem.h);
    st.osf.d = w.table(st.osf.h);
    for (auto& g : st.groups) {
      g.procs.d = w.table(g.procs.h);
      g.col.d = w.table(g.col.h);
      g.rowpair.d = w.table(g.rowpair.h);
    }
  }
  k.end = w.b.off;
}

// Host check of a chunk before anything is copied or launched: every device pointer of the node copies, sums and
// song copies lies in the arena, the spectra scratch, the workspace or the parameter buffer, and every work item
// indexes an existing node copy within its range.  Returns an empty string when the chunk is consistent.
std::string check_chunk(const mg_console* c, const ScoreChunk& k) {
  auto in = [&](const void* p, size_t bytes) {
    const char* q = static_cast<const char*>(p);
    auto inside = [&](const char* b, size_t n) { return b && q >= b && q + bytes <= b + n; };
    return inside(c->arena, c->arena_bytes) || inside(c->scratch, c->scratch_bytes) ||
           inside(c->score_ws, c->score_ws_bytes) ||
           inside(reinterpret_cast<const char*>(c->d_params), sizeof(float) * (size_t)c->nparams);
  };
  if (k.end > c->score_ws_bytes) return "chunk exceeds the scoring workspace";
  for (size_t v = 0; v < k.vp.size(); ++v) {
    const ProcDev& d = k.vp[v];
    const size_t st = (size_t)2 * d.ld * sizeof(float);
    if (!in(d.u, st) || !in(d.y, st) || !in(d.stats, kStatsFloats * sizeof(float)) || !in(d.p, sizeof(float)))
      return "node copy " + std::to_string(v) + ": signal or parameter pointer out of range";
    if (d.fpart && !in(d.fpart, (size_t)d.nfpart * kNPart * sizeof(float)))
      return "node copy " + std::to_string(v) + ": partials out of range";
    if ((d.type == T_C || d.type == T_N) &&
        (!in(d.carry, (size_t)d.nchunks * 4) || !in(d.chunkagg, (size_t)d.nchunks * 4) ||
         !in(d.cflag, (size_t)d.nchunks * 8)))
      return "node copy " + std::to_string(v) + ": scan carries out of range";
    if (d.type == T_R || d.type == T_D) {
      const size_t N = (size_t)d.f << d.logN;
      if (!in(d.T1, N * sizeof(float2)) || !in(d.Hz, N * sizeof(float2)) ||
          !in(d.taps, (size_t)2 * d.Nh * sizeof(float)))
        return "node copy " + std::to_string(v) + ": FFT buffers out of range";
    }
    if (d.type == T_E && (!in(d.hspec, kEqOsM * sizeof(float)) || !in(d.ybar, st)))
      return "node copy " + std::to_string(v) + ": equalizer spectrum or wet signal out of range";
  }
  const int V = (int)k.vp.size();
  for (const auto& st : k.stages) {
    for (int v : st.procs.h)
      if (v < 0 || v >= V) return "stage list indexes a missing node copy";
    for (const Item& it : st.elem.h) {
      const ProcDev& d = k.vp[it.proc];
      const int lim = (st.type == T_C || st.type == T_N) ? d.nchunks : (d.L + c->elem_tile - 1) / c->elem_tile;
      if (it.proc < 0 || it.proc >= V || it.idx < 0 || it.idx >= lim) return "elementwise item out of range";
    }
    for (const Item& it : st.osf.h)
      if (it.proc < 0 || it.proc >= V || it.idx < 0 || it.idx >= k.vp[it.proc].nfpart) return "equalizer item out of range";
    for (const auto& g : st.groups) {
      for (const Item& it : g.col.h) {
        const ProcDev& d = k.vp[it.proc];
        if (it.idx < 0 || it.idx >= (d.f << d.logN1) / d.colG) return "column item out of range";
      }
      for (const Item& it : g.rowpair.h)
        if (it.idx < 0 || it.idx > (1 << k.vp[it.proc].logN2) / 2) return "row item out of range";
    }
  }
  for (size_t s = 0; s + 1 < k.sum_beg.size(); ++s) {
    const size_t st = (size_t)2 * k.sum_ld[s] * sizeof(float);
    if (!in(k.sum_out[s], st)) return "sum output out of range";
    for (int j = k.sum_beg[s]; j < k.sum_beg[s + 1]; ++j)
      if (!in(k.sum_in[j], st)) return "sum input out of range";
  }
  for (const SongDev& sd : k.vs)
    if (!in(sd.mix, (size_t)2 * sd.ld * sizeof(float)) || !in(sd.lpart, (size_t)18 * sd.lcap * sizeof(float)))
      return "song copy buffers out of range";
  for (int r = 0; r < 3; ++r)
    for (const int4& it : k.litems[r])
      if (it.x < 0 || it.x >= (int)k.vs.size()) return "loss item indexes a missing song copy";
  return std::string();
}

// Forward of the node copies of one (level, type): the stage's kernels without the parameter-only work (FIR
// synthesis, equalizer spectrum; with kept spectra also the filter transform), which the copies share with the
// nodes they copy.
void vstage_forward(mg_console* c, const LaunchCtx& x, Stage& s) {
  StageScope scope(c, s.type);
  switch (s.type) {
    case T_G:
    case T_S:
      run_items(c, F_GS_FWD, s.elem, [&](const Item* it, int n) { launch_gs_fwd(x, it, n); });
      break;
    case T_C:
    case T_N:
      run_items(c, F_DYN_FWD, s.elem, [&](const Item* it, int n) { launch_dyn_fwd(x, it, n); });
      break;
    case T_E:
      run_items(c, F_EQ_OS_FWD, s.osf, [&](const Item* it, int n) { launch_eq_os_fwd(x, it, n); });
      break;
    default:
      for (auto& g : s.groups) {
        run_procs(c, F_SCALE, g.procs, [&](const int* p, int n) { launch_chan_scale(x, p, n, 0); });
        if (!c->retain) {
          run_items(c, F_COL_FWD, g.col, [&](const Item* it, int n) { launch_col_fwd_taps(x, it, n, g.col.maxv); });
          run_items(c, F_ROW_HZ, g.rowpair, [&](const Item* it, int n) { launch_row_fwd_hz(x, it, n, g.rowpair.maxv); });
        }
        run_items(c, F_COL_FWD, g.col, [&](const Item* it, int n) { launch_col_fwd_audio(x, it, n, g.col.maxv); });
        run_items(c, F_ROW_CONV, g.rowpair, [&](const Item* it, int n) { launch_row_conv_fwd(x, it, n, g.rowpair.maxv, false); });
        run_items(c, F_COL_OUT, g.col, [&](const Item* it, int n) { launch_col_inv_out(x, it, n, g.col.maxv); });
      }
  }
}

// The score budget: the workspace limit of the descriptor when set, else 60 % of the device memory free at the
// first scoring call (at most 64 GiB).
size_t score_budget(mg_console* c) {
  if (c->score_budget) return c->score_budget;
  if (c->desc.workspace_limit_bytes > 0) {
    c->score_budget = (size_t)c->desc.workspace_limit_bytes;
  } else {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = (size_t)1 << 30;
    const size_t b = std::min((size_t)(0.6 * (double)(free_b + c->score_ws_bytes)), (size_t)64 << 30);
    c->score_budget = std::max(b, (size_t)64 << 20);
  }
  return c->score_budget;
}

// Full masked render of one candidate (no copies): the path of a candidate whose copies alone exceed the budget.
void score_full(mg_console* c, const uint8_t* d_mask_j, float* d_la_row) {
  cudaMemcpyAsync(c->d_mask, d_mask_j, c->P, cudaMemcpyDeviceToDevice, c->stream);
  LaunchCtx x = make_ctx(c, c->d_mask);
  render(c, x);
  loss_forward(c, x, 2, nullptr, d_la_row, 1);
}

// Makes the arena hold the base render of mask m0 from the last call's surviving chunk, without rendering: per
// song, nothing to do when m0 equals the old base there; the recomputed outputs and the L_a of a candidate whose
// mask equals m0 there are copied in (device to device, on the stream).  False (nothing copied) when some song
// matches neither.
bool promote_base(mg_console* c, const std::vector<uint8_t>& m0) {
  auto& kp = c->score_keep;
  const int ns = (int)c->songs.size();
  std::vector<int> pick(ns, -1);
  for (int si = 0; si < ns; ++si) {
    const int b = c->songs[si].pbeg, e = c->songs[si].pend;
    auto same = [&](const uint8_t* m) { return std::equal(m0.begin() + b, m0.begin() + e, m + b); };
    if (same(kp.m0.data())) continue;
    for (int j = 0; j < kp.nc && pick[si] < 0; ++j)
      if (kp.vsong[(size_t)j * ns + si] >= 0 && same(kp.masks.data() + (size_t)j * c->P)) pick[si] = j;
    if (pick[si] < 0) return false;
  }
  for (int si = 0; si < ns; ++si) {
    if (pick[si] < 0) continue;
    const size_t bytes = (size_t)2 * c->songs[si].ld * sizeof(float);
    for (const auto& cp : kp.promo[(size_t)pick[si] * ns + si])
      if (cudaMemcpyAsync(cp.first, cp.second, bytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess) return false;
    const int vs = kp.vsong[(size_t)pick[si] * ns + si];
    if (cudaMemcpyAsync(c->d_scratch_la + si, kp.vla + vs, sizeof(float), cudaMemcpyDeviceToDevice, c->stream) !=
        cudaSuccess)
      return false;
  }
  return true;
}

mg_status prune_scores_batched(mg_console* c, const uint8_t* d_masks, int n_masks, float* d_la) {
  const int P = c->P, ns = (int)c->songs.size();
  std::vector<uint8_t> hm((size_t)n_masks * P);
  CK(cudaMemcpyAsync(hm.data(), d_masks, hm.size(), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (uint8_t& v : hm) v = v ? 1 : 0;
  // base mask: per processor the value most candidates have (ties: 1)
  c->score_m0.assign(P, 1);
  bool all_ones = true;
  for (int i = 0; i < P; ++i) {
    int ones = 0;
    for (int j = 0; j < n_masks; ++j) ones += hm[(size_t)j * P + i];
    c->score_m0[i] = 2 * ones >= n_masks ? 1 : 0;
    all_ones = all_ones && c->score_m0[i];
  }
  std::vector<CandPlan> plans(n_masks);
  for (int j = 0; j < n_masks; ++j) plans[j] = plan_candidate(c, hm.data() + (size_t)j * P, c->score_m0.data());
  // the base: kept from the last call where, song by song, the new base mask equals the old base or one of its
  // candidates (whose recomputed outputs are copied into the arena), else rendered
  bool base_ready = false;
  if (c->score_keep.valid) base_ready = promote_base(c, c->score_m0);
  c->score_keep.valid = false;
  if (!base_ready) {
    if (!all_ones) CK(cudaMemcpyAsync(c->d_mask, c->score_m0.data(), P, cudaMemcpyHostToDevice, c->stream));
    LaunchCtx xb = make_ctx(c, all_ones ? nullptr : c->d_mask);
    if (!(c->fwd_valid && all_ones)) render(c, xb);
    loss_forward(c, xb, 2, nullptr, c->d_scratch_la, 1);
  }
  // candidates in chunks whose copies fit the budget; a candidate that alone exceeds it is rendered in full
  const size_t budget = score_budget(c);
  std::vector<int> full;
  int j = 0;
  while (j < n_masks) {
    if (plans[j].bytes + (64 << 10) > budget) {
      full.push_back(j++);
      continue;
    }
    int j1 = j;
    size_t bytes = 64 << 10;
    while (j1 < n_masks && plans[j1].bytes + (64 << 10) <= budget && bytes + plans[j1].bytes <= budget)
      bytes += plans[j1++].bytes;
    if (ensure_score_ws(c, bytes) != MG_OK) return MG_ERR_OOM;
    ScoreChunk k;
    build_chunk(c, plans, hm.data(), j, j1, k);
    if (k.end > c->score_ws_bytes || c->debug_sync) {
      const std::string bad = check_chunk(c, k);
      if (!bad.empty()) return fail(c, MG_ERR_INVALID, "candidate scoring: " + bad);
    }
    if (!c->score_blob.empty())
      CK(cudaMemcpyAsync(c->score_ws + k.table_begin, c->score_blob.data(), c->score_blob.size(),
                         cudaMemcpyHostToDevice, c->stream));
    const int V = (int)k.vp.size();
    CK(cudaMemsetAsync(k.flags, 0, k.flags_bytes, c->stream));
    LaunchCtx xv = make_ctx(c, k.d_vmask);
    xv.procs = k.d_vp;
    xv.q = k.vq;
    if (V > 0) {
      run(c, F_MISC, [&] { launch_gather_q(c->stream, c->d_params + c->npp, k.d_vsrc, k.vq, V); });
      for (int level = 0; level < 2; ++level) {
        if (level == 1 && !k.m_items.h.empty()) {
          StageScope scope(c, 8);
          run_items(c, F_SUM, k.m_items, [&](const Item* it, int n) {
            launch_sum(c->stream, k.d_sum_out, k.d_sum_in, k.d_sum_beg, k.d_sum_L, k.d_sum_ld, it, n, c->elem_tile);
          });
        }
        for (auto& st : k.stages)
          if (st.level == level) vstage_forward(c, xv, st);
      }
    }
    if (!k.vs.empty()) {
      {
        StageScope scope(c, 8);
        run_items(c, F_SUM, k.o_items, [&](const Item* it, int n) {
          launch_sum(c->stream, k.d_sum_out, k.d_sum_in, k.d_sum_beg, k.d_sum_L, k.d_sum_ld, it, n, c->elem_tile);
        });
      }
      StageScope scope(c, 7);
      for (int r = 0; r < c->nres; ++r)
        if (!k.litems[r].empty())
          run(c, F_LOSS_FWD, [&] {
            launch_loss_frames(xv, k.d_vs, c->d_res, k.d_litems[r], (int)k.litems[r].size(), 1, c->loss_max_dy);
          });
      run(c, F_FINALIZE, [&] {
        launch_loss_finalize_mode(xv, k.d_vs, (int)k.vs.size(), c->d_res, c->nres, c->d_alphas, 2, nullptr, k.vla, 1);
      });
    }
    run(c, F_MISC, [&] {
      launch_score_scatter(c->stream, k.d_map, k.vla, c->d_scratch_la, d_la + (size_t)j * ns, (j1 - j) * ns, ns);
    });
    CK(cudaGetLastError());
    // the next chunk's tables overwrite these: the host copy of the next blob is ordered after this chunk's
    // kernels on the stream, and the blob itself is staged before cudaMemcpyAsync returns
    if (j1 == n_masks && full.empty()) {     // the last chunk survives until the next call
      auto& kp = c->score_keep;
      kp.m0 = c->score_m0;
      kp.nc = j1 - j;
      kp.masks.assign(hm.begin() + (size_t)j * P, hm.begin() + (size_t)j1 * P);
      kp.promo = std::move(k.promo);
      kp.vsong = k.map;
      kp.vla = k.vla;
      kp.valid = true;
    }
    j = j1;
  }
  for (int jj : full) score_full(c, d_masks + (size_t)jj * P, d_la + (size_t)jj * ns);
  CK(cudaGetLastError());
  return MG_OK;
}

}  // namespace

// ==================================================================================================
// C ABI
// ==================================================================================================
extern "C" {

mg_status mg_plan(const mg_console_desc* desc, const mg_song_desc* songs, int32_t n_songs, mg_console_info* out) {
  if (!out) return fail(nullptr, MG_ERR_INVALID, "out is null");
  mg_console tmp;
  mg_status st = validate(&tmp, desc, songs, n_songs);
  if (st != MG_OK) {
    g_static_err = tmp.err;
    return st;
  }
  plan(&tmp, desc, songs, n_songs);
  fill_info(&tmp, out);
  size_t shared_scratch = 0, keep_scratch = 0;
  const size_t arena = layout_arena(&tmp, desc, &shared_scratch, &keep_scratch);
  const bool keep = desc->retain_spectra == 1;
  out->device_bytes = (int64_t)console_device_bytes(&tmp, arena, keep ? keep_scratch : shared_scratch);
  out->launches_per_step = 0;
  out->retains_spectra = keep ? 1 : 0;
  return MG_OK;
}

mg_status mg_console_create(const mg_console_desc* desc, const mg_song_desc* songs, int32_t n_songs, cudaStream_t stream,
                            mg_console** out) {
  if (!out) return fail(nullptr, MG_ERR_INVALID, "out is null");
  *out = nullptr;
  mg_console* c = new (std::nothrow) mg_console();
  if (!c) return fail(nullptr, MG_ERR_OOM, "host allocation failed");
  c->stream = stream;
  {
    const char* dbg = std::getenv("MG_DEBUG_SYNC");
    c->debug_sync = dbg && dbg[0] == '1';
    const char* tma = std::getenv("MG_DYN_TMA");
    c->dyn_tma = !(tma && tma[0] == '0');
  }
  mg_status st = validate(c, desc, songs, n_songs);
  if (st == MG_OK) {
    std::lock_guard<std::mutex> lock(g_device_mutex);
    st = create_impl(c, desc, songs, n_songs);
  }
  if (st != MG_OK) {
    g_static_err = c->err;
    {
      std::lock_guard<std::mutex> lock(g_device_mutex);
      destroy_impl(c);
    }
    delete c;
    return st;
  }
  *out = c;
  return MG_OK;
}

mg_status mg_graph_plan(const mg_console_desc* desc, const mg_graph_desc* graph, const mg_song_desc* song,
                        mg_console_info* out, int32_t* step_type, int32_t* n_steps) {
  if (!out) return fail(nullptr, MG_ERR_INVALID, "out is null");
  mg_console tmp;
  mg_status st = validate_graph(&tmp, desc, graph, song);
  if (st == MG_OK) st = plan_graph(&tmp, desc, graph, song);
  if (st != MG_OK) {
    g_static_err = tmp.err;
    return st;
  }
  fill_info(&tmp, out);
  size_t shared_scratch = 0, keep_scratch = 0;
  const size_t arena = layout_arena(&tmp, desc, &shared_scratch, &keep_scratch);
  const bool keep = desc->retain_spectra == 1;
  out->device_bytes = (int64_t)console_device_bytes(&tmp, arena, keep ? keep_scratch : shared_scratch);
  out->launches_per_step = 0;
  out->retains_spectra = keep ? 1 : 0;
  if (n_steps) *n_steps = (int32_t)tmp.gstep_type.size();
  if (step_type)
    for (size_t k = 0; k < tmp.gstep_type.size(); ++k) step_type[k] = tmp.gstep_type[k];
  return MG_OK;
}

mg_status mg_graph_console_create(const mg_console_desc* desc, const mg_graph_desc* graph, const mg_song_desc* song,
                                  cudaStream_t stream, mg_console** out) {
  if (!out) return fail(nullptr, MG_ERR_INVALID, "out is null");
  *out = nullptr;
  mg_console* c = new (std::nothrow) mg_console();
  if (!c) return fail(nullptr, MG_ERR_OOM, "host allocation failed");
  c->stream = stream;
  {
    const char* dbg = std::getenv("MG_DEBUG_SYNC");
    c->debug_sync = dbg && dbg[0] == '1';
    const char* tma = std::getenv("MG_DYN_TMA");
    c->dyn_tma = !(tma && tma[0] == '0');
  }
  mg_status st = validate_graph(c, desc, graph, song);
  if (st == MG_OK) st = plan_graph(c, desc, graph, song);
  if (st == MG_OK) {
    std::lock_guard<std::mutex> lock(g_device_mutex);
    st = create_impl(c, desc, song, 1);
  }
  if (st != MG_OK) {
    g_static_err = c->err;
    {
      std::lock_guard<std::mutex> lock(g_device_mutex);
      destroy_impl(c);
    }
    delete c;
    return st;
  }
  *out = c;
  return MG_OK;
}

mg_status mg_console_destroy(mg_console* c) {
  if (!c) return MG_ERR_INVALID;
  cudaStreamSynchronize(c->stream);
  {
    std::lock_guard<std::mutex> lock(g_device_mutex);
    destroy_impl(c);
  }
  delete c;
  return MG_OK;
}

mg_status mg_console_get_info(const mg_console* c, mg_console_info* out) {
  if (!c || !out) return MG_ERR_INVALID;
  fill_info(c, out);
  return MG_OK;
}

mg_status mg_processor_fft(const mg_console* c, int32_t* f, int32_t* log_n, int32_t* log_n1) {
  if (!c) return MG_ERR_INVALID;
  for (int i = 0; i < c->P; ++i) {
    const HostProc& p = c->procs[i];
    const bool four = p.type == T_R || p.type == T_D;
    if (f) f[i] = four ? p.f : 0;
    if (log_n) log_n[i] = four ? p.logN : 0;
    if (log_n1) log_n1[i] = four ? p.logN1 : 0;
  }
  return MG_OK;
}

mg_status mg_processor_layout(const mg_console* c, int32_t* types, int64_t* param_offset, int32_t* song) {
  if (!c) return MG_ERR_INVALID;
  for (int i = 0; i < c->P; ++i) {
    if (types) types[i] = c->procs[i].type;
    if (param_offset) param_offset[i] = c->procs[i].poff;
    if (song) song[i] = c->procs[i].song;
  }
  return MG_OK;
}

static mg_status copy_vec(mg_console* c, float* dst, const float* src, int64_t n, int on_device, bool to_dev) {
  if (!c || !dst || !src) return fail(c, MG_ERR_INVALID, "null pointer");
  if (n != c->nparams) return fail(c, MG_ERR_INVALID, "size must equal n_params");
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : (to_dev ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost);
  CK(cudaMemcpyAsync(dst, src, sizeof(float) * n, k, c->stream));
  if (!on_device && !to_dev) CK(cudaStreamSynchronize(c->stream));
  return MG_OK;
}

mg_status mg_set_params(mg_console* c, const float* params, int64_t n, int32_t on_device) {
  mg_status s = copy_vec(c, c ? c->d_params : nullptr, params, n, on_device, true);
  if (s == MG_OK) c->fwd_valid = false;
  if (c) c->score_keep.valid = false;
  return s;
}
mg_status mg_get_params(const mg_console* c, float* out, int64_t n, int32_t on_device) {
  mg_console* m = const_cast<mg_console*>(c);
  return copy_vec(m, out, m ? m->d_params : nullptr, n, on_device, false);
}
mg_status mg_get_grads(const mg_console* c, float* out, int64_t n, int32_t on_device) {
  mg_console* m = const_cast<mg_console*>(c);
  return copy_vec(m, out, m ? m->d_grads : nullptr, n, on_device, false);
}

mg_status mg_set_alpha_p(mg_console* c, float alpha_p) {
  if (!c) return MG_ERR_INVALID;
  c->alpha_p = alpha_p;
  launch_set_hyper(c->stream, c->d_hyper, alpha_p, 0, 0, 0, 0, 0, 0);
  c->fwd_valid = false;
  c->score_keep.valid = false;
  CK(cudaGetLastError());
  return MG_OK;
}

mg_status mg_forward_loss(mg_console* c, const uint8_t* d_mask, float* d_losses, float* d_mix) {
  if (!c) return MG_ERR_INVALID;
  if (c->h_err && *(volatile int*)c->h_err)
    return fail(c, MG_ERR_TIMEOUT, "a chained envelope scan waited longer than its limit; the last results are not valid");
  if (d_mask) CK(cudaMemcpyAsync(c->d_mask, d_mask, c->P, cudaMemcpyDeviceToDevice, c->stream));
  LaunchCtx x = make_ctx(c, d_mask ? c->d_mask : nullptr);
  render(c, x);
  loss_forward(c, x, 1, d_losses, nullptr, 0);
  if (d_mix) run(c, F_MISC, [&] { launch_copy_mix(c->stream, c->d_songs, (int)c->songs.size(), d_mix, c->d_mixoff); });
  CK(cudaGetLastError());
  c->fwd_valid = d_mask == nullptr;
  c->score_keep.valid = false;
  return MG_OK;
}

mg_status mg_backward(mg_console* c) {
  if (!c) return MG_ERR_INVALID;
  if (c->h_err && *(volatile int*)c->h_err)
    return fail(c, MG_ERR_TIMEOUT, "a chained envelope scan waited longer than its limit; the last results are not valid");
  if (!c->fwd_valid) return fail(c, MG_ERR_STATE, "mg_backward needs a preceding unmasked mg_forward_loss with unchanged state");
  LaunchCtx x = make_ctx(c, nullptr);
  backward_pass(c, x);
  CK(cudaGetLastError());
  return MG_OK;
}

mg_status mg_prune_scores(mg_console* c, const uint8_t* d_masks, int32_t n_masks, float* d_la) {
  if (!c || !d_masks || !d_la || n_masks < 0) return fail(c, MG_ERR_INVALID, "null pointer or negative count");
  if (c->h_err && *(volatile int*)c->h_err)
    return fail(c, MG_ERR_TIMEOUT, "a chained envelope scan waited longer than its limit; the last results are not valid");
  if (n_masks == 0) return MG_OK;
  mg_status st = MG_OK;
  if (c->per_node || c->score_mode == 1 || c->is_graph) {
    c->score_keep.valid = false;
    // one full masked render per candidate
    for (int j = 0; j < n_masks; ++j) score_full(c, d_masks + (size_t)j * c->P, d_la + (size_t)j * c->songs.size());
    CK(cudaGetLastError());
  } else {
    st = prune_scores_batched(c, d_masks, n_masks, d_la);
  }
  c->fwd_valid = false;
  return st;
}

mg_status mg_debug_chain_hold(mg_console* c, int32_t on) {
  if (!c) return MG_ERR_INVALID;
  c->chain_hold = on ? 1 : 0;
  if (!on && c->h_err) *(volatile int*)c->h_err = 0;   // releasing the hold also clears a reported timeout
  if (c->graph) {                                      // the captured step holds the old setting
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  return MG_OK;
}

mg_status mg_set_score_mode(mg_console* c, int32_t mode) {
  if (!c || mode < 0 || mode > 1) return fail(c, MG_ERR_INVALID, "score mode must be 0 or 1");
  c->score_mode = mode;
  return MG_OK;
}

mg_status mg_adam_step(mg_console* c, float lr, float beta1, float beta2, float eps, float weight_decay) {
  if (!c) return MG_ERR_INVALID;
  launch_set_hyper(c->stream, c->d_hyper, 0, lr, beta1, beta2, eps, weight_decay, 1);
  run(c, F_ADAM, [&] { launch_adam2(c->stream, c->d_hyper, c->d_step, c->d_params, c->d_grads, c->d_m, c->d_v, c->nparams); });
  c->fwd_valid = false;
  c->score_keep.valid = false;
  CK(cudaGetLastError());
  return MG_OK;
}

mg_status mg_reset_optimizer(mg_console* c) {
  if (!c) return MG_ERR_INVALID;
  CK(cudaMemsetAsync(c->d_m, 0, sizeof(float) * c->nparams, c->stream));
  CK(cudaMemsetAsync(c->d_v, 0, sizeof(float) * c->nparams, c->stream));
  CK(cudaMemsetAsync(c->d_step, 0, sizeof(int), c->stream));
  return MG_OK;
}

mg_status mg_train_step(mg_console* c, float lr, float beta1, float beta2, float eps, float weight_decay, float* d_losses) {
  if (!c) return MG_ERR_INVALID;
  if (c->h_err && *(volatile int*)c->h_err)
    return fail(c, MG_ERR_TIMEOUT, "a chained envelope scan waited longer than its limit; the last results are not valid");
  launch_set_hyper(c->stream, c->d_hyper, 0, lr, beta1, beta2, eps, weight_decay, 1);
  if (c->per_node) {  // one-by-one processing runs eagerly (no graph)
    LaunchCtx x = make_ctx(c, nullptr);
    render(c, x);
    loss_forward(c, x, 1, d_losses, nullptr, 0);
    backward_pass(c, x);
    run(c, F_ADAM, [&] { launch_adam2(c->stream, c->d_hyper, c->d_step, c->d_params, c->d_grads, c->d_m, c->d_v, c->nparams); });
    c->fwd_valid = false;
    c->score_keep.valid = false;
    CK(cudaGetLastError());
    return MG_OK;
  }
  if (!c->graph || c->graph_losses != d_losses || c->graph_profiled != c->profiling) {
    if (c->graph) {
      cudaGraphExecDestroy(c->graph);
      c->graph = nullptr;
    }
    c->graph_pairs.clear();
    c->ev_next = 0;
    cudaGraph_t g;
    std::lock_guard<std::mutex> capture_lock(g_device_mutex);
    c->capturing = true;
    c->launches = 0;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    LaunchCtx x = make_ctx(c, nullptr);
    render(c, x);
    loss_forward(c, x, 1, d_losses, nullptr, 0);
    backward_pass(c, x);
    run(c, F_ADAM, [&] { launch_adam2(c->stream, c->d_hyper, c->d_step, c->d_params, c->d_grads, c->d_m, c->d_v, c->nparams); });
    c->capturing = false;
    c->launches_step = c->launches;
    CK(cudaStreamEndCapture(c->stream, &g));
    CK(cudaGraphInstantiate(&c->graph, g, 0));
    cudaGraphDestroy(g);
    c->graph_losses = d_losses;
    c->graph_profiled = c->profiling;
  }
  CK(cudaGraphLaunch(c->graph, c->stream));
  if (c->profiling) {
    CK(cudaStreamSynchronize(c->stream));
    for (auto& pr : c->graph_pairs) accumulate_pair(c, pr.first, pr.second.first, pr.second.second);
  }
  c->fwd_valid = false;
  c->score_keep.valid = false;
  return MG_OK;
}

mg_status mg_prune(mg_console* c, const uint8_t* h_keep) {
  if (!c || !h_keep) return fail(c, MG_ERR_INVALID, "null pointer");
  CK(cudaStreamSynchronize(c->stream));
  std::lock_guard<std::mutex> lock(g_device_mutex);   // rebuilds device tables (allocation and release)
  for (int i = 0; i < c->P; ++i)
    if (!h_keep[i]) c->procs[i].present = 0;
  if (build_tables(c) != MG_OK) return MG_ERR_CUDA;
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  c->fwd_valid = false;
  c->score_keep.valid = false;
  CK(cudaStreamSynchronize(c->stream));
  return MG_OK;
}

mg_status mg_get_present(const mg_console* c, uint8_t* h_present) {
  if (!c || !h_present) return MG_ERR_INVALID;
  for (int i = 0; i < c->P; ++i) h_present[i] = (uint8_t)c->procs[i].present;
  return MG_OK;
}

mg_status mg_evaluate(mg_console* c, float* d_out) {
  if (!c || !d_out) return fail(c, MG_ERR_INVALID, "null pointer");
  launch_eval(c->stream, c->d_songs, (int)c->songs.size(), c->d_ev_items, (int)c->ev_items.size(), c->d_ev_begin,
              c->ev_seg_len, c->d_ev_lo, c->d_ev_hi, c->d_ev_out, d_out, c->tab.ptw);
  CK(cudaGetLastError());
  return MG_OK;
}

mg_status mg_update_audio(mg_console* c, int32_t song, const float* sources, const float* target, int32_t on_device) {
  if (!c || song < 0 || song >= (int)c->songs.size() || !sources) return fail(c, MG_ERR_INVALID, "bad song or null sources");
  const HostSong& hs = c->songs[song];
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  // Sources the device can read (device memory, or page-locked host memory mapped into the address space) go
  // into both rows of every track input in one kernel launch; pageable host memory is copied track by track
  // (once across, then a device-side copy of the left row to the right one).
  const float* readable = on_device ? sources : nullptr;
  if (!on_device) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, sources) == cudaSuccess && a.type == cudaMemoryTypeHost && a.devicePointer)
      readable = static_cast<const float*>(a.devicePointer);
    else
      cudaGetLastError();   // pageable memory: not an error
  }
  if (readable && c->d_track_in) {
    launch_ingest_song(c->stream, readable, c->d_track_in + c->track_in_base[song], hs.K, hs.L, hs.ld);
  } else {
    for (int t = 0; t < hs.K; ++t) {
      float* dst = (float*)(c->arena + (c->is_graph ? c->o_src[t] : c->chains[hs.tracks_chain[t]].o_in));
      CK(cudaMemcpyAsync(dst, sources + (size_t)t * hs.L, sizeof(float) * hs.L, k, c->stream));
      CK(cudaMemcpyAsync(dst + hs.ld, dst, sizeof(float) * hs.L, cudaMemcpyDeviceToDevice, c->stream));
    }
  }
  if (target) {
    CK(cudaMemcpy2DAsync(c->arena + hs.o_tgt, (size_t)hs.ld * sizeof(float), target, (size_t)hs.L * sizeof(float),
                         (size_t)hs.L * sizeof(float), 2, k, c->stream));
    // target spectrograms and their norms of this song only
    LaunchCtx x = make_ctx(c, nullptr);
    for (int r = 0; r < c->nres; ++r) {
      const int2 rg = c->song_litems[song][r];
      if (rg.y > 0) launch_loss_frames(x, c->d_songs, c->d_res, c->loss_items[r].d + rg.x, rg.y, 0, c->loss_max_dy);
    }
    launch_loss_finalize_mode(x, c->d_songs + song, 1, c->d_res, c->nres, c->d_alphas, 0, nullptr, nullptr, 0);
  }
  c->fwd_valid = false;
  c->score_keep.valid = false;
  CK(cudaGetLastError());
  return MG_OK;
}

mg_status mg_set_launch_mode(mg_console* c, int32_t per_node) {
  if (!c) return MG_ERR_INVALID;
  c->per_node = per_node != 0;
  return MG_OK;
}

mg_status mg_set_profiling(mg_console* c, int32_t on) {
  if (!c) return MG_ERR_INVALID;
  c->profiling = on != 0;
  return MG_OK;
}

int32_t mg_num_kernel_families(void) { return F_COUNT; }
const char* mg_kernel_family_name(int32_t f) { return (f >= 0 && f < F_COUNT) ? kFamilyNames[f] : ""; }

mg_status mg_get_kernel_times(mg_console* c, double* ms, int64_t* launches, int32_t n) {
  if (!c) return MG_ERR_INVALID;
  CK(cudaStreamSynchronize(c->stream));
  for (auto& pr : c->pending) accumulate_pair(c, pr.first, pr.second.first, pr.second.second);
  c->pending.clear();
  if (!c->capturing && c->graph_pairs.empty()) c->ev_next = 0;
  for (int i = 0; i < n && i < F_COUNT; ++i) {
    if (ms) ms[i] = c->fam_ms[i];
    if (launches) launches[i] = c->fam_n[i];
  }
  return MG_OK;
}

mg_status mg_get_stage_times(mg_console* c, double* ms, int64_t* launches, int32_t n) {
  if (!c) return MG_ERR_INVALID;
  double tmp[F_COUNT];
  mg_status s = mg_get_kernel_times(c, tmp, nullptr, F_COUNT);   // folds pending event pairs in
  if (s != MG_OK) return s;
  for (int i = 0; i < n && i < 10; ++i) {
    if (ms) ms[i] = c->stage_ms[i];
    if (launches) launches[i] = c->stage_n[i];
  }
  return MG_OK;
}

mg_status mg_reset_kernel_times(mg_console* c) {
  if (!c) return MG_ERR_INVALID;
  for (int i = 0; i < 10; ++i) {
    c->stage_ms[i] = 0;
    c->stage_n[i] = 0;
  }
  for (int i = 0; i < F_COUNT; ++i) {
    c->fam_ms[i] = 0;
    c->fam_n[i] = 0;
  }
  return MG_OK;
}

mg_status mg_debug_read(const mg_console* cc, int32_t proc, int32_t what, float* host_out, int64_t n) {
  mg_console* c = const_cast<mg_console*>(cc);
  if (!c || !host_out || proc < 0 || proc >= c->P) return fail(c, MG_ERR_INVALID, "bad processor or null output");
  const ProcDev& d = c->hpd[proc];
  const HostProc& p = c->procs[proc];
  const float* src = nullptr;
  int64_t rows = 2, cols = 0, ld = 0;
  switch (what) {
    case 0: src = d.y; cols = p.L; ld = p.ld; break;
    case 1: src = d.taps; cols = p.Nh; ld = p.Nh; break;
    case 2: src = d.dtaps; cols = p.Nh; ld = p.Nh; break;
    case 3: src = d.du; cols = p.L; ld = p.ld; break;
    case 4: src = d.stats; rows = 1; cols = 16; ld = 16; break;
    case 5: src = d.dy; cols = p.L; ld = p.ld; break;
    default: return fail(c, MG_ERR_INVALID, "unknown buffer");
  }
  if (!src) return fail(c, MG_ERR_INVALID, "buffer not present for this processor");
  if (n != rows * cols) return fail(c, MG_ERR_INVALID, "size mismatch");
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemcpy2D(host_out, cols * sizeof(float), src, ld * sizeof(float), cols * sizeof(float), rows,
                  cudaMemcpyDeviceToHost));
  return MG_OK;
}

const char* mg_last_error(const mg_console* c) { return c ? c->err.c_str() : g_static_err.c_str(); }

}  // extern "C"

// Internal declarations shared by the kernels and the host engine of the mixing-console library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mg {

enum ProcType { T_E = 0, T_C = 1, T_N = 2, T_S = 3, T_G = 4, T_D = 5, T_R = 6, NTYPES = 7 };

constexpr int kTwLog = 13;                 // shared twiddle table exp(-2 pi i j / 8192)
constexpr int kTwN = 1 << kTwLog;
constexpr int kTwFineLog = 26;            // fine table exp(-2 pi i j / 2^26), j < 8192: twiddles of N <= 2^26
constexpr int kNPart = 8;                  // partial sums per work item
// Per-node statistics: 0 E_ybar_mid, 1 E_u_mid, 2 c1, 3 c2, 4..11 backward sums, 16..21 the channel scales of
// the packed stereo transforms (u, taps, dL/dy_bar; left then right)
constexpr int kStatsFloats = 32;
constexpr int kScaleU = 16, kScaleH = 18, kScaleD = 20;
constexpr int kEqTaps = 2047;              // Sec. 3.3
constexpr int kEqHalf = 1023;
constexpr int kEqParams = 1024;
constexpr int kDlyFir = 39;                // Sec. 3.7
constexpr int kDlyHalf = 19;
constexpr int kDlyTaps = 20;
constexpr int kDlyPer = 22;                // Re z, Im z, 20 log-magnitudes
constexpr int kRevFft = 384;               // Sec. 3.4
constexpr int kRevHop = 192;
constexpr int kRevBins = 193;
constexpr int kRevParams = 192;
constexpr int kRevFG = 16;                 // frames per reverb work item
constexpr int kDynChunk = 4096;            // samples per envelope-scan work item (256 threads x 16)
constexpr int kElemTile = 4096;            // samples per elementwise work item (default; tuned per console)
constexpr int kElemTileMin = 1024;         // smallest candidate of the packing tuner
constexpr int kLossPerDiv = 4;             // loss work items hold 8192 / n_fft frames, or down to a quarter of that
constexpr float kEnvEps = 1e-8f;           // G_u = ln(g + eps)
constexpr int kLossFrameBuf = 8192 + 512 + 128;   // padded frames of one loss work item (float2)
// floats of the loss adjoint's band gradients that fit next to the frames in the 227 KB of shared memory a
// CTA may hold (1 KB left for the kernel's static shared memory)
constexpr int kLossMaxDy = (227 * 1024 - 1024 - kLossFrameBuf * 8) / 4;
constexpr int kEqOsM = 8192;               // overlap-save FFT size of the equalizer
constexpr int kEqOsFwdBlock = kEqOsM - 2 * kEqHalf;        // 6146 outputs per forward block
constexpr int kEqChunk = 8;                 // equalizer backward: blocks per work item (spectra summed in registers)

struct Item {
  int proc;
  int idx;
};

// Device view of one processor node (flattened over all songs).
struct ProcDev {
  int type, song, qidx, L, ld;             // ld: channel stride of every [2][ld] buffer
  int present;                             // 0 once removed by structural pruning
  int rev;                                 // rank among reverbs (noise index), -1 otherwise
  const float* u;                          // forward input  [2][ld]
  float* y;                                // forward output [2][ld]
  const float* dy;                         // adjoint of y
  float* du;                               // adjoint of u
  const float* p;                          // parameters of this processor
  float* gp;                               // gradient of those parameters
  float* fpart;                            // forward partials  [items][kNPart]
  float* bpart;                            // backward partials [items][kNPart]
  int nfpart, nbpart;                      // number of partial rows written by the main pass
  float* stats;                            // [kStatsFloats]: 0 E_ybar_mid, 1 E_u_mid, 2 c1, 3 c2, 4.. backward sums,
                                           // kScaleU.. channel scales of the packed transforms
  // LTI processors (r, d): four-step FFT convolution of size N = N1 * N2 = f 2^logN, N1 = f 2^logN1 (rows),
  // N2 = 2^logN2 (columns), f in {1, 3}
  int logN, logN1, logN2, colG;            // colG: columns per column-pass work item
  int f;
  float2 cfn[5];                           // exp(-2 pi i r / N), r < f (transposition twiddles when f = 3, 5)
  int n0, Nh;                              // FIR: first tap time, number of taps
  float2* T1;
  float2* T2;
  float2* Hz;
  float* taps;                             // [2][Nh]
  float* dtaps;                            // [2][Nh]
  float* aux;                              // type scratch (delay: c_m and d_m; reverb: adjoint partials;
                                           // compressor, noisegate: dL/dg per sample)
  // envelope scans (c, n)
  float* carry;                            // [nchunks] forward state entering each chunk
  float* chunkagg;                         // [nchunks] per-chunk aggregates
  unsigned long long* cflag;               // [nchunks] chained-scan states: launch generation << 32 | state bits
  const void* umap;                        // c, n: tensor map (TMA) of u as rows of 32 floats, or nullptr
  const void* dymap;                       // c, n: the same of dL/dy (backward), or nullptr
  int nchunks;
  // reverb
  const float2* nspec;                     // [2][F][193] STFT of the fixed mid/side noise
  int nframes;                             // F
  // equalizer (overlap-save)
  float* hspec;                            // [8192] real spectrum of the FIR on the overlap-save grid
  float* ybar;                             // [2][ld] wet signal kept by the forward for the backward
  float2* dhspec;                          // [backward items][8192] summed spectra of the tap correlation
  float2* eqg;                             // [forward blocks][8192] spectra D H of the equalizer backward
};

struct LossRes {                           // one STFT resolution of Eq. (21)
  int nfft, log_nfft, hop, nbands;
  int per;                                 // frames per work item (at most 8192 / nfft; packing tuner)
  const float* win;                        // [nfft] periodic Hann
  const float* aw2;                        // [nfft/2+1] squared A-weighting gain
  const int* band_beg;                     // [nbands+1] CSR over (bin, weight) by band
  const int* band_bin;
  const float* band_w;
  const int* bin_beg;                      // [nfft/2+2] CSR over (band, weight) by bin
  const int* bin_band;
  const float* bin_w;
};

struct SongDev {
  int L, ld, nframes[3], first_frame[3];
  const float* mix;                        // [2][ld]
  float* dmix;                             // [2][ld]
  const float* target;
  float* Y[3];                             // target spectrograms [frames][nbands][4] (L, R, M, S)
  float* Yh[3];                            // spectrograms of the mix kept by the training forward, same layout
  float* dF[3];                            // backward per-frame gradients [frames][nfft] (packed complex)
  float* lpart;                            // loss partials [3][lcap][6]
  int litems[3];                           // items per resolution
  int lcap;
  int pbeg, pend;                          // canonical processor range of the song
  float* coef;                             // [3 res][3 sets][2]: backward coefficients
  double* ynorm2;                          // [3 res][3 sets] squared Frobenius norms of the target
};

// ----------------------------------------------------------------------------------------------
// launch wrappers (kernels live in the k_*.cu files)
// ----------------------------------------------------------------------------------------------
struct Tables {
  const float2* tw;                        // exp(-2 pi i j / 8192)
  const float2* twf;                       // exp(-2 pi i j / 2^26), j < 8192 (fine factor of large-N twiddles)
  const float2* c3;                        // [14][3] exp(-2 pi i r / (3 2^a)): twiddles of 3 2^a-point FFTs
  const float2* ptw;                       // pass twiddles of the 2^a-point FFTs (layout of ptw_base)
  const float2* ptw3;                      // pass twiddles of the 3 2^a-point FFTs (layout of ptwf_base)
  const float2* ptw5;                      // pass twiddles of the 5 2^a-point FFTs
  const float* cos_eq;                     // cos(2 pi m / 2047), m < 2047
  const float* cos_dl;                     // cos(2 pi m / 39), m < 39
  const float* rev_win;                    // periodic Hann 384
  const float2* rev_cs;                    // (cos, sin)(2 pi m / 384), m < 384
  const float* hann_eq;                    // symmetric Hann v[n], n = -1023..1023
  const float* hann_dl;                    // symmetric Hann v[n], n = -19..19
  const float2* dly_w;                     // exp(+2 pi i q / D), q < D (delay slot length D)
};

struct LaunchCtx {
  cudaStream_t stream;
  const ProcDev* procs;                    // device
  const float* q;                          // dry/wet logits [P]
  const uint8_t* mask;                     // [P] or null (all ones)
  const float* hyper;                      // device: 0 alpha_p, 1 lr, 2 beta1, 3 beta2, 4 eps, 5 weight decay
  float alpha_g;
  double fs;
  int elem_tile;                           // samples per work item of the gain/pan and imager kernels
  unsigned* chain;                         // device [2]: launch generation and work ticket of the chained scans
  int* err;                                // host-mapped error word: 1 = a chained scan's wait ran out
  int chain_hold;                          // test hook: the first work item does not publish its state
  int dyn_tma;                             // the scans' nodes may carry tensor maps (their launches reserve the stage)
  Tables tab;
};

// elementwise processors, sums, ingest
void launch_gs_fwd(const LaunchCtx&, const Item* items, int n);
void launch_gs_bwd(const LaunchCtx&, const Item* items, int n);
void launch_sum(cudaStream_t, float* const* outs, const float* const* ins, const int* in_beg, const int* L,
                const int* ld, const Item* items, int n, int tile);
void launch_ingest(cudaStream_t, const float* mono, float* stereo, int L, int ld);
void launch_ingest_song(cudaStream_t, const float* mono, float* const* dst, int K, int L, int ld);
// envelope scans: chained single-pass forward (items in chunk order) and backward (items in reverse chunk order)
void launch_dyn_fwd(const LaunchCtx&, const Item* items, int n);
void launch_dyn_bwd(const LaunchCtx&, const Item* items, int n);
// LTI processors
void launch_eq_fir(const LaunchCtx&, const int* procs, int n);
void launch_eq_fir_adj(const LaunchCtx&, const int* procs, int n);
void launch_dly_prep(const LaunchCtx&, const int* procs, int n);
void launch_dly_fir(const LaunchCtx&, const Item* items, int n);
void launch_dly_adj(const LaunchCtx&, const Item* items, int n);
void launch_rev_fir(const LaunchCtx&, const Item* items, int n);
void launch_rev_adj(const LaunchCtx&, const Item* items, int n);
void launch_rev_adj_fin(const LaunchCtx&, const int* procs, int n);
void launch_rev_noise_stft(const LaunchCtx&, const Item* items, int n, const float* noise, int noise_len);
void init_col_attributes();      // column passes of the four-step convolution (called by the last)
void init_dyn_attributes();      // compressor / gate scans (called by the last)
void init_row_bwd_attributes();  // backward row pass (called by the next)
void init_kernel_attributes();
void init_loss_attributes();
void init_fir_attributes();
void init_eqos_attributes();
void launch_eq_spec(const LaunchCtx&, const int* procs, int n);
void launch_eq_os_fwd(const LaunchCtx&, const Item* items, int n);
void launch_eq_os_bwd(const LaunchCtx&, const Item* items, int n);
void launch_eq_os_du(const LaunchCtx&, const Item* items, int n);
void launch_eq_dh_reduce(const LaunchCtx&, const int* procs, int n);
void launch_col_fwd_audio(const LaunchCtx&, const Item* items, int n, int maxN2G);
void launch_col_fwd_taps(const LaunchCtx&, const Item* items, int n, int maxN2G);
void launch_row_fwd_hz(const LaunchCtx&, const Item* items, int n, int maxN1);
void launch_row_conv_fwd(const LaunchCtx&, const Item* items, int n, int maxN1, bool bwd_keep_u);
void launch_col_inv_out(const LaunchCtx&, const Item* items, int n, int maxN2G);
void launch_col_dybar(const LaunchCtx&, const Item* items, int n, int maxN2G);
void launch_eval(cudaStream_t st, const SongDev* songs, int n_songs, const int2* items, int n_items,
                 const int* item_begin, int seg_len, const int* band_lo, const int* band_hi, double* seg_out,
                 float* out_song, const float2* ptw);
void init_eval_attributes();
void launch_col_inv_out_keep(const LaunchCtx&, const Item* items, int n, int maxN2G);
void launch_col_dybar_keep(const LaunchCtx&, const Item* items, int n, int maxN2G);
void launch_row_bwd2(const LaunchCtx&, const Item* items, int n, int maxN1);
void launch_col_du(const LaunchCtx&, const Item* items, int n, int maxN2G);
// channel scales of the packed stereo transforms: which 0 = input u and taps (forward), 1 = dL/dy (backward)
void launch_chan_scale(const LaunchCtx&, const int* procs, int n, int which);
void launch_col_dh(const LaunchCtx&, const Item* items, int n, int maxN2G);
// reductions, loss, optimiser
void launch_node_stats(const LaunchCtx&, const int* procs, int n, int fwd);
// max_dy: floats of the adjoint's band-gradient buffer, max over resolutions of (8192 / n_fft) bands 4
void launch_loss_frames(const LaunchCtx&, const SongDev* songs, const LossRes* res, const int4* items, int n,
                        int mode, int max_dy);
void launch_loss_finalize_mode(const LaunchCtx&, const SongDev* songs, int nsongs, const LossRes* res, int nres,
                               const float* alphas, int mode, float* out_losses, float* out_la, int la_stride);
void launch_loss_gather(const LaunchCtx&, const SongDev* songs, const LossRes* res, int nres, const Item* items,
                        int n);
void launch_grad_finalize2(const LaunchCtx&, const int* procs, int n, float* gq);
void launch_adam2(cudaStream_t, const float* hyper, int* step, float* p, const float* g, float* m, float* v,
                  int64_t n);
void launch_set_hyper(cudaStream_t, float* hyper, float alpha_p, float lr, float b1, float b2, float eps, float wd,
                      int which);
void launch_copy_mix(cudaStream_t, const SongDev* songs, int nsongs, float* out, const int64_t* offs);
// candidate scoring
void launch_gather_q(cudaStream_t, const float* q, const int* src, float* dst, int n);
void launch_score_scatter(cudaStream_t, const int* map, const float* vla, const float* base_la, float* out, int n,
                          int nsongs);

}  // namespace mg

// Column passes of the four-step FFT convolution (see k_conv_common.cuh).
#include <cstdint>
#include <cstdio>

#include "k_conv_common.cuh"

namespace mg {

namespace {

// COL_INV_OUT_KEEP / COL_DYBAR_KEEP: the retained-spectra variants.  The forward's inverse column pass reads the
// product rows from T2 and also stores the wet signal y_bar in natural order over T2 (the positions the CTA read);
// the backward's dL/dy_bar pass then loads y_bar from there instead of transforming the product again.
enum ColMode {
  COL_FWD_AUDIO = 0, COL_FWD_TAPS = 1, COL_INV_OUT = 2, COL_DYBAR = 3, COL_DU = 4, COL_DH = 5,
  COL_INV_OUT_KEEP = 6, COL_DYBAR_KEEP = 7
};

// A column tile is G adjacent columns of the N1 x N2 grid (N2 * G <= 8192 elements, 512 threads).  Because the
// block size is a multiple of G, every thread stays on one column g and handles the rows r0 + s * RS
// (RS = 512 / G, s < kSlots): the global positions of its elements step by RS * N1, its loads are independent
// and issued eight at a time before the shared-memory stores, and the epilogues batch their side loads
// (input u, upstream gradient dy) four slots at a time.
constexpr int kSlots = 8192 / kColThreads;

// Transposition twiddles of the tile's columns, W(n1 k2) = lo[k2 mod 64] hi[k2 / 64] (W = exp(-2 pi i / N),
// N2 / 64 <= 32 hi entries), both factors from the accurate table; column gg at ctw + gg * kColTwS.  The column
// stride is 4 (mod 16) float2 so that the eight columns x four rows of a warp's lookups spread evenly over the
// bank pairs.  Visible after the caller's next barrier.
constexpr int kColTwS = 100;
__device__ __forceinline__ void col_tw_init(float2* ctw, const ProcDev& P, int n1b, int G, int N2, const Tables& tab) {
  for (int e = threadIdx.x; e < G * kColTwS; e += blockDim.x) {
    const int gg = e / kColTwS, j = e - gg * kColTwS;
    const unsigned n1 = (unsigned)(n1b + gg);
    const unsigned k2 = j < 64 ? (unsigned)j : (unsigned)(j - 64) << 6;   // the lo power, or the hi power
    ctw[e] = k2 < (unsigned)N2 ? twiddle_node(P, n1 * k2, false, tab) : make_float2(1.f, 0.f);
  }
}

template <int MODE>
__global__ void __launch_bounds__(kColThreads, 2) k_col(LaunchCtx c, const Item* __restrict__ items) {
  extern __shared__ float2 sm[];
  __shared__ float red[2 * 32];
  __shared__ float2 ctw[8 * kColTwS];
  const Item it = items[blockIdx.x];
  const ProcDev& P = c.procs[it.proc];
  const int G = P.colG, logG = __ffs(G) - 1;
  const int logN2 = P.logN2, N2 = 1 << logN2, N1 = rows_len(P);
  const int64_t N = fft_len(P);
  const int cs = col_stride(N2, G);
  constexpr bool kOut = MODE == COL_INV_OUT || MODE == COL_INV_OUT_KEEP;
  constexpr bool kDybar = MODE == COL_DYBAR || MODE == COL_DYBAR_KEEP;

  const int g = threadIdx.x & (G - 1), r0 = threadIdx.x >> logG;
  const int RS = blockDim.x >> logG;
  const int n1 = it.idx * G + g;
  const int64_t nbase = (int64_t)n1 + (int64_t)r0 * N1;
  const int64_t nstep = (int64_t)RS * N1;
  float2* col = sm + g * cs;
  auto row_of = [&](int s) { return r0 + s * RS; };
  auto live = [&](int s) { return row_of(s) < N2; };
  auto pos = [&](int s) { return nbase + (int64_t)s * nstep; };

  // The column transforms run with the batch-fastest thread order (eight adjacent columns of one row per
  // quarter warp), so their first pass reads, and a forward transform's last pass writes, global memory
  // directly.  Forward transforms end with the transposition twiddle W(n1 k2), W = exp(-2 pi i / N).
  constexpr bool kTwid = !(MODE == COL_INV_OUT || MODE == COL_DU || MODE == COL_DH || MODE == COL_INV_OUT_KEEP);
  const int n1b = it.idx * G;
  if (kTwid) col_tw_init(ctw, P, n1b, G, N2, c.tab);
  auto tw_store = [&](float2* dst) {
    return [&, dst](int gg, int k2, float2 v) {
      const float2* t = ctw + gg * kColTwS;
      dst[n1b + gg + (int64_t)N1 * k2] = cmul(v, cmul(t[k2 & 63], t[64 + (k2 >> 6)]));
    };
  };

  if (MODE == COL_FWD_AUDIO || MODE == COL_FWD_TAPS) {   // forward pass of the input or the taps, in place
    const float* u = P.u;
    const int L = P.L, ld = P.ld;
    const float2 sc = chan_scale(P, MODE == COL_FWD_AUDIO ? kScaleU : kScaleH);
    fft_p_io<false, 1, true>(sm, logN2, G, cs, c.tab.ptw, [&](int gg, int n2) {
      const int64_t n = n1b + gg + (int64_t)N1 * n2;
      if (MODE == COL_FWD_AUDIO) return n < L ? make_float2(u[n] * sc.x, u[ld + n] * sc.y) : make_float2(0.f, 0.f);
      const float2 t = tap_at(P, n, N);
      return make_float2(t.x * sc.x, t.y * sc.y);
    }, tw_store(MODE == COL_FWD_TAPS ? P.Hz : P.T1));
    return;
  }

  // ---- load: the inverse transform reads the rows of T1 / T2 in its first pass ----
  if (MODE != COL_DYBAR_KEEP) {
    const float2* src = (MODE == COL_INV_OUT || MODE == COL_DH) ? P.T1 : P.T2;
    fft_p_io<true, 1, true>(sm, logN2, G, cs, c.tab.ptw,
                            [&](int gg, int n2) { return src[n1b + gg + (int64_t)N1 * n2]; });
  }

  const float inv_n = ldexpf(1.f, -P.logN) / (float)P.f;
  // 1/N divided by the channel scales of the two transformed operands
  const float2 su = chan_scale(P, kScaleU), sh = chan_scale(P, kScaleH), sd = chan_scale(P, kScaleD);
  const float2 inv_uh = make_float2(inv_n / (su.x * sh.x), inv_n / (su.y * sh.y));
  auto unscale = [](float2 v, float2 s) { return make_float2(v.x * s.x, v.y * s.y); };
  if (kOut) {
    const float w = dry_wet_w(c, P.qidx), wd = dry_wet_d(c, P.qidx);
    float acc[2] = {0.f, 0.f};
#pragma unroll 1
    for (int h = 0; h < kSlots; h += 4) {
      float ul[4], ur[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t n = pos(h + j);
        ul[j] = ur[j] = 0.f;
        if (live(h + j) && n < P.L) {
          ul[j] = P.u[n];
          ur[j] = P.u[P.ld + n];
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t n = pos(h + j);
        if (!live(h + j) || n >= P.L) continue;
        const float2 yb = unscale(col[pidx(row_of(h + j))], inv_uh);
        if (MODE == COL_INV_OUT_KEEP) P.T2[n] = yb;
        P.y[n] = w * yb.x + wd * ul[j];
        P.y[P.ld + n] = w * yb.y + wd * ur[j];
        const float ym = yb.x + yb.y, um = ul[j] + ur[j];
        acc[0] += ym * ym;
        acc[1] += um * um;
      }
    }
    float out[2];
    block_sum<2>(acc, red, out);
    if (threadIdx.x == 0) {
      P.fpart[it.idx * kNPart + 0] = out[0];
      P.fpart[it.idx * kNPart + 1] = out[1];
    }
    return;
  }
  if (kDybar) {
    // y_bar -> dL/dy_bar = w dy + c1 (y_bar_l + y_bar_r) on both channels; dw partial; then forward FFT.
    // Retained spectra: y_bar is read in natural order from T2; otherwise it is the inverse column FFT above.
    const float w = dry_wet_w(c, P.qidx);
    const float c1 = P.stats[2];
    float acc[1] = {0.f};
#pragma unroll 1
    for (int h = 0; h < kSlots; h += 4) {
      float2 yb[4];
      float gl[4], gr[4], ul[4], ur[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t n = pos(h + j);
        yb[j] = make_float2(0.f, 0.f);
        gl[j] = gr[j] = ul[j] = ur[j] = 0.f;
        if (live(h + j) && n < P.L) {
          yb[j] = MODE == COL_DYBAR_KEEP ? P.T2[n] : unscale(col[pidx(row_of(h + j))], inv_uh);
          gl[j] = P.dy[n];
          gr[j] = P.dy[P.ld + n];
          ul[j] = P.u[n];
          ur[j] = P.u[P.ld + n];
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (!live(h + j)) continue;
        acc[0] += gl[j] * (yb[j].x - ul[j]) + gr[j] * (yb[j].y - ur[j]);
        const float gm = c1 * (yb[j].x + yb[j].y);
        // rows past the signal are zero (gl = gr = 0 and y_bar = 0 there)
        col[pidx(row_of(h + j))] = make_float2(sd.x * (w * gl[j] + gm), sd.y * (w * gr[j] + gm));
      }
    }
    float out[1];
    block_sum<1>(acc, red, out);   // also acts as the barrier before the FFT
    if (threadIdx.x == 0) P.bpart[it.idx * kNPart + 0] = out[0];
    fft_p_io<false, 1, true>(sm, logN2, G, cs, c.tab.ptw, fftp::SmemIO(), tw_store(P.T2));
    return;
  }
  if (MODE == COL_DU) {
    const float wd = dry_wet_d(c, P.qidx);
    const float c2 = P.stats[3];
    const float2 inv_dh = make_float2(inv_n / (sd.x * sh.x), inv_n / (sd.y * sh.y));
#pragma unroll 1
    for (int h = 0; h < kSlots; h += 4) {
      float gl[4], gr[4], um[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t n = pos(h + j);
        gl[j] = gr[j] = um[j] = 0.f;
        if (live(h + j) && n < P.L) {
          gl[j] = P.dy[n];
          gr[j] = P.dy[P.ld + n];
          um[j] = c2 * (P.u[n] + P.u[P.ld + n]);
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t n = pos(h + j);
        if (!live(h + j) || n >= P.L) continue;
        const float2 dw = unscale(col[pidx(row_of(h + j))], inv_dh);
        P.du[n] = wd * gl[j] + dw.x + um[j];
        P.du[P.ld + n] = wd * gr[j] + dw.y + um[j];
      }
    }
    return;
  }
  if (MODE == COL_DH) {
    const float2 inv_du = make_float2(inv_n / (sd.x * su.x), inv_n / (sd.y * su.y));
#pragma unroll 4
    for (int s = 0; s < kSlots; ++s) {
      if (!live(s)) continue;
      const int64_t n = pos(s);
      int64_t j = -1;
      if (n < (int64_t)P.n0 + P.Nh) j = n - P.n0;
      else if (n >= N + P.n0) j = n - N - P.n0;
      if (j >= 0 && j < P.Nh) {
        // dL/dh[t] = sum_n dL/dy_bar[n] u[n - t] is identically zero for lags t >= L: store the exact zero
        // instead of the FFT rounding residue (the delay's Eq. 19 direction takes sgn(0) = 0 there)
        const float2 v = (j + P.n0 >= P.L) ? make_float2(0.f, 0.f) : unscale(col[pidx(row_of(s))], inv_du);
        P.dtaps[j] = v.x;
        P.dtaps[P.Nh + j] = v.y;
      }
    }
  }
}

// Channel scales of one node (one CTA per node): per channel the energy of four consecutive samples out of every
// 128, and of the taps: every 32nd tap of the reverb's dense FIR, all 20 x 39 nonzero taps c_m of the delay's
// sparse one (a stride would miss whole 39-tap windows).  The scale s = 1/sqrt(e) brings that energy to one, so
// both channels of a packed transform sit at the same level up to the sampling error of the estimate; 1 for a
// silent channel.  (Power-of-two scales, exact to apply, left the channels up to 2x apart in amplitude, and the
// weaker channel's error moved by that factor with the estimate's rounding.)
// which 0: the input u and the taps (in the stereo form the transforms use); 1: dL/dy.  Fixed-order sums.
__device__ __forceinline__ float unit_scale(float e) {
  if (!(e > 0.f) || !isfinite(e)) return 1.f;
  return 1.f / sqrtf(e);
}

__global__ void __launch_bounds__(256) k_chan_scale(LaunchCtx c, const int* __restrict__ procs, int which) {
  __shared__ float red[4 * 32];
  const ProcDev& P = c.procs[procs[blockIdx.x]];
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  const float* x = which == 0 ? P.u : P.dy;
  // self-check of the operands: a missing or misaligned signal, a row stride shorter than the signal, or missing
  // taps skip the node (its scales stay as they were) and are reported
  if (x == nullptr || ((uintptr_t)x & 15) != 0 || P.ld < P.L || (P.ld & 3) != 0 || P.stats == nullptr ||
      (which == 0 && P.taps == nullptr) || (which == 0 && P.type == T_D && P.aux == nullptr)) {
    if (threadIdx.x == 0)
      printf("k_chan_scale: node %d which %d skipped (x %p, L %d, ld %d, taps %p, stats %p)\n", procs[blockIdx.x], which,
             (const void*)x, P.L, P.ld, (const void*)P.taps, (const void*)P.stats);
    return;
  }
  const int nq = P.L >> 2;                    // whole quads of samples
  for (int q = threadIdx.x * 32; q < nq; q += blockDim.x * 32) {   // every 32nd quad
    const float4 a = reinterpret_cast<const float4*>(x)[q];
    const float4 b = reinterpret_cast<const float4*>(x + P.ld)[q];
    acc[0] += a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w;
    acc[1] += b.x * b.x + b.y * b.y + b.z * b.z + b.w * b.w;
  }
  if (which == 0 && P.type == T_D) {
    for (int j = threadIdx.x; j < kDlyTaps * kDlyFir; j += blockDim.x) {   // c_m of both channels
      const float a = P.aux[j], b = P.aux[kDlyTaps * kDlyFir + j];
      acc[2] += a * a;
      acc[3] += b * b;
    }
  } else if (which == 0)
    for (int j = threadIdx.x * 32; j < P.Nh; j += blockDim.x * 32) {   // every 32nd tap
      const float2 t = tap_at(P, (int64_t)j + P.n0 >= 0 ? (int64_t)j + P.n0 : fft_len(P) + j + P.n0, fft_len(P));
      acc[2] += t.x * t.x;
      acc[3] += t.y * t.y;
    }
  float out[4];
  block_sum<4>(acc, red, out);
  if (threadIdx.x == 0) {
    if (which == 0) {
      P.stats[kScaleU] = unit_scale(out[0]);
      P.stats[kScaleU + 1] = unit_scale(out[1]);
      P.stats[kScaleH] = unit_scale(out[2]);
      P.stats[kScaleH + 1] = unit_scale(out[3]);
    } else {
      P.stats[kScaleD] = unit_scale(out[0]);
      P.stats[kScaleD + 1] = unit_scale(out[1]);
    }
  }
}

template <int MODE>
void launch_col(const LaunchCtx& c, const Item* items, int n, int maxN2G) {
  if (!n) return;
  (void)maxN2G;
  const size_t smem = (size_t)kColBuf * sizeof(float2);
  k_col<MODE><<<n, kColThreads, smem, c.stream>>>(c, items);
}

}  // namespace

void init_col_attributes() {
  const int big = kColBuf * (int)sizeof(float2);
  cudaFuncSetAttribute(k_col<COL_FWD_AUDIO>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_col<COL_FWD_TAPS>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_col<COL_INV_OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_col<COL_DYBAR>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_col<COL_DU>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_col<COL_DH>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_col<COL_INV_OUT_KEEP>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_col<COL_DYBAR_KEEP>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

void launch_chan_scale(const LaunchCtx& c, const int* procs, int n, int which) {
  if (n) k_chan_scale<<<n, 256, 0, c.stream>>>(c, procs, which);
}
void launch_col_fwd_audio(const LaunchCtx& c, const Item* items, int n, int m) { launch_col<COL_FWD_AUDIO>(c, items, n, m); }
void launch_col_fwd_taps(const LaunchCtx& c, const Item* items, int n, int m) { launch_col<COL_FWD_TAPS>(c, items, n, m); }
void launch_col_inv_out(const LaunchCtx& c, const Item* items, int n, int m) { launch_col<COL_INV_OUT>(c, items, n, m); }
void launch_col_dybar(const LaunchCtx& c, const Item* items, int n, int m) { launch_col<COL_DYBAR>(c, items, n, m); }
void launch_col_du(const LaunchCtx& c, const Item* items, int n, int m) { launch_col<COL_DU>(c, items, n, m); }
void launch_col_dh(const LaunchCtx& c, const Item* items, int n, int m) { launch_col<COL_DH>(c, items, n, m); }
void launch_col_inv_out_keep(const LaunchCtx& c, const Item* items, int n, int m) { launch_col<COL_INV_OUT_KEEP>(c, items, n, m); }
void launch_col_dybar_keep(const LaunchCtx& c, const Item* items, int n, int m) { launch_col<COL_DYBAR_KEEP>(c, items, n, m); }

}  // namespace mg

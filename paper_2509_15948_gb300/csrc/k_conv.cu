// FIR convolution of the LTI processors (reverb Sec. 3.4, multitap delay Eq. 17; the equalizer of Eq. 8 in the
// allocation-free entry) and its adjoint, by one zero-padded FFT of size N = N1 * N2 >= L + |taps| per node
// (exact linear convolution), N = f 2^k with f in {1, 3} (whichever is smaller: the odd factor cuts the
// average padding from ~1.5x to ~1.2x), N1 = f 2^a rows, N2 = 2^b columns, evaluated with the four-step
// algorithm in two shared-memory passes:
//   column pass: N2-point FFTs over n2 of x[n1 + N1 n2] for a group of G adjacent n1, twiddle
//                exp(-+2 pi i n1 k2 / N); stored in place, so row k2 holds A[n1][k2] contiguously;
//   row pass:    N1-point FFTs of row k2 give X[k2 + N2 k1] at row k2, position k1 (transposed order).
// A convolution never needs natural order: the row pass multiplies the transposed spectra and runs the
// inverse row FFT immediately, the inverse column pass returns to natural time order.
// Both channels travel as one complex signal z = left + i right; a stereo FIR (h_l, h_r) acts on the packed
// spectrum as Y[k] = Z[k] A[k] + conj(Z[-k]) B[k] with A = (H_l + H_r)/2, B = (H_l - H_r)/2, where the
// mirror bin -k sits in row N2 - k2.
#include <algorithm>

#include "mg_fftp.cuh"

namespace mg {

namespace {

constexpr int kColThreads = 512;
constexpr int kRowThreads = 512;   // largest row block: N1 = 3072 (one thread per 8 elements of a row pair)
// Shared-memory layouts (padded, see mg_fftp.cuh).  Column pass: column g, row r at sm[g * col_stride + pidx(r)],
// with col_stride = 16 (mod 16) + 16 / G so that the G columns and 16 / G rows a half-warp touches fall in
// distinct bank pairs.  Row pass: row slot s, position k1 at sm[s * pstride(N1) + pidx(k1)].
constexpr int kColBuf = 8192 + 512 + 160;
constexpr int kMaxRow = 3072;      // longest row N1 (3 x 1024)
__host__ __device__ constexpr int col_stride(int N2, int G) { return ((N2 + (N2 >> 4) + 15) & ~15) + 16 / G; }

__device__ __forceinline__ int mirror_pos(int k2, int k1, int N1) { return k2 == 0 ? (k1 ? N1 - k1 : 0) : (N1 - 1 - k1); }

__device__ __forceinline__ int rows_len(const ProcDev& P) { return P.f << P.logN1; }
__device__ __forceinline__ int64_t fft_len(const ProcDev& P) { return (int64_t)P.f << P.logN; }

// Transposition twiddle exp(-+2 pi i m / N), m < N: the power-of-two tables, times exp(-2 pi i (m mod 3) / N)
// when N = 3 2^logN.
__device__ __forceinline__ float2 twiddle_node(const ProcDev& P, unsigned m, bool inverse, const Tables& tab) {
  if (P.f == 1) return twiddle_tab(m, P.logN, inverse, tab);
  const unsigned q = m / 3u, r = m - 3u * q;
  float2 w = twiddle_tab(q, P.logN, false, tab);
  if (r) w = cmul(w, P.c3n[r]);
  if (inverse) w.y = -w.y;
  return w;
}

// Row FFTs (length N1 = f 2^logN1) of nb padded rows with batch stride bs.
template <bool INV>
__device__ __forceinline__ void row_fft(float2* d, const ProcDev& P, int nb, int bs, const Tables& tab) {
  if (P.f == 1) fft_p<INV>(d, P.logN1, nb, bs, tab.ptw);
  else fft_p3<INV>(d, P.logN1, nb, bs, tab.ptw3);
}

// Tap value of the stereo FIR at circular position n (time n, or n - N for the negative taps).
__device__ __forceinline__ float2 tap_at(const ProcDev& P, int64_t n, int64_t N) {
  int64_t j;
  if (n < (int64_t)P.n0 + P.Nh) j = n - P.n0;
  else if (n >= N + P.n0) j = n - N - P.n0;
  else return make_float2(0.f, 0.f);
  if (j < 0 || j >= P.Nh) return make_float2(0.f, 0.f);
  const float a = P.taps[j];
  if (P.type == T_E) return make_float2(a, a);
  const float b = P.taps[P.Nh + j];
  if (P.type == T_R) return make_float2(a + b, a - b);   // h_l = h_m + h_s, h_r = h_m - h_s
  return make_float2(a, b);
}

// Packed-stereo FIR spectra at a bin and its mirror: A = (H_l + H_r)/2, B = (H_l - H_r)/2.
__device__ __forceinline__ void fir_ab(float2 hz, float2 hzm, float2& A, float2& B) {
  const float2 hl = cscale(cadd(hz, cconj(hzm)), 0.5f);
  const float2 d = csub(hz, cconj(hzm));
  const float2 hr = make_float2(0.5f * d.y, -0.5f * d.x);     // d / (2i)
  A = cscale(cadd(hl, hr), 0.5f);
  B = cscale(csub(hl, hr), 0.5f);
}

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

template <int MODE>
__global__ void __launch_bounds__(kColThreads, 2) k_col(LaunchCtx c, const Item* __restrict__ items) {
  extern __shared__ float2 sm[];
  __shared__ float red[2 * 32];
  __shared__ float2 tws[kSlots * 8];   // W(n1 RS s) of the block's columns, [s][g]
  const Item it = items[blockIdx.x];
  const ProcDev& P = c.procs[it.proc];
  const int G = P.colG, logG = __ffs(G) - 1;
  const int logN2 = P.logN2, N2 = 1 << logN2, N1 = rows_len(P);
  const int64_t N = fft_len(P);
  const int cs = col_stride(N2, G);
  constexpr bool kInv = MODE == COL_INV_OUT || MODE == COL_DYBAR || MODE == COL_DU || MODE == COL_DH ||
                        MODE == COL_INV_OUT_KEEP;
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

  // Forward passes end with the transposition twiddle W(n1 k2), W = exp(-2 pi i / N); for k2 = r0 + s RS it
  // is W(n1 r0) W(n1 RS s): the first factor is the thread's own, the second comes from a per-block table.
  constexpr bool kTwid = !(MODE == COL_INV_OUT || MODE == COL_DU || MODE == COL_DH || MODE == COL_INV_OUT_KEEP);
  float2 w_r0 = make_float2(1.f, 0.f);
  if (kTwid) {
    if (r0 < N2) w_r0 = twiddle_node(P, (unsigned)n1 * (unsigned)r0, false, c.tab);
    if ((int)threadIdx.x < kSlots * G) {   // visible after the barriers of the load and the FFT
      const int ts = threadIdx.x >> logG, tg = threadIdx.x & (G - 1);
      const unsigned step = (unsigned)(RS * ts);
      tws[threadIdx.x] = step < (unsigned)N2 ? twiddle_node(P, (unsigned)(it.idx * G + tg) * step, false, c.tab)
                                              : make_float2(1.f, 0.f);
    }
  }
  auto tw_at = [&](int s) { return cmul(w_r0, tws[s * G + g]); };

  // ---- load ----
  if (MODE != COL_DYBAR_KEEP) {
    const float2* src = (MODE == COL_INV_OUT || MODE == COL_DH) ? P.T1 : P.T2;
#pragma unroll
    for (int h = 0; h < kSlots; h += 8) {
      float2 v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        v[j] = make_float2(0.f, 0.f);
        if (live(h + j)) {
          const int64_t n = pos(h + j);
          if (MODE == COL_FWD_AUDIO) {
            if (n < P.L) v[j] = make_float2(P.u[n], P.u[P.ld + n]);
          } else if (MODE == COL_FWD_TAPS) {
            v[j] = tap_at(P, n, N);
          } else {
            v[j] = src[n];
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (live(h + j)) col[pidx(row_of(h + j))] = v[j];
    }
    __syncthreads();
    fft_p<kInv>(sm, logN2, G, cs, c.tab.ptw);
  }

  if (!kInv && !kDybar) {  // forward column pass: twiddle, store in place (row k2)
    float2* dst = MODE == COL_FWD_TAPS ? P.Hz : P.T1;
#pragma unroll 4
    for (int s = 0; s < kSlots; ++s) {
      if (!live(s)) continue;
      dst[pos(s)] = cmul(col[pidx(row_of(s))], tw_at(s));
    }
    return;
  }

  const float inv_n = ldexpf(1.f, -P.logN) / (float)P.f;
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
        const float2 yb = cscale(col[pidx(row_of(h + j))], inv_n);
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
          yb[j] = MODE == COL_DYBAR_KEEP ? P.T2[n] : cscale(col[pidx(row_of(h + j))], inv_n);
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
        col[pidx(row_of(h + j))] = make_float2(w * gl[j] + gm, w * gr[j] + gm);
      }
    }
    float out[1];
    block_sum<1>(acc, red, out);   // also acts as the barrier before the FFT
    if (threadIdx.x == 0) P.bpart[it.idx * kNPart + 0] = out[0];
    fft_p<false>(sm, logN2, G, cs, c.tab.ptw);
#pragma unroll 4
    for (int s = 0; s < kSlots; ++s) {
      if (!live(s)) continue;
      P.T2[pos(s)] = cmul(col[pidx(row_of(s))], tw_at(s));
    }
    return;
  }
  if (MODE == COL_DU) {
    const float wd = dry_wet_d(c, P.qidx);
    const float c2 = P.stats[3];
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
        const float2 dw = cscale(col[pidx(row_of(h + j))], inv_n);
        P.du[n] = wd * gl[j] + dw.x + um[j];
        P.du[P.ld + n] = wd * gr[j] + dw.y + um[j];
      }
    }
    return;
  }
  if (MODE == COL_DH) {
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
        const float2 v = (j + P.n0 >= P.L) ? make_float2(0.f, 0.f) : cscale(col[pidx(row_of(s))], inv_n);
        P.dtaps[j] = v.x;
        P.dtaps[P.Nh + j] = v.y;
      }
    }
  }
}

// Row pass of the filter spectrum: forward N1-point FFTs of rows a and b = N2 - a of Hz, in place.
__global__ void __launch_bounds__(kRowThreads, 2) k_row_fwd_hz(LaunchCtx c, const Item* __restrict__ items) {
  extern __shared__ float2 sm[];
  const Item it = items[blockIdx.x];
  const ProcDev& P = c.procs[it.proc];
  const int N1 = rows_len(P), N2 = 1 << P.logN2, rs = pstride(N1);
  const int a = it.idx, b = (N2 - it.idx) & (N2 - 1);
  const int nr = a == b ? 1 : 2;
  for (int e = threadIdx.x; e < nr * N1; e += blockDim.x) {
    const int slot = e >= N1, k1 = e - slot * N1;
    sm[slot * rs + pidx(k1)] = P.Hz[(int64_t)(slot ? b : a) * N1 + k1];
  }
  __syncthreads();
  row_fft<false>(sm, P, nr, rs, c.tab);
  for (int e = threadIdx.x; e < nr * N1; e += blockDim.x) {
    const int slot = e >= N1, k1 = e - slot * N1;
    P.Hz[(int64_t)(slot ? b : a) * N1 + k1] = sm[slot * rs + pidx(k1)];
  }
}

// Loads rows a and b (b may equal a) of src into smem slots 0/1 and runs their forward FFTs.
__device__ __forceinline__ void load_rows_fft(float2* s, const float2* src, int a, int b, const ProcDev& P,
                                              const Tables& tab) {
  const int N1 = rows_len(P), rs = pstride(N1);
  const int nr = a == b ? 1 : 2;
#pragma unroll 8
  for (int e = threadIdx.x; e < nr * N1; e += blockDim.x) {
    const int slot = e >= N1, k1 = e - slot * N1;
    s[slot * rs + pidx(k1)] = src[(int64_t)(slot ? b : a) * N1 + k1];
  }
  __syncthreads();
  row_fft<false>(s, P, nr, rs, tab);
}

// Transposition twiddles of rows a and b, W(n1 k2) = lo[n1 mod T] hi[n1 / T] (W = exp(-2 pi i / N), T = 64 or
// the largest power of two dividing N1 when smaller, N1 / T <= 48), both factors from the accurate table:
// per row slot kRowTwT lo entries, then the hi entries.  Visible after the caller's next barrier.
constexpr int kRowTwT = 64, kRowTwS = 128;
__device__ __forceinline__ void row_tw_init(float2* tt, const ProcDev& P, int a, int b, const Tables& tab) {
  const int N1 = rows_len(P), logT = min(6, __ffs(N1) - 1), T = 1 << logT, H = N1 >> logT;
  for (int e = threadIdx.x; e < 2 * (T + H); e += blockDim.x) {
    const int slot = e >= T + H, j = e - slot * (T + H);
    const unsigned k2 = slot ? b : a;
    const unsigned m = j < T ? (unsigned)j * k2 : (unsigned)((j - T) << logT) * k2;
    tt[slot * kRowTwS + (j < T ? j : kRowTwT + j - T)] = twiddle_node(P, m, false, tab);
  }
}

// Inverse row FFT of the slots in o, twiddle exp(+2 pi i n1 k2 / N) (the conjugate of the tt entries), store
// rows a, b of dst.
__device__ __forceinline__ void inv_rows_store(float2* o, float2* dst, int a, int b, const ProcDev& P,
                                               const Tables& tab, const float2* tt) {
  const int N1 = rows_len(P), rs = pstride(N1), logT = min(6, __ffs(N1) - 1);
  const int nr = a == b ? 1 : 2;
  __syncthreads();
  row_fft<true>(o, P, nr, rs, tab);
#pragma unroll 4
  for (int e = threadIdx.x; e < nr * N1; e += blockDim.x) {
    const int slot = e >= N1, n1 = e - slot * N1;
    const int k2 = slot ? b : a;
    const float2* t = tt + slot * kRowTwS;
    const float2 w = cmul(t[n1 & ((1 << logT) - 1)], t[kRowTwT + (n1 >> logT)]);
    dst[(int64_t)k2 * N1 + n1] = cmul(o[slot * rs + pidx(n1)], cconj(w));
  }
}

// Every bin of rows a, b = N2 - a together with its mirror -k, once per pair: for a != b the partner of
// (a, k1) is (b, N1 - 1 - k1); for a == b (rows 0 and N2/2) both bins lie in the same row and a pair is
// visited from its smaller position (bins 0 and N1/2 of row 0 are their own mirrors).  The pairs of a thread
// are taken NB at a time: load(gP, gQ) fetches the global operands of all NB pairs first (independent loads in
// flight together), then op(pP, pQ, gP, gQ, v) runs on each; pP, pQ are the shared-memory positions (slot
// layout of load_rows_fft), gP, gQ the positions in the row-major grid.
template <int NB, typename Ld, typename Op>
__device__ __forceinline__ void for_mirror_pairs(int a, int b, int N1, Ld&& load, Op&& op) {
  const int qs = a == b ? 0 : pstride(N1);
  using V = decltype(load(int64_t(0), int64_t(0)));
  for (int k0 = threadIdx.x; k0 < N1; k0 += NB * blockDim.x) {
    V v[NB];
    int kk[NB], mk[NB];
    bool ok[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      kk[j] = k0 + j * blockDim.x;
      mk[j] = mirror_pos(a, kk[j], N1);
      ok[j] = kk[j] < N1 && !(a == b && mk[j] < kk[j]);
      if (ok[j]) v[j] = load((int64_t)a * N1 + kk[j], (int64_t)b * N1 + mk[j]);
    }
#pragma unroll
    for (int j = 0; j < NB; ++j)
      if (ok[j]) op(pidx(kk[j]), qs + pidx(mk[j]), (int64_t)a * N1 + kk[j], (int64_t)b * N1 + mk[j], v[j]);
  }
}

struct HzPair {
  float2 hP, hQ;
};
struct HzUPair {
  float2 hP, hQ, uP, uQ;
};

// Forward convolution: spectrum Z of u (rows of T1 after the column pass), Y = Z A + conj(Z_-) B, inverse row
// FFT.  KEEP = false: the result goes back to T1.  KEEP = true (retained spectra, and the recomputing
// backward): T1 keeps Z for the FIR gradient and the result goes to T2.  The product is formed in place,
// each thread owning a bin and its mirror.
template <bool KEEP>
__global__ void __launch_bounds__(kRowThreads, 2) k_row_conv(LaunchCtx c, const Item* __restrict__ items) {
  extern __shared__ float2 sm[];
  const Item it = items[blockIdx.x];
  const ProcDev& P = c.procs[it.proc];
  const int N1 = rows_len(P), N2 = 1 << P.logN2;
  const int a = it.idx, b = (N2 - it.idx) & (N2 - 1);
  __shared__ float2 tt[2 * kRowTwS];
  row_tw_init(tt, P, a, b, c.tab);
  float2* s = sm;
  load_rows_fft(s, P.T1, a, b, P, c.tab);
  for_mirror_pairs<4>(a, b, N1, [&](int64_t gP, int64_t gQ) { return HzPair{P.Hz[gP], P.Hz[gQ]}; },
                      [&](int pP, int pQ, int64_t gP, int64_t gQ, const HzPair& v) {
    const float2 zP = s[pP], zQ = s[pQ];
    float2 AP, BP, AQ, BQ;
    fir_ab(v.hP, v.hQ, AP, BP);
    fir_ab(v.hQ, v.hP, AQ, BQ);
    if (KEEP) {
      P.T1[gP] = zP;
      P.T1[gQ] = zQ;
    }
    s[pP] = cadd(cmul(zP, AP), cmul(cconj(zQ), BP));
    s[pQ] = cadd(cmul(zQ, AQ), cmul(cconj(zP), BQ));
  });
  inv_rows_store(s, KEEP ? P.T2 : P.T1, a, b, P, c.tab, tt);
}

// Second backward step.  Rows of T2 hold the column-transformed dL/dy_bar; T1 holds the spectrum of u.
//   dU  = Dz conj(A) + conj(Dz_-) conj(B)                    (correlation with the FIR: adjoint of y = h * u)
//   dH  = D_l conj(U_l) + i D_r conj(U_r)                      (dL/dh_c[j] = sum_n dL/dy_bar_c[n] u_c[n - j])
// dU is formed in place over the spectrum of dL/dy_bar; dH goes to global memory over the input spectrum in
// T1 (each grid position belongs to one pair of one thread, which has read its U there before), so the block
// holds two rows of shared memory instead of four.  Inverse row FFTs: dU to T2, then dH (reloaded from T1,
// still in L2) to T1.
__device__ __forceinline__ float2 fir_grad_bin(float2 dz, float2 dzm, float2 zu, float2 zum) {
  const float2 ul = cscale(cadd(zu, cconj(zum)), 0.5f);
  const float2 du_ = csub(zu, cconj(zum));
  const float2 ur = make_float2(0.5f * du_.y, -0.5f * du_.x);
  const float2 dl = cscale(cadd(dz, cconj(dzm)), 0.5f);
  const float2 dd = csub(dz, cconj(dzm));
  const float2 dr = make_float2(0.5f * dd.y, -0.5f * dd.x);
  const float2 hl = cmulc(dl, ul), hr = cmulc(dr, ur);
  return make_float2(hl.x - hr.y, hl.y + hr.x);   // hl + i hr
}

__global__ void __launch_bounds__(kRowThreads, 2) k_row_bwd2(LaunchCtx c, const Item* __restrict__ items) {
  extern __shared__ float2 sm[];
  const Item it = items[blockIdx.x];
  const ProcDev& P = c.procs[it.proc];
  const int N1 = rows_len(P), N2 = 1 << P.logN2;
  const int a = it.idx, b = (N2 - it.idx) & (N2 - 1);
  float2* s = sm;
  __shared__ float2 tt[2 * kRowTwS];
  row_tw_init(tt, P, a, b, c.tab);
  load_rows_fft(s, P.T2, a, b, P, c.tab);
  for_mirror_pairs<4>(a, b, N1,
                      [&](int64_t gP, int64_t gQ) { return HzUPair{P.Hz[gP], P.Hz[gQ], P.T1[gP], P.T1[gQ]}; },
                      [&](int pP, int pQ, int64_t gP, int64_t gQ, const HzUPair& v) {
    const float2 dzP = s[pP], dzQ = s[pQ];
    float2 AP, BP, AQ, BQ;
    fir_ab(v.hP, v.hQ, AP, BP);
    fir_ab(v.hQ, v.hP, AQ, BQ);
    s[pP] = cadd(cmul(dzP, cconj(AP)), cmul(cconj(dzQ), cconj(BP)));
    s[pQ] = cadd(cmul(dzQ, cconj(AQ)), cmul(cconj(dzP), cconj(BQ)));
    P.T1[gP] = fir_grad_bin(dzP, dzQ, v.uP, v.uQ);
    P.T1[gQ] = fir_grad_bin(dzQ, dzP, v.uQ, v.uP);
  });
  inv_rows_store(s, P.T2, a, b, P, c.tab, tt);
  __syncthreads();   // the dH rows written to T1 are visible to the whole block, and s is free again
  const int nr = a == b ? 1 : 2, rs = pstride(N1);
#pragma unroll 8
  for (int e = threadIdx.x; e < nr * N1; e += blockDim.x) {
    const int slot = e >= N1, k1 = e - slot * N1;
    s[slot * rs + pidx(k1)] = P.T1[(int64_t)(slot ? b : a) * N1 + k1];
  }
  inv_rows_store(s, P.T1, a, b, P, c.tab, tt);
}

template <int MODE>
void launch_col(const LaunchCtx& c, const Item* items, int n, int maxN2G) {
  if (!n) return;
  (void)maxN2G;
  const size_t smem = (size_t)kColBuf * sizeof(float2);
  k_col<MODE><<<n, kColThreads, smem, c.stream>>>(c, items);
}

}  // namespace

void init_kernel_attributes() {
  const int big = kColBuf * (int)sizeof(float2);
  cudaFuncSetAttribute(k_col<COL_FWD_AUDIO>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_col<COL_FWD_TAPS>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_col<COL_INV_OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_col<COL_DYBAR>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_col<COL_DU>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_col<COL_DH>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_col<COL_INV_OUT_KEEP>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_col<COL_DYBAR_KEEP>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_row_fwd_hz, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * pstride(kMaxRow) * (int)sizeof(float2));
  cudaFuncSetAttribute(k_row_conv<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * pstride(kMaxRow) * (int)sizeof(float2));
  cudaFuncSetAttribute(k_row_conv<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * pstride(kMaxRow) * (int)sizeof(float2));
  cudaFuncSetAttribute(k_row_bwd2, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * pstride(kMaxRow) * (int)sizeof(float2));
}

void launch_col_fwd_audio(const LaunchCtx& c, const Item* items, int n, int m) { launch_col<COL_FWD_AUDIO>(c, items, n, m); }
void launch_col_fwd_taps(const LaunchCtx& c, const Item* items, int n, int m) { launch_col<COL_FWD_TAPS>(c, items, n, m); }
void launch_col_inv_out(const LaunchCtx& c, const Item* items, int n, int m) { launch_col<COL_INV_OUT>(c, items, n, m); }
void launch_col_dybar(const LaunchCtx& c, const Item* items, int n, int m) { launch_col<COL_DYBAR>(c, items, n, m); }
void launch_col_du(const LaunchCtx& c, const Item* items, int n, int m) { launch_col<COL_DU>(c, items, n, m); }
void launch_col_dh(const LaunchCtx& c, const Item* items, int n, int m) { launch_col<COL_DH>(c, items, n, m); }
void launch_col_inv_out_keep(const LaunchCtx& c, const Item* items, int n, int m) { launch_col<COL_INV_OUT_KEEP>(c, items, n, m); }
void launch_col_dybar_keep(const LaunchCtx& c, const Item* items, int n, int m) { launch_col<COL_DYBAR_KEEP>(c, items, n, m); }

// Row kernels run one thread per 8 elements of a row pair (2 N1 elements, fft_p's limit of 16 per thread with
// radix-16 passes keeping every thread busy), so the block size follows the largest N1 of the launch.
int row_threads(int maxN1) { return std::max(32, std::min(kRowThreads, maxN1 / 8)); }

void launch_row_fwd_hz(const LaunchCtx& c, const Item* items, int n, int maxN1) {
  if (n) k_row_fwd_hz<<<n, row_threads(maxN1), (size_t)2 * pstride(maxN1) * sizeof(float2), c.stream>>>(c, items);
}

void launch_row_conv_fwd(const LaunchCtx& c, const Item* items, int n, int maxN1, bool keep) {
  if (!n) return;
  const size_t smem = (size_t)2 * pstride(maxN1) * sizeof(float2);
  if (keep) k_row_conv<true><<<n, row_threads(maxN1), smem, c.stream>>>(c, items);
  else k_row_conv<false><<<n, row_threads(maxN1), smem, c.stream>>>(c, items);
}

void launch_row_bwd2(const LaunchCtx& c, const Item* items, int n, int maxN1) {
  if (!n) return;
  const size_t smem = (size_t)2 * pstride(maxN1) * sizeof(float2);
  k_row_bwd2<<<n, row_threads(maxN1), smem, c.stream>>>(c, items);
}

}  // namespace mg

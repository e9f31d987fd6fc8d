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
// mirror bin -k sits in row N2 - k2.  The rounding error of a packed transform scales with the larger channel,
// so before packing every channel of u, of the taps and of dL/dy_bar is multiplied by a scale that brings the
// channels to a common level (k_chan_scale); the products are bilinear per channel, and the output passes
// divide by the product of the scales involved (two roundings, far below the transforms' own).
#pragma once
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

// Transposition twiddle exp(-+2 pi i m / N), m < N: the power-of-two tables, times exp(-2 pi i (m mod f) / N)
// when N = f 2^logN, f = 3 or 5.
__device__ __forceinline__ float2 twiddle_node(const ProcDev& P, unsigned m, bool inverse, const Tables& tab) {
  if (P.f == 1) return twiddle_tab(m, P.logN, inverse, tab);
  const unsigned q = m / (unsigned)P.f, r = m - (unsigned)P.f * q;
  float2 w = twiddle_tab(q, P.logN, false, tab);
  if (r) w = cmul(w, P.cfn[r]);
  if (inverse) w.y = -w.y;
  return w;
}

// Row FFTs (length N1 = f 2^logN1) of nb padded rows with batch stride bs; inputs through ld(slot, k1) and
// outputs through st(slot, k1, v) when those are functors (see fft_p_io).
template <bool INV, class LD = fftp::SmemIO, class ST = fftp::SmemIO>
__device__ __forceinline__ void row_fft(float2* d, const ProcDev& P, int nb, int bs, const Tables& tab, LD ld = LD(),
                                        ST st = ST()) {
  if (P.f == 1) fft_p_io<INV, 1>(d, P.logN1, nb, bs, tab.ptw, ld, st);
  else if (P.f == 3) fft_pf_io<INV, 3>(d, P.logN1, nb, bs, tab.ptw3, ld, st);
  else fft_pf_io<INV, 5>(d, P.logN1, nb, bs, tab.ptw5, ld, st);
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

// Channel scales of a packed transform (left, right), set by k_chan_scale; 1 before it ran.
__device__ __forceinline__ float2 chan_scale(const ProcDev& P, int slot) {
  const float a = P.stats[slot], b = P.stats[slot + 1];
  return make_float2(a > 0.f ? a : 1.f, b > 0.f ? b : 1.f);
}

// Packed-stereo FIR spectra at a bin and its mirror: A = (H_l + H_r)/2, B = (H_l - H_r)/2.
__device__ __forceinline__ void fir_ab(float2 hz, float2 hzm, float2& A, float2& B) {
  const float2 hl = cscale(cadd(hz, cconj(hzm)), 0.5f);
  const float2 d = csub(hz, cconj(hzm));
  const float2 hr = make_float2(0.5f * d.y, -0.5f * d.x);     // d / (2i)
  A = cscale(cadd(hl, hr), 0.5f);
  B = cscale(csub(hl, hr), 0.5f);
}

// Forward FFTs of rows a and b (b may equal a) of src into smem slots 0/1; the first pass reads the rows from
// global memory directly.  The buffer must be free when the call starts.
__device__ __forceinline__ void load_rows_fft(float2* s, const float2* src, int a, int b, const ProcDev& P,
                                              const Tables& tab) {
  const int N1 = rows_len(P), rs = pstride(N1);
  const int nr = a == b ? 1 : 2;
  const float2* ra = src + (int64_t)a * N1;
  const float2* rb = src + (int64_t)b * N1;
  row_fft<false>(s, P, nr, rs, tab, [=](int slot, int k1) { return (slot ? rb : ra)[k1]; });
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

// Inverse row FFT of the slots in o (or, with ld a functor, of rows read through it), twiddle
// exp(+2 pi i n1 k2 / N) (the conjugate of the tt entries), rows a, b stored to dst by the last pass.  Opens with
// a barrier and ends without one.
template <class LD = fftp::SmemIO>
__device__ __forceinline__ void inv_rows_store(float2* o, float2* dst, int a, int b, const ProcDev& P,
                                               const Tables& tab, const float2* tt, LD ld = LD()) {
  const int N1 = rows_len(P), rs = pstride(N1), logT = min(6, __ffs(N1) - 1);
  const int nr = a == b ? 1 : 2;
  float2* da = dst + (int64_t)a * N1;
  float2* db = dst + (int64_t)b * N1;
  __syncthreads();
  row_fft<true>(o, P, nr, rs, tab, ld, [=](int slot, int n1, float2 v) {
    const float2* t = tt + slot * kRowTwS;
    const float2 w = cmul(t[n1 & ((1 << logT) - 1)], t[kRowTwT + (n1 >> logT)]);
    (slot ? db : da)[n1] = cmul(v, cconj(w));
  });
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

// Row kernels run one thread per 8 elements of a row pair (2 N1 elements, fft_p's limit of 16 per thread with
// radix-16 passes keeping every thread busy), so the block size follows the largest N1 of the launch.
inline int row_threads(int maxN1) { return std::max(32, std::min(kRowThreads, maxN1 / 8)); }

}  // namespace

}  // namespace mg

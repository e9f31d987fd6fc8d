// Shared-memory Stockham FFT, radix 16 (plus one radix-8/4/2 pass for the remaining factor), on a padded
// layout: element e of a transform sits at offset pidx(e) = e + e/16 inside its batch, which makes the
// strided stores of every pass free of bank conflicts.  Used by the hot convolution and loss kernels.
//
// Stockham pass of radix R with p = product of the previous radices: butterfly i (k = i mod p) reads
// x[i + r M/R], multiplies by w_{Rp}^{r k}, runs an R-point DFT in registers and writes the R results to
// (i - k) R + k + q p.  The powers w^1, w^2, w^4, w^8 of a butterfly come from a pass twiddle table laid out
// per pass as rows of p consecutive k, so that the loads of a warp (consecutive k) are coalesced; the other
// powers are products.
#pragma once
#include <type_traits>

#include "mg_fft.cuh"

namespace mg {

__device__ __forceinline__ int pidx(int e) { return e + (e >> 4); }
// batch stride of a padded transform of size M (odd, to spread consecutive batches over the banks)
__host__ __device__ constexpr int pstride(int M) { return M + (M >> 4) + 1; }

// Pass twiddle table of the power-of-two transforms (M <= 8192).  The pass with p = 2^lp (lp = 4, 8, 12) and
// radix R = 2^logr owns logr rows of p entries; row j, entry k is w^(2^j k), w = exp(-2 pi i / (R p)), which is
// entry (2^j k) 2^(13 - lp - logr) of the 8192-point table exp(-2 pi i j / 8192).
constexpr int kPtwCount = 6816;
__host__ __device__ constexpr int ptw_base(int lp, int logr) {
  return (lp == 4 ? 0 : (lp == 8 ? 160 : 2720)) + (1 << lp) * (logr * (logr - 1) / 2);
}
// index into the 8192-point table of entry e of the pass twiddle table
__host__ __device__ inline int ptw_source(int e) {
  int lp = 4, start = 0;
  if (e >= 2720) { lp = 12; start = 2720; }
  else if (e >= 160) { lp = 8; start = 160; }
  const int p = 1 << lp, row = (e - start) / p, k = (e - start) % p;
  const int logr = row < 1 ? 1 : (row < 3 ? 2 : (row < 6 ? 3 : 4));
  const int j = row - logr * (logr - 1) / 2;
  return ((1 << j) * k) << (13 - lp - logr);
}

// Pass twiddle tables of the transforms of size M = F 2^a, F = 3 (1 <= a <= kPtw3MaxA) or F = 5
// (1 <= a <= kPtw5MaxA).  Region a starts at 4F (2^a - 2); in it, the twiddled pass number j (p = F 16^j,
// radix 16 except the last) starts at 4F (16^j - 1) / 15 and owns logr rows of p entries: row r, entry k is
// exp(-2 pi i m / M), m = (2^r k) 2^(a - 4 j - logr).
constexpr int kPtw3MaxA = 10;
constexpr int kPtw3Count = 12 * ((2 << kPtw3MaxA) - 2);
constexpr int kPtw5MaxA = 9;
constexpr int kPtw5Count = 20 * ((2 << kPtw5MaxA) - 2);
__host__ __device__ constexpr int ptwf_base(int f, int a, int lp2) {
  return 4 * f * ((1 << a) - 2) + 4 * f * (((1 << lp2) - 1) / 15);
}
__host__ __device__ constexpr int ptw3_base(int a, int lp2) { return ptwf_base(3, a, lp2); }

namespace fftp {

// Where a pass takes its inputs or puts its outputs: SmemIO is the shared buffer itself; any other type is a
// functor, ld(batch, element) -> float2 for the first pass of a transform and st(batch, element, value) for the
// last, so a transform can read from and write to global memory directly (the element is the natural input
// position, resp. the natural output bin).
struct SmemIO {};
template <class T>
constexpr bool is_io = !std::is_same<T, SmemIO>::value;

template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {  // a * (-i) forward, a * (+i) inverse
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <bool INV>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  const float2 t = csub(a, b);
  a = cadd(a, b);
  b = t;
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
  const float2 b0 = cadd(x0, x2), b1 = csub(x0, x2), b2 = cadd(x1, x3), b3 = mul_mi<INV>(csub(x1, x3));
  x0 = cadd(b0, b2);
  x2 = csub(b0, b2);
  x1 = cadd(b1, b3);
  x3 = csub(b1, b3);
}

__device__ __forceinline__ float2 w16(int m, bool inv) {
  // exp(-+2 pi i m / 16) for the products n2 k1 of the 4 x 4 decomposition
  constexpr float c8 = 0.92387953251128674f, s8 = 0.38268343236508978f, r2 = 0.70710678118654752f;
  float2 w;
  switch (m) {
    case 1: w = make_float2(c8, -s8); break;
    case 2: w = make_float2(r2, -r2); break;
    case 3: w = make_float2(s8, -c8); break;
    case 4: w = make_float2(0.f, -1.f); break;
    case 6: w = make_float2(-r2, -r2); break;
    default: w = make_float2(-c8, s8); break;  // m = 9
  }
  if (inv) w.y = -w.y;
  return w;
}

// 16-point DFT in place: n = 4 n1 + n2, k = k1 + 4 k2.
template <bool INV>
__device__ __forceinline__ void dft16(float2 (&x)[16]) {
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4<INV>(x[n2], x[4 + n2], x[8 + n2], x[12 + n2]);
  // now x[4 k1 + n2] holds Y[n2][k1]; twiddle by w16^(n2 k1)
#pragma unroll
  for (int n2 = 1; n2 < 4; ++n2)
#pragma unroll
    for (int k1 = 1; k1 < 4; ++k1) x[4 * k1 + n2] = cmul(x[4 * k1 + n2], w16(n2 * k1, INV));
  // DFT over n2 for every k1 (contiguous group 4 k1 .. 4 k1 + 3) gives X[k1 + 4 k2] at index 4 k1 + k2
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4<INV>(x[4 * k1], x[4 * k1 + 1], x[4 * k1 + 2], x[4 * k1 + 3]);
  // transpose 4 x 4: natural order X[k] at index k
  float2 t[16];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) t[k1 + 4 * k2] = x[4 * k1 + k2];
#pragma unroll
  for (int j = 0; j < 16; ++j) x[j] = t[j];
}

// 8-point DFT in place: n = 4 n1 + n2 (n1 < 2), k = k1 + 2 k2.
template <bool INV>
__device__ __forceinline__ void dft8(float2 (&x)[8]) {
  constexpr float r2 = 0.70710678118654752f;
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft2<INV>(x[n2], x[4 + n2]);
  // x[4 k1 + n2] = Y[n2][k1]; twiddle k1 = 1 by w8^n2
  const float2 w1 = make_float2(r2, INV ? r2 : -r2), w3 = make_float2(-r2, INV ? r2 : -r2);
  x[5] = cmul(x[5], w1);
  x[6] = mul_mi<INV>(x[6]);
  x[7] = cmul(x[7], w3);
  dft4<INV>(x[0], x[1], x[2], x[3]);
  dft4<INV>(x[4], x[5], x[6], x[7]);
  // X[k1 + 2 k2] at index 4 k1 + k2
  float2 t[8];
#pragma unroll
  for (int k1 = 0; k1 < 2; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) t[k1 + 2 * k2] = x[4 * k1 + k2];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = t[j];
}

template <bool INV, int R>
__device__ __forceinline__ void dftR(float2 (&x)[R]) {
  if constexpr (R == 16) dft16<INV>(x);
  else if constexpr (R == 8) dft8<INV>(x);
  else if constexpr (R == 4) dft4<INV>(x[0], x[1], x[2], x[3]);
  else dft2<INV>(x[0], x[1]);
}

// Multiplies x[r] by w^r, r = 1..R-1, for the butterfly whose twiddle row entries start at t (row stride p,
// conjugated for the inverse).  Only w^1, w^2, w^4, w^8 are loaded; the others are products of at most three of
// them (error a few ulp, no extra loads).
template <bool INV, int R>
__device__ __forceinline__ void twiddle(float2 (&x)[R], const float2* __restrict__ t, int p) {
  auto ld = [&](int j) {
    float2 w = t[j * p];
    if (INV) w.y = -w.y;
    return w;
  };
  const float2 w1 = ld(0);
  x[1] = cmul(x[1], w1);
  if constexpr (R >= 4) {
    const float2 w2 = ld(1), w3 = cmul(w1, w2);
    x[2] = cmul(x[2], w2);
    x[3] = cmul(x[3], w3);
    if constexpr (R >= 8) {
      const float2 w4 = ld(2), w5 = cmul(w1, w4), w6 = cmul(w2, w4), w7 = cmul(w3, w4);
      x[4] = cmul(x[4], w4);
      x[5] = cmul(x[5], w5);
      x[6] = cmul(x[6], w6);
      x[7] = cmul(x[7], w7);
      if constexpr (R >= 16) {
        const float2 w8 = ld(3);
        x[8] = cmul(x[8], w8);
        x[9] = cmul(x[9], cmul(w1, w8));
        x[10] = cmul(x[10], cmul(w2, w8));
        x[11] = cmul(x[11], cmul(w3, w8));
        x[12] = cmul(x[12], cmul(w4, w8));
        x[13] = cmul(x[13], cmul(w5, w8));
        x[14] = cmul(x[14], cmul(w6, w8));
        x[15] = cmul(x[15], cmul(w7, w8));
      }
    }
  }
}

// AL (transforms of at least 256 points): the load stride M/R and the store stride p are multiples of 16, or
// p = 1 with R = 16 and 16-aligned outputs, so every padded address is a base plus a multiple of a per-pass
// padded stride; otherwise each address is padded on its own.  BF (nb a power of two): consecutive threads take
// consecutive batches of one butterfly index instead of consecutive butterflies of one batch, so that loads and
// stores through ld / st of batches that sit side by side in global memory (adjacent columns) coalesce.
template <bool INV, int R, int LOGR, int SLOTS, bool AL, bool BF = false, class LD = SmemIO, class ST = SmemIO>
__device__ __forceinline__ void pass(float2* __restrict__ d, int logM, int nb, int bs, int lp,
                                     const float2* __restrict__ ptw, LD ld = LD(), ST st = ST()) {
  constexpr int PER = SLOTS * 16 / R;
  const int MR = 1 << (logM - LOGR), p = 1 << lp, total = nb << (logM - LOGR);
  const int nth = blockDim.x, tid = threadIdx.x;
  const int lstr = MR + (MR >> 4), sstr = p == 1 ? 1 : p + (p >> 4);
  const int lognb = BF ? __ffs(nb) - 1 : 0;
  auto batch_of = [&](int it) { return BF ? (it & (nb - 1)) : it >> (logM - LOGR); };
  float2 v[PER][R];
  int ob[PER];
#pragma unroll
  for (int s = 0; s < PER; ++s) {
    const int it = tid + s * nth;
    ob[s] = -1;
    if (it < total) {
      const int b = batch_of(it), i = BF ? it >> lognb : it & (MR - 1), k = i & (p - 1);
      if constexpr (is_io<LD>) {
#pragma unroll
        for (int r = 0; r < R; ++r) v[s][r] = ld(b, i + r * MR);
      } else if (AL) {
        const float2* src = d + b * bs + pidx(i);
#pragma unroll
        for (int r = 0; r < R; ++r) v[s][r] = src[r * lstr];
      } else {
        const float2* src = d + b * bs;
#pragma unroll
        for (int r = 0; r < R; ++r) v[s][r] = src[pidx(i + r * MR)];
      }
      if (p > 1) twiddle<INV, R>(v[s], ptw + ptw_base(lp, LOGR) + k, p);
      dftR<INV, R>(v[s]);
      const int e0 = (i - k) * R + k;   // + q p
      ob[s] = is_io<ST> ? e0 : b * bs + (AL ? pidx(e0) : e0);
    }
  }
  // in place over the shared buffer, every read of the pass precedes every write; a pass that reads global
  // memory or writes it has no such hazard (the caller makes the buffer free before a transform starts)
  if constexpr (!is_io<LD> && !is_io<ST>) __syncthreads();
#pragma unroll
  for (int s = 0; s < PER; ++s) {
    if (ob[s] >= 0) {
      if constexpr (is_io<ST>) {
        const int b = batch_of(tid + s * nth);
#pragma unroll
        for (int q = 0; q < R; ++q) st(b, ob[s] + q * p, v[s][q]);
      } else if (AL) {
        float2* dst = d + ob[s];
#pragma unroll
        for (int q = 0; q < R; ++q) dst[q * sstr] = v[s][q];
      } else {
        const int b = batch_of(tid + s * nth);
        const int e0 = ob[s] - b * bs;
        float2* dst = d + b * bs;
#pragma unroll
        for (int q = 0; q < R; ++q) dst[pidx(e0 + q * p)] = v[s][q];
      }
    }
  }
  if constexpr (!is_io<ST>) __syncthreads();
}

// ---- transforms of size M = F 2^a, F = 3 or 5 (one radix-F pass, then radix 16 / 8 / 4 / 2) ----

template <bool INV>
__device__ __forceinline__ void dft3(float2& x0, float2& x1, float2& x2) {
  constexpr float h = 0.86602540378443865f;   // sin(2 pi / 3)
  const float2 s = cadd(x1, x2), d = csub(x1, x2);
  const float2 m = make_float2(x0.x - 0.5f * s.x, x0.y - 0.5f * s.y);
  // forward: X1 = m - i h d, X2 = m + i h d (inverse: signs of the i h d term swapped)
  const float2 ihd = make_float2(-h * d.y, h * d.x);
  x0 = cadd(x0, s);
  x1 = INV ? cadd(m, ihd) : csub(m, ihd);
  x2 = INV ? csub(m, ihd) : cadd(m, ihd);
}

// 5-point DFT: with s1 = x1 + x4, d1 = x1 - x4, s2 = x2 + x3, d2 = x2 - x3 and c1, c2, s1', s2' the cosines and
// sines of 2 pi / 5 and 4 pi / 5, X1 = x0 + c1 s1 + c2 s2 - i (s1' d1 + s2' d2), X4 its counterpart with +i,
// X2 = x0 + c2 s1 + c1 s2 - i (s2' d1 - s1' d2), X3 with +i (forward; the inverse swaps the signs of the i terms).
template <bool INV>
__device__ __forceinline__ void dft5(float2& x0, float2& x1, float2& x2, float2& x3, float2& x4) {
  constexpr float c1 = 0.30901699437494742f, c2 = -0.80901699437494742f;   // cos(2 pi / 5), cos(4 pi / 5)
  constexpr float q1 = 0.95105651629515357f, q2 = 0.58778525229247313f;    // sin(2 pi / 5), sin(4 pi / 5)
  const float2 s1 = cadd(x1, x4), d1 = csub(x1, x4), s2 = cadd(x2, x3), d2 = csub(x2, x3);
  const float2 a1 = make_float2(x0.x + c1 * s1.x + c2 * s2.x, x0.y + c1 * s1.y + c2 * s2.y);
  const float2 a2 = make_float2(x0.x + c2 * s1.x + c1 * s2.x, x0.y + c2 * s1.y + c1 * s2.y);
  const float2 b1 = make_float2(q1 * d1.x + q2 * d2.x, q1 * d1.y + q2 * d2.y);   // times -i below
  const float2 b2 = make_float2(q2 * d1.x - q1 * d2.x, q2 * d1.y - q1 * d2.y);
  const float2 ib1 = make_float2(-b1.y, b1.x), ib2 = make_float2(-b2.y, b2.x);  // i b
  x0 = cadd(x0, cadd(s1, s2));
  x1 = INV ? cadd(a1, ib1) : csub(a1, ib1);
  x4 = INV ? csub(a1, ib1) : cadd(a1, ib1);
  x2 = INV ? cadd(a2, ib2) : csub(a2, ib2);
  x3 = INV ? csub(a2, ib2) : cadd(a2, ib2);
}

template <bool INV, int F>
__device__ __forceinline__ void dftF(float2 (&v)[F]) {
  if constexpr (F == 3) dft3<INV>(v[0], v[1], v[2]);
  else dft5<INV>(v[0], v[1], v[2], v[3], v[4]);
}

// floor(x / F) for 0 <= x < 2^31: multiply-high by the rounded-up 2^33 / 3, resp. 2^34 / 5 (exact over that range)
template <int F>
__device__ __forceinline__ int divF(int x) {
  if constexpr (F == 3) return (int)(__umulhi((unsigned)x, 0xAAAAAAABu) >> 1);
  else return (int)(__umulhi((unsigned)x, 0xCCCCCCCDu) >> 2);
}
__device__ __forceinline__ int div3(int x) { return divF<3>(x); }

// First pass (p = 1, no twiddles): butterfly i < 2^a reads x[i + r 2^a], writes F i + q.
template <bool INV, int F, class LD = SmemIO>
__device__ __forceinline__ void passF(float2* __restrict__ d, int a, int nb, int bs, LD ld = LD()) {
  constexpr int PER = (16 + F - 1) / F;       // 16 elements per thread -> at most 16/F butterflies
  const int MR = 1 << a, total = nb << a, nth = blockDim.x, tid = threadIdx.x;
  float2 v[PER][F];
  int ob[PER];
#pragma unroll
  for (int s = 0; s < PER; ++s) {
    const int it = tid + s * nth;
    ob[s] = -1;
    if (it < total) {
      const int b = it >> a, i = it & (MR - 1);
      if constexpr (is_io<LD>) {
#pragma unroll
        for (int r = 0; r < F; ++r) v[s][r] = ld(b, i + r * MR);
      } else {
        const float2* src = d + b * bs;
#pragma unroll
        for (int r = 0; r < F; ++r) v[s][r] = src[pidx(i + r * MR)];
      }
      dftF<INV, F>(v[s]);
      ob[s] = b * bs;
    }
  }
  if constexpr (!is_io<LD>) __syncthreads();
#pragma unroll
  for (int s = 0; s < PER; ++s) {
    if (ob[s] >= 0) {
      const int i = (tid + s * nth) & (MR - 1);
#pragma unroll
      for (int q = 0; q < F; ++q) d[ob[s] + pidx(F * i + q)] = v[s][q];
    }
  }
  __syncthreads();
}

// Later passes: p = F 2^lp2, radix R = 2^LOGR; butterfly i < M / R, k = i mod p, twiddle w_M^{r k M / (R p)}.
template <bool INV, int R, int LOGR, int F, class ST = SmemIO>
__device__ __forceinline__ void passm(float2* __restrict__ d, int a, int nb, int bs, int lp2,
                                      const float2* __restrict__ ptwf, ST st = ST()) {
  constexpr int PER = 16 / R;
  const int MR = F << (a - LOGR), p = F << lp2, total = nb * MR;
  const int nth = blockDim.x, tid = threadIdx.x;
  float2 v[PER][R];
  int ob[PER];
#pragma unroll
  for (int s = 0; s < PER; ++s) {
    const int it = tid + s * nth;
    ob[s] = -1;
    if (it < total) {
      const int b = divF<F>(it >> (a - LOGR)), i = it - b * MR;   // it / MR, MR = F 2^(a - LOGR)
      const int k = i - p * divF<F>(i >> lp2);                      // i mod p, p = F 2^lp2
      const float2* src = d + b * bs;
#pragma unroll
      for (int r = 0; r < R; ++r) v[s][r] = src[pidx(i + r * MR)];
      if (k) twiddle<INV, R>(v[s], ptwf + ptwf_base(F, a, lp2) + k, p);
      dftR<INV, R>(v[s]);
      ob[s] = b * bs + (i - k) * R + k;
    }
  }
  if constexpr (!is_io<ST>) __syncthreads();
#pragma unroll
  for (int s = 0; s < PER; ++s) {
    if (ob[s] >= 0) {
      const int b = divF<F>((tid + s * nth) >> (a - LOGR));
      const int e0 = ob[s] - b * bs;
      if constexpr (is_io<ST>) {
#pragma unroll
        for (int q = 0; q < R; ++q) st(b, e0 + q * p, v[s][q]);
      } else {
        float2* dst = d + b * bs;
#pragma unroll
        for (int q = 0; q < R; ++q) dst[pidx(e0 + q * p)] = v[s][q];
      }
    }
  }
  if constexpr (!is_io<ST>) __syncthreads();
}

}  // namespace fftp

// FFTs of size M = F 2^a (a >= 1) over nb batches in the padded layout, in place; same contract as fft_p.
namespace fftp {
// passm from p = F 2^LP2 on, the last one writing through st
template <bool INV, int F, int A, int LP2, class ST>
__device__ __forceinline__ void fft_pf_from(float2* __restrict__ d, int nb, int bs, const float2* __restrict__ ptwf,
                                            ST st) {
  constexpr int left = A - LP2;
  if constexpr (left > 4) {
    passm<INV, 16, 4, F>(d, A, nb, bs, LP2, ptwf);
    fft_pf_from<INV, F, A, LP2 + 4, ST>(d, nb, bs, ptwf, st);
  } else {
    passm<INV, 1 << left, left, F, ST>(d, A, nb, bs, LP2, ptwf, st);
  }
}

template <bool INV, int F, int A, class LD, class ST>
__device__ __forceinline__ void fft_pf_fixed(float2* __restrict__ d, int nb, int bs, const float2* __restrict__ ptwf,
                                             LD ld, ST st) {
  passF<INV, F, LD>(d, A, nb, bs, ld);
  fft_pf_from<INV, F, A, 0, ST>(d, nb, bs, ptwf, st);
}

template <bool INV, int F>
__device__ __forceinline__ void fft_pf_generic(float2* __restrict__ d, int a, int nb, int bs,
                                               const float2* __restrict__ ptwf) {
  passF<INV, F>(d, a, nb, bs);
  int lp2 = 0;
  for (; a - lp2 >= 4; lp2 += 4) passm<INV, 16, 4, F>(d, a, nb, bs, lp2, ptwf);
  const int rem = a - lp2;
  if (rem == 3) passm<INV, 8, 3, F>(d, a, nb, bs, lp2, ptwf);
  else if (rem == 2) passm<INV, 4, 2, F>(d, a, nb, bs, lp2, ptwf);
  else if (rem == 1) passm<INV, 2, 1, F>(d, a, nb, bs, lp2, ptwf);
}

// Transforms of a size without a compile-time variant: the functors run as a staging loop before / after.
template <bool INV, class LD>
__device__ __forceinline__ void stage_in(float2* __restrict__ d, int M, int nb, int bs, LD ld) {
  if constexpr (is_io<LD>) {
    for (int e = threadIdx.x; e < nb * M; e += blockDim.x) {
      const int b = e / M, j = e - b * M;
      d[b * bs + pidx(j)] = ld(b, j);
    }
    __syncthreads();
  }
}
template <bool INV, class ST>
__device__ __forceinline__ void stage_out(const float2* __restrict__ d, int M, int nb, int bs, ST st) {
  if constexpr (is_io<ST>) {
    for (int e = threadIdx.x; e < nb * M; e += blockDim.x) {
      const int b = e / M, j = e - b * M;
      st(b, j, d[b * bs + pidx(j)]);
    }
  }
}
}  // namespace fftp

// FFTs of size M = F 2^a (F = 3 or 5), with the inputs taken through ld and the outputs put through st (the
// fftp::SmemIO defaults keep them in the buffer).  With st a functor the call ends without a barrier.  The row
// lengths of the convolutions (F 2^a, a = 8..10 for F = 3, 7..9 for F = 5) run unrolled pass sequences.
template <bool INV, int F, class LD = fftp::SmemIO, class ST = fftp::SmemIO>
__device__ void fft_pf_io(float2* __restrict__ d, int a, int nb, int bs, const float2* __restrict__ ptwf,
                          LD ld = LD(), ST st = ST()) {
  if constexpr (F == 3) {
    switch (a) {
      case 10: fftp::fft_pf_fixed<INV, 3, 10>(d, nb, bs, ptwf, ld, st); return;
      case 9: fftp::fft_pf_fixed<INV, 3, 9>(d, nb, bs, ptwf, ld, st); return;
      case 8: fftp::fft_pf_fixed<INV, 3, 8>(d, nb, bs, ptwf, ld, st); return;
      default: break;
    }
  } else {
    switch (a) {
      case 9: fftp::fft_pf_fixed<INV, 5, 9>(d, nb, bs, ptwf, ld, st); return;
      case 8: fftp::fft_pf_fixed<INV, 5, 8>(d, nb, bs, ptwf, ld, st); return;
      case 7: fftp::fft_pf_fixed<INV, 5, 7>(d, nb, bs, ptwf, ld, st); return;
      default: break;
    }
  }
  fftp::stage_in<INV>(d, F << a, nb, bs, ld);
  fftp::fft_pf_generic<INV, F>(d, a, nb, bs, ptwf);
  fftp::stage_out<INV>(d, F << a, nb, bs, st);
}

template <bool INV, class LD = fftp::SmemIO, class ST = fftp::SmemIO>
__device__ void fft_p3_io(float2* __restrict__ d, int a, int nb, int bs, const float2* __restrict__ ptw3, LD ld = LD(),
                          ST st = ST()) {
  fft_pf_io<INV, 3>(d, a, nb, bs, ptw3, ld, st);
}

// FFTs of size M = 3 * 2^a (a >= 1) over nb batches in the padded layout, in place; same contract as fft_p.
template <bool INV>
__device__ void fft_p3(float2* __restrict__ d, int a, int nb, int bs, const float2* __restrict__ ptw3) {
  fft_p3_io<INV>(d, a, nb, bs, ptw3);
}

// FFTs of size M = 2^logM (M <= 8192) over nb batches, padded layout (element e of batch b at
// d[b * bs + pidx(e)]), in place.  Requires nb * M <= 16 * SLOTS * blockDim.x (SLOTS x 16 elements per thread
// and pass).  Forward: exp(-2 pi i nk/M); inverse: exp(+...), unscaled.  The caller synchronises before the
// call; the call ends with a barrier.
namespace fftp {
template <bool INV, int SLOTS, bool AL, bool BF = false>
__device__ __forceinline__ void fft_p_impl(float2* __restrict__ d, int logM, int nb, int bs,
                                           const float2* __restrict__ ptw) {
  int lp = 0;
  for (; logM - lp >= 4; lp += 4) pass<INV, 16, 4, SLOTS, AL, BF>(d, logM, nb, bs, lp, ptw);
  const int rem = logM - lp;
  if (rem == 3) pass<INV, 8, 3, SLOTS, AL, BF>(d, logM, nb, bs, lp, ptw);
  else if (rem == 2) pass<INV, 4, 2, SLOTS, AL, BF>(d, logM, nb, bs, lp, ptw);
  else if (rem == 1) pass<INV, 2, 1, SLOTS, AL, BF>(d, logM, nb, bs, lp, ptw);
}
}  // namespace fftp

namespace fftp {
// The same passes for a size known at compile time: with logM and every pass offset literal, the strides,
// masks, shifts and twiddle-table bases of the inlined passes fold into immediates.  The first pass reads
// through ld, the last writes through st.
template <bool FIRST, class LD>
__device__ __forceinline__ auto first_ld(LD ld) {
  if constexpr (FIRST) return ld;
  else return SmemIO();
}

// BF applies to the passes that read or write global memory (the first with ld, the last with st); the passes
// between keep the batch-major order, whose shared-memory stores are free of bank conflicts.
template <bool INV, int SLOTS, bool BF, int LOGM, int LP, class LD, class ST>
__device__ __forceinline__ void fft_p_from(float2* __restrict__ d, int nb, int bs, const float2* __restrict__ ptw,
                                           LD ld, ST st) {
  constexpr bool AL = LOGM >= 8;
  constexpr int left = LOGM - LP;
  const auto l = first_ld<LP == 0>(ld);
  using L = std::remove_const_t<decltype(l)>;
  if constexpr (left > 4) {
    pass<INV, 16, 4, SLOTS, AL, BF && is_io<L>, L, SmemIO>(d, LOGM, nb, bs, LP, ptw, l, SmemIO());
    fft_p_from<INV, SLOTS, BF, LOGM, LP + 4, LD, ST>(d, nb, bs, ptw, ld, st);
  } else {
    pass<INV, 1 << left, left, SLOTS, AL, BF && (is_io<L> || is_io<ST>), L, ST>(d, LOGM, nb, bs, LP, ptw, l, st);
  }
}
}  // namespace fftp

// FFTs of size 2^logM as fft_p, with the inputs taken through ld and the outputs put through st (the
// fftp::SmemIO defaults keep them in the buffer).  With st a functor the call ends without a barrier; with ld
// a functor the caller must not be using the buffer any more when the call starts.
// BF: the batch-fastest thread order of the passes (nb must be a power of two).
template <bool INV, int SLOTS = 1, bool BF = false, class LD = fftp::SmemIO, class ST = fftp::SmemIO>
__device__ void fft_p_io(float2* __restrict__ d, int logM, int nb, int bs, const float2* __restrict__ ptw,
                         LD ld = LD(), ST st = ST()) {
  switch (logM) {   // the sizes of the console's transforms run with compile-time strides
    case 13: fftp::fft_p_from<INV, SLOTS, BF, 13, 0>(d, nb, bs, ptw, ld, st); return;
    case 12: fftp::fft_p_from<INV, SLOTS, BF, 12, 0>(d, nb, bs, ptw, ld, st); return;
    case 11: fftp::fft_p_from<INV, SLOTS, BF, 11, 0>(d, nb, bs, ptw, ld, st); return;
    case 10: fftp::fft_p_from<INV, SLOTS, BF, 10, 0>(d, nb, bs, ptw, ld, st); return;
    case 9: fftp::fft_p_from<INV, SLOTS, BF, 9, 0>(d, nb, bs, ptw, ld, st); return;
    case 8: fftp::fft_p_from<INV, SLOTS, BF, 8, 0>(d, nb, bs, ptw, ld, st); return;
    default: break;
  }
  fftp::stage_in<INV>(d, 1 << logM, nb, bs, ld);
  if (logM >= 8) fftp::fft_p_impl<INV, SLOTS, true, BF>(d, logM, nb, bs, ptw);
  else fftp::fft_p_impl<INV, SLOTS, false, BF>(d, logM, nb, bs, ptw);
  fftp::stage_out<INV>(d, 1 << logM, nb, bs, st);
}

template <bool INV, int SLOTS = 1>
__device__ void fft_p(float2* __restrict__ d, int logM, int nb, int bs, const float2* __restrict__ ptw) {
  fft_p_io<INV, SLOTS>(d, logM, nb, bs, ptw);
}

}  // namespace mg

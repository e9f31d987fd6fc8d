// Shared-memory complex FFT (Stockham autosort, radix 4 with one radix-2 pass for odd log sizes) and
// complex helpers.  Used for the convolutions of the equalizer / reverb / delay (Sec. 3.3, 3.4, 3.7) and
// for the STFTs of the loss (Sec. 5.1).
#pragma once
#include <cuda_runtime.h>
#include "mg_internal.cuh"

namespace mg {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cmuli(float2 a) { return make_float2(-a.y, a.x); }  // i * a

// exp(sign * 2 pi i m / N) for power-of-two N (m < 2^23 so that 2m/N is exact in fp32).
__device__ __forceinline__ float2 twiddle_pow2(unsigned m, int logN, bool inverse) {
  float s, c;
  sincospif(ldexpf((float)m, 1 - logN), &s, &c);
  return make_float2(c, inverse ? s : -s);
}

// exp(-+2 pi i m / 2^logN), m < 2^logN <= 2^26, from the tables: the top 13 bits of m index the coarse table,
// the rest the fine one, and the two entries are multiplied (about 1.5 ulp).
__device__ __forceinline__ float2 twiddle_tab(unsigned m, int logN, bool inverse, const Tables& t) {
  float2 w;
  if (logN <= kTwLog) {
    w = t.tw[m << (kTwLog - logN)];
  } else {
    const int lo = logN - kTwLog;
    w = cmul(t.tw[m >> lo], t.twf[(m & ((1u << lo) - 1)) << (kTwFineLog - logN)]);
  }
  if (inverse) w.y = -w.y;
  return w;
}

// In-place FFTs of size M = 2^logM over nb batches held in shared memory: element e of batch b sits at
// d[b * bs + e * es].  Forward: X[k] = sum_n x[n] exp(-2 pi i nk/M); inverse: exp(+...), unscaled.
// Each pass reads all operands into registers, synchronises, then writes, so the caller must
// synchronise before the call (data visible) and may rely on a barrier at exit.
// MAXPER bounds the radix-4 butterflies per thread: nb * M / 4 <= MAXPER * blockDim.x.
template <bool INV, int MAXPER>
__device__ void fft_smem(float2* __restrict__ d, int logM, int nb, int es, int bs, const float2* __restrict__ tw) {
  const int M = 1 << logM;
  const int nth = blockDim.x, tid = threadIdx.x;
  int lp = 0;
  for (; lp + 2 <= logM; lp += 2) {
    const int p = 1 << lp, q = M >> 2, total = nb * q;
    float2 v[MAXPER][4];
    int ob[MAXPER], oj[MAXPER];
#pragma unroll
    for (int s = 0; s < MAXPER; ++s) {
      const int it = tid + s * nth;
      ob[s] = -1;
      if (it < total) {
        int b, i;
        if (es == 1) {
          b = it >> (logM - 2);
          i = it & (q - 1);
        } else {
          b = it % nb;
          i = it / nb;
        }
        const int k = i & (p - 1);
        const float2* src = d + b * bs;
        float2 x0 = src[i * es], x1 = src[(i + q) * es], x2 = src[(i + 2 * q) * es], x3 = src[(i + 3 * q) * es];
        if (p > 1) {
          const int sh = kTwLog - lp - 2;
          float2 w1 = tw[k << sh], w2 = tw[(2 * k) << sh], w3 = tw[(3 * k) << sh];
          if (INV) {
            w1.y = -w1.y;
            w2.y = -w2.y;
            w3.y = -w3.y;
          }
          x1 = cmul(x1, w1);
          x2 = cmul(x2, w2);
          x3 = cmul(x3, w3);
        }
        const float2 a0 = cadd(x0, x2), a1 = csub(x0, x2), a2 = cadd(x1, x3), a3 = csub(x1, x3);
        const float2 ia3 = INV ? cmuli(a3) : make_float2(a3.y, -a3.x);  // +i a3 (inverse) or -i a3 (forward)
        v[s][0] = cadd(a0, a2);
        v[s][1] = cadd(a1, ia3);
        v[s][2] = csub(a0, a2);
        v[s][3] = csub(a1, ia3);
        ob[s] = b;
        oj[s] = (i - k) * 4 + k;
      }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < MAXPER; ++s) {
      if (ob[s] >= 0) {
        float2* dst = d + ob[s] * bs;
        dst[oj[s] * es] = v[s][0];
        dst[(oj[s] + p) * es] = v[s][1];
        dst[(oj[s] + 2 * p) * es] = v[s][2];
        dst[(oj[s] + 3 * p) * es] = v[s][3];
      }
    }
    __syncthreads();
  }
  if (lp < logM) {  // final radix-2 pass, p = M / 2
    const int p = 1 << lp, h = M >> 1, total = nb * h;
    float2 v[2 * MAXPER][2];
    int ob[2 * MAXPER], oj[2 * MAXPER];
#pragma unroll
    for (int s = 0; s < 2 * MAXPER; ++s) {
      const int it = tid + s * nth;
      ob[s] = -1;
      if (it < total) {
        int b, i;
        if (es == 1) {
          b = it >> (logM - 1);
          i = it & (h - 1);
        } else {
          b = it % nb;
          i = it / nb;
        }
        const int k = i & (p - 1);
        const float2* src = d + b * bs;
        float2 x0 = src[i * es], x1 = src[(i + h) * es];
        if (p > 1) {
          float2 w = tw[k << (kTwLog - lp - 1)];
          if (INV) w.y = -w.y;
          x1 = cmul(x1, w);
        }
        v[s][0] = cadd(x0, x1);
        v[s][1] = csub(x0, x1);
        ob[s] = b;
        oj[s] = (i - k) * 2 + k;
      }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < 2 * MAXPER; ++s) {
      if (ob[s] >= 0) {
        float2* dst = d + ob[s] * bs;
        dst[oj[s] * es] = v[s][0];
        dst[(oj[s] + p) * es] = v[s][1];
      }
    }
    __syncthreads();
  }
}

// Block-wide sum of NV floats per thread into out[0..NV) (thread 0 result), deterministic order.
template <int NV>
__device__ __forceinline__ void block_sum(float (&v)[NV], float* red /* smem >= NV * 32 */, float* out) {
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    float x = v[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    v[j] = x;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) red[j * 32 + wid] = v[j];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      float x = lane < nw ? red[j * 32 + lane] : 0.f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if (lane == 0) out[j] = x;
    }
  }
  __syncthreads();
}

__device__ __forceinline__ float sigmoidf_(float x) { return 1.f / (1.f + __expf(-x)); }

__device__ __forceinline__ float dry_wet_w(const LaunchCtx& c, int qidx) {
  const float w = 1.f / (1.f + expf(-c.q[qidx]));
  return c.mask ? w * (float)c.mask[qidx] : w;
}

// The dry weight 1 - w, evaluated as sigmoid(-q) (1 where the mask is 0) so that it keeps full relative
// precision when w is close to 1.
__device__ __forceinline__ float dry_wet_d(const LaunchCtx& c, int qidx) {
  if (c.mask && !c.mask[qidx]) return 1.f;
  return 1.f / (1.f + expf(c.q[qidx]));
}

}  // namespace mg

// Evaluation metrics of the matched mix against the target (Sec. 5.3): SI-SDR over the stereo signal and the
// MIR feature distances of Eq. (27) over disjoint 8 s segments: RMS and crest factor per channel, stereo
// width ||l - r|| / ||l + r||, stereo imbalance (||l||^2 - ||r||^2) / (||l||^2 + ||r||^2), and the 24-band
// Zwicker Bark spectrum of the mid signal (l + r) / 2 from Hann-windowed 8192-sample frames with hop 8192
// (mean power per band, in dB).  A song shorter than 8 s is one segment.
//
// One CTA per (song, segment): the segment statistics of the estimate and the reference, their Bark spectra
// (two consecutive frames of one signal packed as one complex FFT), and the SI-SDR sums over the segment
// (the last segment of a song also takes the samples after the last full segment).  A per-song kernel
// combines the segments in a fixed order (double precision).
#include "mg_fftp.cuh"

namespace mg {

namespace {
constexpr int kEvThreads = 512;
constexpr int kBarkFrame = 8192;
constexpr int kBarkLog = 13;
constexpr int kBands = 24;
// per item (doubles): 0-7 energies, 8-11 peaks, 12-59 band powers (estimate, reference), 60-61 and 63 SI-SDR
// sums, 62 frames, 64 segment length
constexpr int kEvStride = 66;

template <int NV>
__device__ __forceinline__ void block_reduce_d(double (&v)[NV], double* red) {
  // sum over the block, result in thread 0
#pragma unroll
  for (int k = 0; k < NV; ++k)
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) red[w * NV + k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0.0;
      for (int j = 0; j < nw; ++j) s += red[j * NV + k];
      v[k] = s;
    }
  __syncthreads();
}

__device__ __forceinline__ float warp_max(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}
}  // namespace

// item = (song, segment); band_lo/band_hi: [24] bin range of each Bark band
__global__ void __launch_bounds__(kEvThreads) k_eval_seg(const SongDev* __restrict__ songs, const int2* __restrict__ items,
                                                         int seg_len, const int* __restrict__ band_lo,
                                                         const int* __restrict__ band_hi, double* __restrict__ out,
                                                         const float2* __restrict__ ptw) {
  extern __shared__ float2 sm[];
  __shared__ double red[16 * 16];
  __shared__ float mred[2][16];
  const int2 it = items[blockIdx.x];
  const SongDev& S = songs[it.x];
  const int nseg = S.L < seg_len ? 1 : S.L / seg_len;
  const int s0 = it.y * (S.L < seg_len ? 0 : seg_len);
  const int s1 = S.L < seg_len ? S.L : s0 + seg_len;
  const int s2 = it.y == nseg - 1 ? S.L : s1;      // SI-SDR sums run to the end of the song on the last segment
  const float* el = S.mix;
  const float* er = S.mix + S.ld;
  const float* rl = S.target;
  const float* rr = S.target + S.ld;
  // statistics: 0..3 est sum l^2, r^2, (l-r)^2, (l+r)^2; 4..7 the same for the reference;
  // SI-SDR sums 8 <e,r>, 9 <r,r>, 10 <e,e>
  double acc[11] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  float pk[4] = {0.f, 0.f, 0.f, 0.f};
  for (int s = s0 + threadIdx.x; s < s2; s += blockDim.x) {
    const float a = el[s], b = er[s], c = rl[s], d = rr[s];
    acc[8] += (double)a * c + (double)b * d;
    acc[9] += (double)c * c + (double)d * d;
    acc[10] += (double)a * a + (double)b * b;
    if (s < s1) {
      acc[0] += (double)a * a;
      acc[1] += (double)b * b;
      acc[2] += (double)(a - b) * (a - b);
      acc[3] += (double)(a + b) * (a + b);
      acc[4] += (double)c * c;
      acc[5] += (double)d * d;
      acc[6] += (double)(c - d) * (c - d);
      acc[7] += (double)(c + d) * (c + d);
      pk[0] = fmaxf(pk[0], fabsf(a));
      pk[1] = fmaxf(pk[1], fabsf(b));
      pk[2] = fmaxf(pk[2], fabsf(c));
      pk[3] = fmaxf(pk[3], fabsf(d));
    }
  }
  block_reduce_d<11>(acc, red);
  float pmax[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) pmax[k] = warp_max(pk[k]);
  double* o = out + (size_t)blockIdx.x * kEvStride;
  {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    for (int k = 0; k < 4; ++k) {
      if (lane == 0) mred[k & 1][w] = pmax[k];
      __syncthreads();
      if (threadIdx.x == 0) {
        float m = 0.f;
        for (int j = 0; j < nw; ++j) m = fmaxf(m, mred[k & 1][j]);
        o[8 + k] = m;
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) {
    for (int k = 0; k < 8; ++k) o[k] = acc[k];
    o[64] = s1 - s0;
    o[60] = acc[8];
    o[61] = acc[9];
    o[63] = acc[10];
  }
  // Bark spectra: frames [s0 + f 8192, ...) inside [s0, s1).  Two consecutive frames of the same signal travel
  // packed as one complex FFT (z = frame f + i frame f+1; signals of very different level are never mixed).
  const int nfr = (s1 - s0) / kBarkFrame;
  const int rs = pstride(kBarkFrame);
  double bacc[2 * kBands];
  for (int k = 0; k < 2 * kBands; ++k) bacc[k] = 0.0;
  for (int sig = 0; sig < 2; ++sig) {
    const float* xl = sig ? rl : el;
    const float* xr = sig ? rr : er;
    for (int f = 0; f < nfr; f += 2) {
      const int b0 = s0 + f * kBarkFrame;
      const bool two = f + 1 < nfr;
      __syncthreads();
      for (int j = threadIdx.x; j < kBarkFrame; j += blockDim.x) {
        const float w = 0.5f * (1.f - cospif(2.f * j / kBarkFrame));
        const int s = b0 + j;
        const float a = 0.5f * (xl[s] + xr[s]) * w;
        const float b = two ? 0.5f * (xl[s + kBarkFrame] + xr[s + kBarkFrame]) * w : 0.f;
        sm[pidx(j)] = make_float2(a, b);
      }
      __syncthreads();
      fft_p<false>(sm, kBarkLog, 1, rs, ptw);
      for (int b = 0; b < kBands; ++b) {
        double p = 0.0;
        for (int k = band_lo[b] + (int)threadIdx.x; k < band_hi[b]; k += blockDim.x) {
          const float2 z = sm[pidx(k)], zm = sm[pidx((kBarkFrame - k) & (kBarkFrame - 1))];
          const float ar = 0.5f * (z.x + zm.x), ai = 0.5f * (z.y - zm.y);      // frame f
          const float br = 0.5f * (z.y + zm.y), bi = 0.5f * (zm.x - z.x);      // frame f + 1
          p += (double)ar * ar + (double)ai * ai + (double)br * br + (double)bi * bi;
        }
        bacc[sig * kBands + b] += p;
      }
    }
  }
  // reduce the band sums over the block in two halves of 24
  for (int h = 0; h < 2; ++h) {
    double v[kBands];
#pragma unroll
    for (int b = 0; b < kBands; ++b) v[b] = bacc[h * kBands + b];
    for (int kb = 0; kb < kBands; kb += 8) {
      double part[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) part[k] = v[kb + k];
      block_reduce_d<8>(part, red);
      if (threadIdx.x == 0)
        for (int k = 0; k < 8; ++k) o[12 + h * kBands + kb + k] = nfr ? part[k] / nfr : 0.0;
    }
  }
  if (threadIdx.x == 0) o[62] = nfr;
}

// out_song [n][6]: SI-SDR (dB), d_rms, d_cf, d_sw, d_si, d_bs (Eq. 27; -inf when the features agree exactly)
__global__ void k_eval_finalize(const int* __restrict__ item_begin,
                                const double* __restrict__ seg, float* __restrict__ out_song) {
  if (threadIdx.x != 0) return;
  const int si = blockIdx.x;
  const int a = item_begin[si], b = item_begin[si + 1];
  double dot = 0.0, rr = 0.0, ee = 0.0;
  double acc[5] = {0, 0, 0, 0, 0};
  int cnt[5] = {0, 0, 0, 0, 0};
  auto q = [](double n, double d) { return d != 0.0 ? n / d : 0.0; };
  for (int i = a; i < b; ++i) {
    const double* o = seg + (size_t)i * kEvStride;
    dot += o[60];
    rr += o[61];
    ee += o[63];
  }
  // SI-SDR: ||alpha r||^2 / ||alpha r - e||^2 with ||alpha r - e||^2 = ||e||^2 - alpha <e, r>, alpha = <e,r>/||r||^2
  const double alpha = q(dot, rr);
  const double tgt = alpha * alpha * rr, res = ee - alpha * dot;
  out_song[si * 6 + 0] = (float)(10.0 * log10(tgt / res));
  for (int i = a; i < b; ++i) {
    const double* o = seg + (size_t)i * kEvStride;
    const double n = o[64];   // samples in the segment
    const double fe[6] = {sqrt(o[0] / n), sqrt(o[1] / n), q(o[8], sqrt(o[0] / n)), q(o[9], sqrt(o[1] / n)),
                          q(sqrt(o[2]), sqrt(o[3])), q(o[0] - o[1], o[0] + o[1])};
    const double fr[6] = {sqrt(o[4] / n), sqrt(o[5] / n), q(o[10], sqrt(o[4] / n)), q(o[11], sqrt(o[5] / n)),
                          q(sqrt(o[6]), sqrt(o[7])), q(o[4] - o[5], o[4] + o[5])};
    for (int k = 0; k < 2; ++k) {
      acc[0] += (fe[k] - fr[k]) * (fe[k] - fr[k]);
      acc[1] += (fe[2 + k] - fr[2 + k]) * (fe[2 + k] - fr[2 + k]);
    }
    cnt[0] += 2;
    cnt[1] += 2;
    acc[2] += (fe[4] - fr[4]) * (fe[4] - fr[4]);
    acc[3] += (fe[5] - fr[5]) * (fe[5] - fr[5]);
    cnt[2] += 1;
    cnt[3] += 1;
    for (int bnd = 0; bnd < kBands; ++bnd) {
      const double de = 10.0 * log10(o[12 + bnd] + 1e-12), dr = 10.0 * log10(o[12 + kBands + bnd] + 1e-12);
      acc[4] += (de - dr) * (de - dr);
    }
    cnt[4] += kBands;
  }
  for (int k = 0; k < 5; ++k) out_song[si * 6 + 1 + k] = acc[k] > 0.0 ? (float)log10(acc[k] / cnt[k]) : -INFINITY;
}

void launch_eval(cudaStream_t st, const SongDev* songs, int n_songs, const int2* items, int n_items,
                 const int* item_begin, int seg_len, const int* band_lo, const int* band_hi, double* seg_out,
                 float* out_song, const float2* ptw) {
  if (!n_items) return;
  k_eval_seg<<<n_items, kEvThreads, pstride(kBarkFrame) * sizeof(float2), st>>>(songs, items, seg_len, band_lo,
                                                                                  band_hi, seg_out, ptw);
  k_eval_finalize<<<n_songs, 32, 0, st>>>(item_begin, seg_out, out_song);
}

void init_eval_attributes() {
  cudaFuncSetAttribute(k_eval_seg, cudaFuncAttributeMaxDynamicSharedMemorySize, pstride(kBarkFrame) * (int)sizeof(float2));
}

}  // namespace mg

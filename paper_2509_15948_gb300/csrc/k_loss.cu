// Multi-resolution STFT loss of Sec. 5.1 (Eqs. 20-21) and its adjoint.
// Per resolution: frames t hop .. t hop + n_fft of the stereo mix (periodic Hann, no centre padding) are
// transformed as one packed complex FFT z = left + i right; per bin the channel spectra are
// X_L = (Z[k] + conj Z[-k]) / 2, X_R = (Z[k] - conj Z[-k]) / 2i, X_M = X_L + X_R, X_S = X_L - X_R;
// magnitudes sqrt(A_k^2 |X|^2 + 1e-8) (A-weighting per bin) are projected on the Mel triangles (CSR by
// band, fixed summation order), compared with the cached target spectrograms, and reduced per work item
// (deterministic partial sums, no atomics).
// Adjoint: the same frames are re-transformed, dL/dY_hat per band goes back to the bins through the
// transposed Mel CSR, to the complex bins through |X|, to the packed Hermitian spectrum, and through one
// inverse FFT to the windowed frame; a gather kernel overlap-adds the frames of all resolutions.
#include "mg_fftp.cuh"

namespace mg {

namespace {
constexpr int kLossThreads = 512;
constexpr float kLogEps = 1e-5f;
constexpr float kMagEps = 1e-8f;
// frames of one item live in a padded layout: frame f, sample j at sm[f * pstride(n) + pidx(j)];
// an item holds 8192 samples (8192 / n_fft <= 128 frames), so the buffer needs 8192 + 512 + 128 entries.
constexpr int kFrameBuf = kLossFrameBuf;

// channel magnitudes^2 of bin k (|X_L|^2, |X_R|^2, |X_M|^2, |X_S|^2) and the complex X_L, X_R
__device__ __forceinline__ void bin_spectra(const float2* Z, int k, int n, float2& XL, float2& XR) {
  const float2 a = Z[pidx(k)], b = Z[pidx((n - k) & (n - 1))];
  XL = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
  // (a - conj b) / 2i
  const float2 d = make_float2(a.x - b.x, a.y + b.y);
  XR = make_float2(0.5f * d.y, -0.5f * d.x);
}

__device__ __forceinline__ float2 chan(int c, float2 XL, float2 XR) {
  if (c == 0) return XL;
  if (c == 1) return XR;
  if (c == 2) return cadd(XL, XR);
  return csub(XL, XR);
}

// After the magnitude pass a frame holds, for bin k in [0, n/2], the weighted magnitudes
// sqrt(A_k^2 |X_c|^2 + 1e-8) of channels 0, 1 at slot pidx(k) and of channels 2, 3 at mag_slot2(k): the
// mirror slot pidx(n - k), or for the self-mirrored bins 0 and n/2 two padding slots no element uses
// (pidx(n) = the last slot of the padded frame, and slot 16).
__device__ __forceinline__ int mag_slot2(int k, int n) {
  return k == 0 ? pidx(n) : (k == (n >> 1) ? 16 : pidx(n - k));
}

__device__ __forceinline__ float4 bin_mags(const LossRes& R, const float2* Z, int k) {
  float2 XL, XR;
  bin_spectra(Z, k, R.nfft, XL, XR);
  const float a = R.aw2[k];
  float m[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const float2 X = chan(c, XL, XR);
    m[c] = sqrtf(a * (X.x * X.x + X.y * X.y) + kMagEps);
  }
  return make_float4(m[0], m[1], m[2], m[3]);
}
}  // namespace

// item (song, res, first frame, frames); mode 0: write target spectrogram + partial sum Y^2 per set;
// mode 1: partial sums of |dlog| and (Y - Yhat)^2 per set; mode 3: mode 1 that also keeps the frame spectra
// (in dF, which the adjoint overwrites frame by frame) and the band values Yhat (training forward);
// mode 2: adjoint frames to dF from the kept spectra and band values.
__global__ void __launch_bounds__(kLossThreads, 2) k_loss_frames(LaunchCtx c, const SongDev* __restrict__ songs,
                                                              const LossRes* __restrict__ resv,
                                                              const int4* __restrict__ items, int mode) {
  extern __shared__ float2 sm[];
  __shared__ float red[6 * 32];
  const int4 it = items[blockIdx.x];
  const SongDev& S = songs[it.x];
  const LossRes& R = resv[it.y];
  const int t0 = it.z, nb = it.w, n = R.nfft, nbands = R.nbands, bs = pstride(n);
  const float* x = mode == 0 ? S.target : S.mix;
  float2* Zk = reinterpret_cast<float2*>(S.dF[it.y]);     // frame spectra kept between mode 3 and mode 2
  if (mode == 2) {
    for (int e = threadIdx.x; e < nb * n; e += blockDim.x) {
      const int f = e >> R.log_nfft, j = e & (n - 1);
      sm[f * bs + pidx(j)] = Zk[(size_t)(t0 + f) * n + j];
    }
    __syncthreads();
  } else {
    // the windowed frames go straight from global memory into the first pass of the transform
    const int L = S.L, ld = S.ld, hop = R.hop;
    const float* win = R.win;
    fft_p_io<false>(sm, R.log_nfft, nb, bs, c.tab.ptw, [=](int f, int j) {
      const int s = (t0 + f) * hop + j;
      const float w = win[j];
      return s < L ? make_float2(x[s] * w, x[ld + s] * w) : make_float2(0.f, 0.f);
    });
    if (mode == 3)
      for (int e = threadIdx.x; e < nb * n; e += blockDim.x) {
        const int f = e >> R.log_nfft, j = e & (n - 1);
        Zk[(size_t)(t0 + f) * n + j] = sm[f * bs + pidx(j)];
      }
  }
  float* Yt = S.Y[it.y];
  float* Yk = S.Yh[it.y];
  if (mode != 2) {
    // magnitudes of the four channels per bin, in place (each thread owns the pair k, n - k; the thread of
    // k = 0 also takes k = n/2)
    const int half = n >> 1, lh = R.log_nfft - 1;
    __syncthreads();   // mode 3: every thread has copied its part of the spectrum out
    for (int e = threadIdx.x; e < nb << lh; e += blockDim.x) {
      const int f = e >> lh, k = e & (half - 1);
      float2* Z = sm + f * bs;
      if (k == 0) {
        const float4 m0 = bin_mags(R, Z, 0), mh = bin_mags(R, Z, half);
        Z[pidx(0)] = make_float2(m0.x, m0.y);
        Z[mag_slot2(0, n)] = make_float2(m0.z, m0.w);
        Z[pidx(half)] = make_float2(mh.x, mh.y);
        Z[mag_slot2(half, n)] = make_float2(mh.z, mh.w);
      } else {
        const float4 m = bin_mags(R, Z, k);
        Z[pidx(k)] = make_float2(m.x, m.y);
        Z[pidx(n - k)] = make_float2(m.z, m.w);
      }
    }
    __syncthreads();
    // band values from the magnitudes: with narrow bands (few Mel weights per band on average) one thread per
    // (frame, band, channel); with wide ones one warp per (frame, band), its lanes striding the band's bins and
    // the four channel sums reduced over the warp (a fixed xor order), so a wide high band no longer holds the
    // whole block at the barrier behind one thread
    float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    auto band_out = [&](int f, int b, int ch, float yh) {
      const int set = ch < 2 ? 0 : ch - 1;
      const size_t yi = ((size_t)(t0 + f) * nbands + b) * 4 + ch;
      float* ydst = Yt + yi;
      if (mode == 3) Yk[yi] = yh;
      if (mode == 0) {
        *ydst = yh;
        acc[set] += yh * yh;
      } else {
        const float y = *ydst;
        acc[2 * set] += fabsf(logf(y + kLogEps) - logf(yh + kLogEps));
        const float d = y - yh;
        acc[2 * set + 1] += d * d;
      }
    };
    if (R.band_beg[nbands] >= 16 * nbands) {
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
      for (int e = wid; e < nb * nbands; e += nw) {
        const int f = e / nbands, b = e - f * nbands;
        const float2* Zf = sm + f * bs;
        float y4[4] = {0.f, 0.f, 0.f, 0.f};
        for (int q = R.band_beg[b] + lane; q < R.band_beg[b + 1]; q += 32) {
          const int k = R.band_bin[q];
          const float wq = R.band_w[q];
          const float2 lr = Zf[pidx(k)], ms = Zf[mag_slot2(k, n)];
          y4[0] = fmaf(wq, lr.x, y4[0]);
          y4[1] = fmaf(wq, lr.y, y4[1]);
          y4[2] = fmaf(wq, ms.x, y4[2]);
          y4[3] = fmaf(wq, ms.y, y4[3]);
        }
#pragma unroll
        for (int c4 = 0; c4 < 4; ++c4)
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) y4[c4] += __shfl_xor_sync(0xffffffffu, y4[c4], o);
        if (lane < 4) band_out(f, b, lane, lane == 0 ? y4[0] : lane == 1 ? y4[1] : lane == 2 ? y4[2] : y4[3]);
      }
    } else {
      for (int e = threadIdx.x; e < nb * nbands * 4; e += blockDim.x) {
        const int f = e / (nbands * 4), r = e - f * (nbands * 4), b = r >> 2, ch = r & 3;
        const float* Zf = reinterpret_cast<const float*>(sm + f * bs);
        float yh = 0.f;
        for (int q = R.band_beg[b]; q < R.band_beg[b + 1]; ++q) {
          const int k = R.band_bin[q];
          const int slot = ch < 2 ? pidx(k) : mag_slot2(k, n);
          yh = fmaf(R.band_w[q], Zf[2 * slot + (ch & 1)], yh);
        }
        band_out(f, b, ch, yh);
      }
    }
    float out[6];
    block_sum<6>(acc, red, out);
    if (threadIdx.x == 0) {
      // partial row: the items of one (song, resolution) cover consecutive groups of R.per frames
      const int row = (t0 - S.first_frame[it.y]) / R.per;
      for (int j = 0; j < 6; ++j) S.lpart[((size_t)it.y * S.lcap + row) * 6 + j] = out[j];
    }
    return;
  }
  // ---- adjoint ----
  float* dY = reinterpret_cast<float*>(sm + kFrameBuf);   // [nb][nbands][4]
  const float* coef = S.coef + it.y * 6;                    // per set: (alpha / count, alpha / (|Y - Yh| |Y|))
  for (int e = threadIdx.x; e < nb * nbands * 4; e += blockDim.x) {
    const int f = e / (nbands * 4), r = e % (nbands * 4), b = r >> 2, ch = r & 3;
    const size_t yi = ((size_t)(t0 + f) * nbands + b) * 4 + ch;
    const float yh = Yk[yi];
    const int set = ch < 2 ? 0 : ch - 1;
    const float y = Yt[yi];
    const float dl = logf(yh + kLogEps) - logf(y + kLogEps);
    const float sg = dl > 0.f ? 1.f : (dl < 0.f ? -1.f : 0.f);
    dY[e] = coef[2 * set] * sg / (yh + kLogEps) + coef[2 * set + 1] * (yh - y);
  }
  __syncthreads();
  // bins -> packed Hermitian spectrum, in place (thread owns the pair k, n - k)
  const int half = n >> 1;
  for (int e = threadIdx.x; e < nb * (half + 1); e += blockDim.x) {
    const int f = e / (half + 1), k = e % (half + 1);
    float2* Z = sm + f * bs;
    float2 XL, XR;
    bin_spectra(Z, k, n, XL, XR);
    const float* dYf = dY + (size_t)f * nbands * 4;
    float2 gl = make_float2(0.f, 0.f), gr = gl;
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) {
      float dm = 0.f;
      for (int q = R.bin_beg[k]; q < R.bin_beg[k + 1]; ++q) dm = fmaf(R.bin_w[q], dYf[R.bin_band[q] * 4 + ch], dm);
      const float2 X = chan(ch, XL, XR);
      const float mag = sqrtf(R.aw2[k] * (X.x * X.x + X.y * X.y) + kMagEps);
      const float2 g = cscale(X, dm * R.aw2[k] / mag);
      if (ch == 0) gl = cadd(gl, g);
      else if (ch == 1) gr = cadd(gr, g);
      else if (ch == 2) { gl = cadd(gl, g); gr = cadd(gr, g); }
      else { gl = cadd(gl, g); gr = csub(gr, g); }
    }
    if (k == 0 || k == half) {
      Z[pidx(k)] = make_float2(gl.x, gr.x);
    } else {
      // G_L[k] = gl/2, G_L[n-k] = conj(gl)/2 (same for R); packed P = G_L + i G_R
      Z[pidx(k)] = make_float2(0.5f * (gl.x - gr.y), 0.5f * (gl.y + gr.x));
      Z[pidx(n - k)] = make_float2(0.5f * (gl.x + gr.y), 0.5f * (gr.x - gl.y));
    }
  }
  __syncthreads();
  // the last pass of the inverse writes the windowed frame gradients
  float2* dF = reinterpret_cast<float2*>(S.dF[it.y]) + (size_t)t0 * n;
  const float* win = R.win;
  fft_p_io<true>(sm, R.log_nfft, nb, bs, c.tab.ptw, fftp::SmemIO(),
                 [=](int f, int j, float2 v) { dF[(size_t)f * n + j] = cscale(v, win[j]); });
}

// dmix[c][s] = sum over resolutions and covering frames of dF (overlap-add, fixed order)
__global__ void __launch_bounds__(256) k_loss_gather(const SongDev* __restrict__ songs, const LossRes* __restrict__ resv,
                                                    int nres, const Item* __restrict__ items) {
  const Item it = items[blockIdx.x];
  const SongDev& S = songs[it.proc];
  const int s0 = it.idx * kElemTile;
  for (int s = s0 + threadIdx.x; s < min(s0 + kElemTile, S.L); s += blockDim.x) {
    float al = 0.f, ar = 0.f;
    for (int r = 0; r < nres; ++r) {
      const LossRes& R = resv[r];
      const int tlast = min(S.nframes[r] - 1, s / R.hop);
      int tfirst = s - R.nfft + 1 <= 0 ? 0 : (s - R.nfft + 1 + R.hop - 1) / R.hop;
      tfirst = max(tfirst, S.first_frame[r]);
      const float2* dF = reinterpret_cast<const float2*>(S.dF[r]);
      for (int t = tfirst; t <= tlast; ++t) {
        const float2 v = dF[(size_t)t * R.nfft + (s - t * R.hop)];
        al += v.x;
        ar += v.y;
      }
    }
    S.dmix[s] = al;
    S.dmix[S.ld + s] = ar;
  }
}

void launch_loss_frames(const LaunchCtx& c, const SongDev* songs, const LossRes* res, const int4* items, int n,
                        int mode, int max_dy) {
  if (!n) return;
  const size_t smem = kFrameBuf * sizeof(float2) + (mode == 2 ? (size_t)max_dy * sizeof(float) : 0);
  k_loss_frames<<<n, kLossThreads, smem, c.stream>>>(c, songs, res, items, mode);
}

void launch_loss_gather(const LaunchCtx& c, const SongDev* songs, const LossRes* res, int nres, const Item* items,
                        int n) {
  if (n) k_loss_gather<<<n, 256, 0, c.stream>>>(songs, res, nres, items);
}

void init_loss_attributes() {
  cudaFuncSetAttribute(k_loss_frames, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kFrameBuf * sizeof(float2) + kLossMaxDy * sizeof(float));
}

}  // namespace mg

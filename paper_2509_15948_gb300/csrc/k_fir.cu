// FIR synthesis of the LTI processors and the adjoints back to their parameters.
//   equalizer (Eq. 7, N = 2047): h[n] = v[n] (1/N) (e^{p_0} + 2 sum_{k>=1} e^{p_k} cos(2 pi k n / N));
//   multitap delay (Eq. 17): 39-tap zero-phase c_m (Eq. 7, N = 39) placed at the integer delays d_m, with the
//     straight-through gradient of Eq. (19) for the angular frequencies z_m (surrogate of Eq. 18);
//   reverb (Sec. 3.4): masked STFT of the fixed noise (Eqs. 9-10) -> inverse STFT by overlap-add.
#include "mg_fft.cuh"

namespace mg {

namespace {

__device__ __forceinline__ float softplusf_(float x) { return x > 20.f ? x : log1pf(expf(x)); }

}  // namespace

// ------------------------------------------------------------------------------------------------
// equalizer
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_eq_fir(LaunchCtx c, const int* __restrict__ procs) {
  __shared__ float ep[kEqParams];
  __shared__ float cs[kEqTaps];
  const ProcDev& P = c.procs[procs[blockIdx.x]];
  for (int k = threadIdx.x; k < kEqParams; k += blockDim.x) ep[k] = expf(P.p[k]);
  for (int m = threadIdx.x; m < kEqTaps; m += blockDim.x) cs[m] = c.tab.cos_eq[m];
  __syncthreads();
  for (int j = threadIdx.x; j < kEqTaps; j += blockDim.x) {
    const int an = abs(j - kEqHalf);
    float acc = 0.f;
    int idx = 0;
    for (int k = 1; k < kEqParams; ++k) {
      idx += an;
      if (idx >= kEqTaps) idx -= kEqTaps;
      acc = fmaf(ep[k], cs[idx], acc);
    }
    P.taps[j] = c.tab.hann_eq[j] * (ep[0] + 2.f * acc) * (1.f / kEqTaps);
  }
}

// dL/dp_k = e^{p_k} (c_k / N) sum_n dh[n] v[n] cos(2 pi k n / N), c_0 = 1, c_k = 2; dh = dh_l + dh_r.
__global__ void __launch_bounds__(256) k_eq_fir_adj(LaunchCtx c, const int* __restrict__ procs) {
  __shared__ float e[kEqParams];
  __shared__ float cs[kEqTaps];
  const ProcDev& P = c.procs[procs[blockIdx.x]];
  for (int m = threadIdx.x; m < kEqTaps; m += blockDim.x) cs[m] = c.tab.cos_eq[m];
  for (int m = threadIdx.x; m <= kEqHalf; m += blockDim.x) {
    const int jp = kEqHalf + m, jm = kEqHalf - m;
    const float dp = (P.dtaps[jp] + P.dtaps[P.Nh + jp]) * c.tab.hann_eq[jp];
    const float dm = (P.dtaps[jm] + P.dtaps[P.Nh + jm]) * c.tab.hann_eq[jm];
    e[m] = m == 0 ? dp : dp + dm;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < kEqParams; k += blockDim.x) {
    float acc = e[0];
    int idx = 0;
    for (int m = 1; m <= kEqHalf; ++m) {
      idx += k;
      if (idx >= kEqTaps) idx -= kEqTaps;
      acc = fmaf(e[m], cs[idx], acc);
    }
    P.gp[k] = expf(P.p[k]) * (k == 0 ? 1.f : 2.f) * (1.f / kEqTaps) * acc;
  }
}

// ------------------------------------------------------------------------------------------------
// multitap delay
// ------------------------------------------------------------------------------------------------
// aux layout: [2][20][39] c_m taps, then [2][20] integer delays (stored as int).
constexpr int kDlyAuxC = 2 * kDlyTaps * kDlyFir;

__device__ __forceinline__ int dly_slot(double fs) { return (int)llrint(0.1 * fs); }

__global__ void __launch_bounds__(256) k_dly_prep(LaunchCtx c, const int* __restrict__ procs) {
  const ProcDev& P = c.procs[procs[blockIdx.x]];
  const int D = dly_slot(c.fs);
  int* dpos = reinterpret_cast<int*>(P.aux + kDlyAuxC);
  for (int e = threadIdx.x; e < kDlyAuxC; e += blockDim.x) {
    const int ch = e / (kDlyTaps * kDlyFir), m = (e / kDlyFir) % kDlyTaps, jj = e % kDlyFir;
    const float* lm = P.p + (ch * kDlyTaps + m) * kDlyPer + 2;
    const int an = abs(jj - kDlyHalf);
    float acc = 0.f;
    int idx = 0;
    for (int k = 1; k <= kDlyHalf; ++k) {
      idx += an;
      if (idx >= kDlyFir) idx -= kDlyFir;
      acc = fmaf(expf(lm[k]), c.tab.cos_dl[idx], acc);
    }
    P.aux[e] = c.tab.hann_dl[jj] * (expf(lm[0]) + 2.f * acc) * (1.f / kDlyFir);
  }
  for (int e = threadIdx.x; e < 2 * kDlyTaps; e += blockDim.x) {
    const int ch = e / kDlyTaps, m = e % kDlyTaps;
    const float* z = P.p + (ch * kDlyTaps + m) * kDlyPer;
    // decided in double precision: z = exp(-j 2 pi d / D) is the impulse at d (Eq. 18, w_D = exp(+j 2 pi / D))
    const double ang = atan2((double)z[1], (double)z[0]);
    const double twopi = 2.0 * 3.14159265358979323846;
    double ph = fmod(-ang, twopi);
    if (ph < 0.0) ph += twopi;
    long long off = llrint((double)D * ph / twopi) % D;
    dpos[e] = m * D + (int)off;
  }
}

__global__ void __launch_bounds__(256) k_dly_fir(LaunchCtx c, const Item* __restrict__ items) {
  __shared__ int dpos[2 * kDlyTaps];
  const Item it = items[blockIdx.x];
  const ProcDev& P = c.procs[it.proc];
  const int* dp = reinterpret_cast<const int*>(P.aux + kDlyAuxC);
  if (threadIdx.x < 2 * kDlyTaps) dpos[threadIdx.x] = dp[threadIdx.x];
  __syncthreads();
  const int j = it.idx * blockDim.x + threadIdx.x;
  if (j >= P.Nh) return;
  const int n = j + P.n0;
  for (int ch = 0; ch < 2; ++ch) {
    float acc = 0.f;
    for (int m = 0; m < kDlyTaps; ++m) {
      const int o = n - dpos[ch * kDlyTaps + m];
      if (o >= -kDlyHalf && o <= kDlyHalf) acc += P.aux[(ch * kDlyTaps + m) * kDlyFir + o + kDlyHalf];
    }
    P.taps[ch * P.Nh + j] = acc;
  }
}

// One CTA per (node, channel, tap m): exact gradient of the 20 log-magnitudes of c_m, and the Eq. (19)
// update direction of z_m: sgn(g) + gamma (|z| - 1) z/|z| with
//   g = sum_q G[q] conj(s'_q(z_hat)),  G[q] = sum_j dL/dh[m D + q + j] c_m[j],
//   s'_q(z) = (1/D) [w^q (1 - z^D) - D z^{D-1} (1 - z w^q)] / (1 - z w^q)^2   (derivative of Eq. 18),
// z_hat = z / max(1, |z|).  Near a pole (|1 - z w^q| < 1e-3) the series sum_k k a^{k-1} is summed directly.
__global__ void __launch_bounds__(256) k_dly_adj(LaunchCtx c, const Item* __restrict__ items) {
  __shared__ float cm[kDlyFir];
  __shared__ float dc[kDlyFir];
  __shared__ float red[2 * 32];
  __shared__ float gsum[2];
  __shared__ float2 zsh[3];   // z^D, z^(D-1), z clamped to the unit disk
  const Item it = items[blockIdx.x];
  const ProcDev& P = c.procs[it.proc];
  const int ch = it.idx / kDlyTaps, m = it.idx % kDlyTaps;
  const int D = dly_slot(c.fs);
  const int* dpos = reinterpret_cast<const int*>(P.aux + kDlyAuxC);
  const int d = dpos[ch * kDlyTaps + m];
  const float* dh = P.dtaps + (size_t)ch * P.Nh;
  const float* pz = P.p + (ch * kDlyTaps + m) * kDlyPer;
  float* gz = P.gp + (ch * kDlyTaps + m) * kDlyPer;
  if (threadIdx.x < kDlyFir) {
    cm[threadIdx.x] = P.aux[(ch * kDlyTaps + m) * kDlyFir + threadIdx.x];
    dc[threadIdx.x] = dh[d + threadIdx.x];   // tap time d + j - 19 -> index d + j (first tap at -19)
  }
  // (b, scalars) the powers of z in double, once per block (FP64 is slow; every thread used to repeat them)
  if (threadIdx.x == 0) {
    const double zr = pz[0], zi = pz[1];
    const double rz = sqrt(zr * zr + zi * zi);
    const double sc = rz > 1.0 ? 1.0 / rz : 1.0;
    const double hr = zr * sc, hi = zi * sc, hrad = rz * sc;
    const double th = atan2(hi, hr);
    double sD, cD, sD1, cD1;
    sincos((double)D * th, &sD, &cD);
    sincos((double)(D - 1) * th, &sD1, &cD1);
    const double pD = hrad > 0.0 ? pow(hrad, (double)D) : 0.0;
    const double pD1 = hrad > 0.0 ? pow(hrad, (double)(D - 1)) : 0.0;
    zsh[0] = make_float2((float)(pD * cD), (float)(pD * sD));
    zsh[1] = make_float2((float)(pD1 * cD1), (float)(pD1 * sD1));
    zsh[2] = make_float2((float)hr, (float)hi);
  }
  __syncthreads();
  // (a) log-magnitudes of c_m
  if (threadIdx.x <= kDlyHalf) {
    const int k = threadIdx.x;
    float acc = 0.f;
    for (int jj = 0; jj < kDlyFir; ++jj) {
      const int idx = (k * abs(jj - kDlyHalf)) % kDlyFir;
      acc = fmaf(dc[jj] * c.tab.hann_dl[jj], c.tab.cos_dl[idx], acc);
    }
    gz[2 + k] = expf(pz[2 + k]) * (k == 0 ? 1.f : 2.f) * (1.f / kDlyFir) * acc;
  }
  // (b) angular frequency
  const float2 zD1 = zsh[1], zh = zsh[2];
  const float2 omz = make_float2(1.f - zsh[0].x, -zsh[0].y);
  double accd[2] = {0.0, 0.0};
  for (int q = threadIdx.x; q < D; q += blockDim.x) {
    float G = 0.f;
    const float* seg = dh + (size_t)m * D + q;
#pragma unroll 13
    for (int jj = 0; jj < kDlyFir; ++jj) G = fmaf(seg[jj], cm[jj], G);
    const float2 wq = c.tab.dly_w[q];
    const float2 a = cmul(zh, wq);
    const float2 oma = make_float2(1.f - a.x, -a.y);
    float2 sp;
    if (oma.x * oma.x + oma.y * oma.y > 1e-6f) {
      const float2 num = csub(cmul(wq, omz), cscale(cmul(zD1, oma), (float)D));
      const float2 den = cmul(oma, oma);
      const float dd = den.x * den.x + den.y * den.y;
      sp = cscale(cmulc(num, den), 1.f / ((float)D * dd));
    } else {  // direct sum near the pole
      double fr = 0.0, fi = 0.0;
      const double ar = a.x, ai = a.y;
      for (int k = D - 1; k >= 1; --k) {   // Horner: f = sum_{k=1}^{D-1} k a^{k-1}
        const double nr = fr * ar - fi * ai + (double)k;
        fi = fr * ai + fi * ar;
        fr = nr;
      }
      const float2 f = make_float2((float)fr, (float)fi);
      sp = cscale(cmul(wq, f), 1.f / (float)D);
    }
    accd[0] += (double)G * sp.x;   // g = sum G conj(s'), accumulated in double (|g| can be far below sum |G s'|)
    accd[1] -= (double)G * sp.y;
  }
  float acc[2] = {0.f, 0.f};
  {
    // block reduction in double: per-warp shuffles, then one warp over the warp totals
    __shared__ double dred[2][32];
    double a0 = accd[0], a1 = accd[1];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a0 += __shfl_down_sync(0xffffffffu, a0, o);
      a1 += __shfl_down_sync(0xffffffffu, a1, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) { dred[0][wid] = a0; dred[1][wid] = a1; }
    __syncthreads();
    if (wid == 0) {
      a0 = lane < nw ? dred[0][lane] : 0.0;
      a1 = lane < nw ? dred[1][lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_down_sync(0xffffffffu, a0, o);
        a1 += __shfl_down_sync(0xffffffffu, a1, o);
      }
      if (lane == 0) { gsum[0] = (float)a0; gsum[1] = (float)a1; }
    }
    __syncthreads();
    (void)acc;
    (void)red;
  }
  if (threadIdx.x == 0) {
    const double zr = pz[0], zi = pz[1];
    const double rz = sqrt(zr * zr + zi * zi);
    const float gr = gsum[0], gi = gsum[1];
    const float gm = sqrtf(gr * gr + gi * gi);
    float outr = 0.f, outi = 0.f;
    if (gm > 0.f) {
      outr = gr / gm;
      outi = gi / gm;
    }
    const float rzf = (float)rz;
    if (rzf > 0.f) {
      const float k = 0.01f * (rzf - 1.f) / rzf;   // gamma (|z| - 1) z / |z|
      outr += k * (float)zr;
      outi += k * (float)zi;
    }
    gz[0] = outr;
    gz[1] = outi;
  }
}

// ------------------------------------------------------------------------------------------------
// reverb
// ------------------------------------------------------------------------------------------------
// 384-point DFTs of the reverb (Sec. 3.4) as 3 x 128 mixed radix in shared memory.  A frame block holds
// nf frames of 384 complex values; the mid and side signals travel packed as one complex signal.
//   inverse: x[128 j1 + j2] = sum_{k1} w3^{j1 k1} w384^{j2 k1} [sum_{k2} X[k1 + 3 k2] w128^{j2 k2}]
//   forward: F[k2 + 128 k1] = sum_{j1} w3^{-j1 k1} w384^{-j1 k2} [sum_{j2} d[j1 + 3 j2] w128^{-j2 k2}]
// Both expect the input permuted to slot f*384 + 128 r + s for index r + 3 s and leave the output in natural
// order (slot f*384 + k).
template <bool INV>
__device__ void dft384_block(float2* sm, int nf, const float2* __restrict__ tw, const float2* __restrict__ cs384) {
  fft_smem<INV, 4>(sm, 7, nf * 3, 1, 128, tw);
  const float c3 = -0.5f, s3 = INV ? 0.86602540378443864676f : -0.86602540378443864676f;  // w3 = e^{+-2 pi i/3}
  for (int e = threadIdx.x; e < nf * 128; e += blockDim.x) {
    const int f = e >> 7, q = e & 127;
    float2* base = sm + f * kRevFft;
    float2 a0 = base[q], a1 = base[128 + q], a2 = base[256 + q];
    float2 w1 = cs384[q], w2 = cs384[(2 * q) % kRevFft];       // (cos, sin)(2 pi m / 384)
    if (!INV) { w1.y = -w1.y; w2.y = -w2.y; }
    a1 = cmul(a1, w1);
    a2 = cmul(a2, w2);
    const float2 s12 = cadd(a1, a2), d12 = csub(a1, a2);
    const float2 t = make_float2(a0.x + c3 * s12.x, a0.y + c3 * s12.y);
    const float2 r = make_float2(-s3 * d12.y, s3 * d12.x);    // i s3 (a1 - a2)
    base[q] = cadd(a0, s12);
    base[128 + q] = cadd(t, r);
    base[256 + q] = csub(t, r);
  }
  __syncthreads();
}

__device__ __forceinline__ int perm384(int k) { return (k % 3) * 128 + k / 3; }

// STFT of the fixed noises (periodic Hann 384, hop 192, no centre padding), mid and side packed:
// item = (node, frame group of 16).
__global__ void __launch_bounds__(512) k_rev_noise_stft(LaunchCtx c, const Item* __restrict__ items,
                                                       const float* __restrict__ noise_all, int noise_len) {
  extern __shared__ float2 sm[];
  const Item it = items[blockIdx.x];
  const ProcDev& P = c.procs[it.proc];
  const int F = P.nframes, t0 = it.idx * kRevFG, nf = min(kRevFG, F - t0);
  const float* nm = noise_all + ((size_t)P.rev * 2 + 0) * noise_len;
  const float* ns = noise_all + ((size_t)P.rev * 2 + 1) * noise_len;
  for (int e = threadIdx.x; e < nf * kRevFft; e += blockDim.x) {
    const int f = e / kRevFft, j = e % kRevFft, s = (t0 + f) * kRevHop + j;
    const float w = c.tab.rev_win[j];
    sm[f * kRevFft + perm384(j)] = make_float2(nm[s] * w, ns[s] * w);
  }
  __syncthreads();
  dft384_block<false>(sm, nf, c.tab.tw, c.tab.rev_cs);
  float2* out = const_cast<float2*>(P.nspec);
  for (int e = threadIdx.x; e < nf * kRevBins; e += blockDim.x) {
    const int f = e / kRevBins, k = e % kRevBins;
    const float2 a = sm[f * kRevFft + k], b = sm[f * kRevFft + ((kRevFft - k) % kRevFft)];
    const float2 xm = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
    const float2 d = make_float2(a.x - b.x, a.y + b.y);
    const float2 xs = make_float2(0.5f * d.y, -0.5f * d.x);
    out[((size_t)0 * F + t0 + f) * kRevBins + k] = xm;
    out[((size_t)1 * F + t0 + f) * kRevBins + k] = xs;
  }
}

__device__ __forceinline__ float rev_env(int n, int F, const float* win) {
  // sum over covering frames of the squared window
  float e = 0.f;
  const int a = n / kRevHop;
#pragma unroll
  for (int t = a - 1; t <= a; ++t) {
    if (t < 0 || t >= F) continue;
    const int jj = n - t * kRevHop;
    if (jj < 0 || jj >= kRevFft) continue;
    const float w = win[jj];
    e += w * w;
  }
  return e;
}

// item = (node, grp): output samples [192 t0, 192 (t0 + 16)) of h_m and h_s (frames t0-1 .. t0+15).
// Per frame: H_x[k] = U_x[k] exp(H0_x[k] + t H_delta_x[k]) (Eq. 10), Hermitian extension (real parts at
// DC and Nyquist), packed X = H_m + i H_s, inverse DFT (frames of h_m and h_s in the real / imaginary part),
// window, overlap-add, normalisation by the summed squared window.
__global__ void __launch_bounds__(512) k_rev_fir(LaunchCtx c, const Item* __restrict__ items) {
  extern __shared__ float2 sm[];
  const Item it = items[blockIdx.x];
  const ProcDev& P = c.procs[it.proc];
  const int F = P.nframes, ng = (F + kRevFG - 1) / kRevFG;
  const int grp = it.idx, t0 = grp * kRevFG, tb = t0 - 1;
  constexpr int NF = kRevFG + 1;
  for (int e = threadIdx.x; e < NF * kRevBins; e += blockDim.x) {
    const int f = e / kRevBins, k = e % kRevBins, t = tb + f;
    float2 hm = make_float2(0.f, 0.f), hs = hm;
    if (t >= 0 && t < F) {
      const int kk = k < kRevParams ? k : kRevParams - 1;
      const float* pm = P.p;                          // [x][H0, p_delta][192]
      const float* ps = P.p + 2 * kRevParams;
      const float mm = expf(pm[kk] + (float)t * (-0.05f * softplusf_(pm[kRevParams + kk])));
      const float ms = expf(ps[kk] + (float)t * (-0.05f * softplusf_(ps[kRevParams + kk])));
      hm = cscale(P.nspec[((size_t)0 * F + t) * kRevBins + k], mm);
      hs = cscale(P.nspec[((size_t)1 * F + t) * kRevBins + k], ms);
    }
    if (k == 0 || k == kRevBins - 1) { hm.y = 0.f; hs.y = 0.f; }
    float2* base = sm + f * kRevFft;
    // X[k] = Hm[k] + i Hs[k]; X[384-k] = conj(Hm[k]) + i conj(Hs[k])
    base[perm384(k)] = make_float2(hm.x - hs.y, hm.y + hs.x);
    if (k > 0 && k < kRevBins - 1) base[perm384(kRevFft - k)] = make_float2(hm.x + hs.y, hs.x - hm.y);
  }
  __syncthreads();
  dft384_block<true>(sm, NF, c.tab.tw, c.tab.rev_cs);
  const int nbeg = t0 * kRevHop, nend = grp == ng - 1 ? P.Nh : min((t0 + kRevFG) * kRevHop, P.Nh);
  for (int n = nbeg + threadIdx.x; n < nend; n += blockDim.x) {
    const int a = n / kRevHop;
    float am = 0.f, as = 0.f, env = 0.f;
    for (int t = a - 1; t <= a; ++t) {
      if (t < 0 || t >= F || t < tb || t > tb + NF - 1) continue;
      const int jj = n - t * kRevHop;
      const float2 v = sm[(t - tb) * kRevFft + jj];
      const float w = c.tab.rev_win[jj];
      am += w * v.x;
      as += w * v.y;
      env += w * w;
    }
    const float inv = env > 1e-11f ? 1.f / (env * (float)kRevFft) : 0.f;
    P.taps[n] = am * inv;
    P.taps[(size_t)P.Nh + n] = as * inv;
  }
}

// item = (node, grp): frames t in [t0, t0 + 16); partial sums of dL/dH0 and dL/dp_delta per bin, for mid and
// side.  dframe_x[j] = w[j] dh_x[192 t + j] / env (dh_m = dh_l + dh_r, dh_s = dh_l - dh_r), packed forward DFT,
// dRe H[k] = c_k Re F[k] / 384, dIm H[k] = c_k Im F[k] / 384 (c_k = 1 at DC / Nyquist where Im is unused).
__global__ void __launch_bounds__(512) k_rev_adj(LaunchCtx c, const Item* __restrict__ items) {
  extern __shared__ float2 sm[];
  const Item it = items[blockIdx.x];
  const ProcDev& P = c.procs[it.proc];
  const int F = P.nframes, ng = (F + kRevFG - 1) / kRevFG;
  const int grp = it.idx, t0 = grp * kRevFG;
  const int nf = min(kRevFG, F - t0);
  for (int e = threadIdx.x; e < nf * kRevFft; e += blockDim.x) {
    const int f = e / kRevFft, jj = e % kRevFft, n = (t0 + f) * kRevHop + jj;
    float2 v = make_float2(0.f, 0.f);
    if (n < P.Nh) {
      const float env = rev_env(n, F, c.tab.rev_win);
      if (env > 1e-11f) {
        const float sc = c.tab.rev_win[jj] / env;
        const float dl = P.dtaps[n], dr = P.dtaps[(size_t)P.Nh + n];
        v = make_float2(sc * (dl + dr), sc * (dl - dr));
      }
    }
    sm[f * kRevFft + perm384(jj)] = v;
  }
  __syncthreads();
  dft384_block<false>(sm, nf, c.tab.tw, c.tab.rev_cs);
  for (int e = threadIdx.x; e < 2 * kRevBins; e += blockDim.x) {
    const int x = e / kRevBins, k = e % kRevBins;
    const int kk = k < kRevParams ? k : kRevParams - 1;
    const float* h0 = P.p + x * 2 * kRevParams;
    const float* pd = h0 + kRevParams;
    const float hd = -0.05f * softplusf_(pd[kk]);
    const float dhd = -0.05f / (1.f + expf(-pd[kk]));    // d H_delta / d p_delta
    const float ck = (k == 0 || k == kRevBins - 1) ? 1.f : 2.f;
    float a0 = 0.f, a1 = 0.f;
    for (int f = 0; f < nf; ++f) {
      const float2 A = sm[f * kRevFft + k], B = sm[f * kRevFft + ((kRevFft - k) % kRevFft)];
      float2 Fx;
      if (x == 0) {
        Fx = make_float2(0.5f * (A.x + B.x), 0.5f * (A.y - B.y));
      } else {
        const float2 d = make_float2(A.x - B.x, A.y + B.y);
        Fx = make_float2(0.5f * d.y, -0.5f * d.x);
      }
      const float dRe = ck * Fx.x * (1.f / kRevFft);
      const float dIm = (k == 0 || k == kRevBins - 1) ? 0.f : ck * Fx.y * (1.f / kRevFft);
      const int t = t0 + f;
      const float2 U = P.nspec[((size_t)x * F + t) * kRevBins + k];
      const float M = expf(h0[kk] + (float)t * hd);
      const float dM = dRe * U.x + dIm * U.y;
      a0 += dM * M;
      a1 += dM * M * (float)t * dhd;
    }
    float* part = P.aux + ((size_t)x * ng + grp) * kRevBins * 2;
    part[k * 2 + 0] = a0;
    part[k * 2 + 1] = a1;
  }
}

__global__ void __launch_bounds__(256) k_rev_adj_fin(LaunchCtx c, const int* __restrict__ procs) {
  const ProcDev& P = c.procs[procs[blockIdx.x]];
  const int ng = (P.nframes + kRevFG - 1) / kRevFG;
  for (int e = threadIdx.x; e < 2 * kRevParams; e += blockDim.x) {
    const int x = e / kRevParams, k = e % kRevParams;
    float a0 = 0.f, a1 = 0.f;
    for (int g = 0; g < ng; ++g) {
      const float* part = P.aux + ((size_t)x * ng + g) * kRevBins * 2;
      a0 += part[k * 2];
      a1 += part[k * 2 + 1];
      if (k == kRevParams - 1) {   // the Nyquist bin reuses parameter 191
        a0 += part[(kRevBins - 1) * 2];
        a1 += part[(kRevBins - 1) * 2 + 1];
      }
    }
    P.gp[x * 2 * kRevParams + k] = a0;
    P.gp[x * 2 * kRevParams + kRevParams + k] = a1;
  }
}

void launch_eq_fir(const LaunchCtx& c, const int* procs, int n) {
  if (n) k_eq_fir<<<n, 256, 0, c.stream>>>(c, procs);
}
void launch_eq_fir_adj(const LaunchCtx& c, const int* procs, int n) {
  if (n) k_eq_fir_adj<<<n, 256, 0, c.stream>>>(c, procs);
}
void launch_dly_prep(const LaunchCtx& c, const int* procs, int n) {
  if (n) k_dly_prep<<<n, 256, 0, c.stream>>>(c, procs);
}
void launch_dly_fir(const LaunchCtx& c, const Item* items, int n) {
  if (n) k_dly_fir<<<n, 256, 0, c.stream>>>(c, items);
}
void launch_dly_adj(const LaunchCtx& c, const Item* items, int n) {
  if (n) k_dly_adj<<<n, 256, 0, c.stream>>>(c, items);
}
void launch_rev_fir(const LaunchCtx& c, const Item* items, int n) {
  if (n) k_rev_fir<<<n, 512, (kRevFG + 1) * kRevFft * sizeof(float2), c.stream>>>(c, items);
}
void launch_rev_adj(const LaunchCtx& c, const Item* items, int n) {
  if (n) k_rev_adj<<<n, 512, kRevFG * kRevFft * sizeof(float2), c.stream>>>(c, items);
}
void init_fir_attributes() {
  cudaFuncSetAttribute(k_rev_fir, cudaFuncAttributeMaxDynamicSharedMemorySize, (kRevFG + 1) * kRevFft * (int)sizeof(float2));
  cudaFuncSetAttribute(k_rev_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, kRevFG * kRevFft * (int)sizeof(float2));
  cudaFuncSetAttribute(k_rev_noise_stft, cudaFuncAttributeMaxDynamicSharedMemorySize, kRevFG * kRevFft * (int)sizeof(float2));
}
void launch_rev_adj_fin(const LaunchCtx& c, const int* procs, int n) {
  if (n) k_rev_adj_fin<<<n, 256, 0, c.stream>>>(c, procs);
}
void launch_rev_noise_stft(const LaunchCtx& c, const Item* items, int n, const float* noise, int noise_len) {
  if (n) k_rev_noise_stft<<<n, 512, kRevFG * kRevFft * sizeof(float2), c.stream>>>(c, items, noise, noise_len);
}

}  // namespace mg

// Equalizer (Sec. 3.3, Eqs. 7-8) by single-pass overlap-save in shared memory.
// The 2047-tap zero-phase FIR is short against an 8192-point FFT, so every block of B = 6146 output samples is
// computed by one CTA from its input segment [s0 - 1023, s0 + B + 1023) without any global FFT scratch:
//   forward:  segment -> FFT -> x H -> IFFT -> B valid outputs, fused with the dry/wet blend and the L_g
//             energies; the wet signal y_bar is kept for the backward;
//   backward: a work item walks kEqChunk consecutive blocks.  Per block: D = FFT(dL/dy_bar on the segment)
//             with dL/dy_bar = w dy + c1 y_bar_mid from the kept y_bar, Ub = FFT(u on the block only); D H is
//             stored, and a second kernel forms du = IFFT(D H) on the block (h is even, so the correlation
//             adjoint is the same convolution).
//             dL/dh[j] = sum_n dL/dy_bar[n] u[n - j] = sum_m u[m] dL/dy_bar[m + j] is split over the blocks by the
//             input position m: a block contributes IFFT(D conj(Ub)) at lags |j| <= 1023 (m + j stays inside the
//             segment, no wrap-around), so the segment spectrum D serves both gradients.  D conj(Ub) is summed
//             over the item's blocks in the item's own row of a global buffer; a per-node kernel adds the items'
//             spectra in a fixed order and runs one inverse FFT whose real part at lags -1023..1023 is dL/dh
//             summed over both channels.
// H is real (h real and even); both channels travel packed as one complex signal.
#include "mg_fftp.cuh"

namespace mg {

namespace {
constexpr int kOsLog = 13;
constexpr int kOsM = 1 << kOsLog;
constexpr int kOsThreads = 512;
constexpr int kOsBwdThreads = 1024;
constexpr int kOsP = pstride(kOsM);   // padded buffer stride
}  // namespace

// Spectrum of the FIR on the 8192-point grid: one CTA per node.
__global__ void __launch_bounds__(kOsThreads) k_eq_spec(LaunchCtx c, const int* __restrict__ procs) {
  extern __shared__ float2 sm[];
  const ProcDev& P = c.procs[procs[blockIdx.x]];
  for (int j = threadIdx.x; j < kOsM; j += blockDim.x) {
    // tap time n = j for j < 1024, n = j - M for j > M - 1024 (circular placement of n in [-1023, 1023])
    int n = j < kOsM / 2 ? j : j - kOsM;
    float v = 0.f;
    if (n >= -kEqHalf && n <= kEqHalf) v = P.taps[n + kEqHalf];
    sm[pidx(j)] = make_float2(v, 0.f);
  }
  __syncthreads();
  fft_p<false>(sm, kOsLog, 1, kOsP, c.tab.ptw);
  for (int k = threadIdx.x; k < kOsM; k += blockDim.x) P.hspec[k] = sm[pidx(k)].x;
}

// item = (node, block): outputs [s0, s0 + 6146).
__global__ void __launch_bounds__(kOsThreads, 2) k_eq_os_fwd(LaunchCtx c, const Item* __restrict__ items) {
  extern __shared__ float2 sm[];
  __shared__ float red[2 * 32];
  const Item it = items[blockIdx.x];
  const ProcDev& P = c.procs[it.proc];
  constexpr int B = kOsM - 2 * kEqHalf;
  const int s0 = it.idx * B, seg = s0 - kEqHalf, L = P.L, ld = P.ld;
  const float* u = P.u;
  // the segment goes straight from global memory into the first pass of the transform
  fft_p_io<false>(sm, kOsLog, 1, kOsP, c.tab.ptw, [=](int, int j) {
    const int s = seg + j;
    return (s >= 0 && s < L) ? make_float2(u[s], u[ld + s]) : make_float2(0.f, 0.f);
  });
  for (int k = threadIdx.x; k < kOsM; k += blockDim.x) sm[pidx(k)] = cscale(sm[pidx(k)], P.hspec[k]);
  __syncthreads();
  const float w = dry_wet_w(c, P.qidx), wd = dry_wet_d(c, P.qidx);
  const float inv = 1.f / kOsM;
  float acc[2] = {0.f, 0.f};
  float* ybar = P.ybar;
  float* y = P.y;
  // the last pass of the inverse writes the B valid outputs, blended with the dry signal
  fft_p_io<true>(sm, kOsLog, 1, kOsP, c.tab.ptw, fftp::SmemIO(), [&](int, int j, float2 v) {
    const int t = j - kEqHalf, s = s0 + t;
    if (t < 0 || t >= B || s >= L) return;
    const float2 yb = cscale(v, inv);
    ybar[s] = yb.x;
    ybar[ld + s] = yb.y;
    const float ul = u[s], ur = u[ld + s];
    y[s] = w * yb.x + wd * ul;
    y[ld + s] = w * yb.y + wd * ur;
    const float ym = yb.x + yb.y, um = ul + ur;
    acc[0] += ym * ym;
    acc[1] += um * um;
  });
  float out[2];
  block_sum<2>(acc, red, out);
  if (threadIdx.x == 0) {
    P.fpart[it.idx * kNPart + 0] = out[0];
    P.fpart[it.idx * kNPart + 1] = out[1];
  }
}

// item = (node, chunk): blocks chunk * kEqChunk ... of B = 6146 samples.  Two padded 8192-point buffers in
// shared memory and 1024 threads; both forward transforms run as one batch, 16 elements per thread.  Per block
// the spectrum D H is stored for k_eq_os_du; the running sum of the correlation spectra stays in a third,
// unpadded 8192-entry buffer (each thread owns the same bins in every block, so the read-modify-write is
// race-free and ordered) and goes to the item's row of dhspec once (205 KB of shared memory, one CTA per SM).  The inverse transform lives in its own kernel: in this loop, next to the forward
// transforms, its index arithmetic would be hoisted into registers that spill.
__global__ void __launch_bounds__(kOsBwdThreads, 1) k_eq_os_bwd(LaunchCtx c, const Item* __restrict__ items) {
  extern __shared__ float2 sm[];
  __shared__ float red[32];
  float2* D = sm;                 // dL/dy_bar on the segment, then its spectrum
  float2* Ub = sm + kOsP;         // u on the block only, then its spectrum
  float2* acc = sm + 2 * kOsP;    // running sum of the item's correlation spectra, written to dhspec at the end
  const Item it = items[blockIdx.x];
  const ProcDev& P = c.procs[it.proc];
  constexpr int B = kOsM - 2 * kEqHalf;   // 6146
  constexpr int kBins = kOsM / kOsBwdThreads;
  float2* dst = P.dhspec + (size_t)it.idx * kOsM;
  const float w = dry_wet_w(c, P.qidx);
  const float c1 = P.stats[2];
  float dwacc[1] = {0.f};
  const int nblk = (P.L + B - 1) / B;
  const int b0 = it.idx * kEqChunk, b1 = min(nblk, b0 + kEqChunk);
  const int L = P.L, ld = P.ld;
  const float *u = P.u, *ybar = P.ybar, *dy = P.dy;
  for (int blk = b0; blk < b1; ++blk) {
    const int seg = blk * B - kEqHalf;
    // D and Ub as one batch of two, their inputs formed in the first pass: batch 0 is dL/dy_bar on the segment
    // (which also accumulates the block's dL/dw), batch 1 the input on the block only
    fft_p_io<false>(D, kOsLog, 2, kOsP, c.tab.ptw, [&](int bt, int j) {
      const int s = seg + j;
      const bool in_blk = j >= kEqHalf && j < kEqHalf + B;
      if (s < 0 || s >= L || (bt && !in_blk)) return make_float2(0.f, 0.f);
      if (bt) return make_float2(u[s], u[ld + s]);
      const float yl = ybar[s], yr = ybar[ld + s];
      const float gl = dy[s], gr = dy[ld + s];
      const float gm = c1 * (yl + yr);
      if (in_blk) dwacc[0] += gl * (yl - u[s]) + gr * (yr - u[ld + s]);
      return make_float2(w * gl + gm, w * gr + gm);
    });
    float2* g = P.eqg + (size_t)blk * kOsM;
#pragma unroll 4
    for (int t = 0; t < kBins; ++t) {
      const int k = threadIdx.x + t * kOsBwdThreads, e = pidx(k);
      const float2 dk = D[e];
      const float2 prod = cmulc(dk, Ub[e]);
      acc[k] = blk == b0 ? prod : cadd(acc[k], prod);
      g[k] = cscale(dk, P.hspec[k]);
    }
    __syncthreads();   // the next block overwrites the buffers
  }
  // each thread writes the bins it accumulated (no barrier needed)
#pragma unroll 4
  for (int t = 0; t < kBins; ++t) {
    const int k = threadIdx.x + t * kOsBwdThreads;
    dst[k] = acc[k];
  }
  float out[1];
  block_sum<1>(dwacc, red, out);
  if (threadIdx.x == 0) P.bpart[it.idx * kNPart] = out[0];
}

// item = (node, block): du on [s0, s0 + 6146) = IFFT(D H) on the block (h even: the adjoint of the
// convolution is the same convolution) plus the dry path and the loudness-gain term.
__global__ void __launch_bounds__(kOsThreads, 2) k_eq_os_du(LaunchCtx c, const Item* __restrict__ items) {
  extern __shared__ float2 sm[];
  const Item it = items[blockIdx.x];
  const ProcDev& P = c.procs[it.proc];
  constexpr int B = kOsM - 2 * kEqHalf;
  const int s0 = it.idx * B;
  const float2* g = P.eqg + (size_t)it.idx * kOsM;
#pragma unroll 4
  for (int k = threadIdx.x; k < kOsM; k += blockDim.x) sm[pidx(k)] = g[k];
  __syncthreads();
  fft_p<true>(sm, kOsLog, 1, kOsP, c.tab.ptw);
  const float wd = dry_wet_d(c, P.qidx), c2 = P.stats[3];
  const float inv = 1.f / kOsM;
  for (int t = threadIdx.x; t < B; t += blockDim.x) {
    const int s = s0 + t;
    if (s >= P.L) break;
    const float2 dw = cscale(sm[pidx(kEqHalf + t)], inv);
    const float um = c2 * (P.u[s] + P.u[P.ld + s]);
    P.du[s] = wd * P.dy[s] + dw.x + um;
    P.du[P.ld + s] = wd * P.dy[P.ld + s] + dw.y + um;
  }
}

// dL/dh (both channels summed into row 0, row 1 zero): the items' correlation spectra added in a fixed
// order, one inverse FFT, lags n = -1023..1023 at circular positions n mod 8192.
__global__ void __launch_bounds__(kOsThreads) k_eq_dh_reduce(LaunchCtx c, const int* __restrict__ procs) {
  extern __shared__ float2 sm[];
  const ProcDev& P = c.procs[procs[blockIdx.x]];
  for (int k = threadIdx.x; k < kOsM; k += blockDim.x) {
    float2 s = make_float2(0.f, 0.f);
    for (int b = 0; b < P.nbpart; ++b) s = cadd(s, P.dhspec[(size_t)b * kOsM + k]);
    sm[pidx(k)] = s;
  }
  __syncthreads();
  fft_p<true>(sm, kOsLog, 1, kOsP, c.tab.ptw);
  const float inv = 1.f / kOsM;
  for (int j = threadIdx.x; j < kEqTaps; j += blockDim.x) {
    P.dtaps[j] = sm[pidx((j - kEqHalf) & (kOsM - 1))].x * inv;
    P.dtaps[P.Nh + j] = 0.f;
  }
}

void launch_eq_spec(const LaunchCtx& c, const int* procs, int n) {
  if (n) k_eq_spec<<<n, kOsThreads, kOsP * sizeof(float2), c.stream>>>(c, procs);
}
void launch_eq_os_fwd(const LaunchCtx& c, const Item* items, int n) {
  if (n) k_eq_os_fwd<<<n, kOsThreads, kOsP * sizeof(float2), c.stream>>>(c, items);
}
void launch_eq_os_bwd(const LaunchCtx& c, const Item* items, int n) {
  if (n) k_eq_os_bwd<<<n, kOsBwdThreads, (2 * kOsP + kOsM) * sizeof(float2), c.stream>>>(c, items);
}
void launch_eq_os_du(const LaunchCtx& c, const Item* items, int n) {
  if (n) k_eq_os_du<<<n, kOsThreads, kOsP * sizeof(float2), c.stream>>>(c, items);
}
void launch_eq_dh_reduce(const LaunchCtx& c, const int* procs, int n) {
  if (n) k_eq_dh_reduce<<<n, kOsThreads, kOsP * sizeof(float2), c.stream>>>(c, procs);
}
void init_eqos_attributes() {
  cudaFuncSetAttribute(k_eq_spec, cudaFuncAttributeMaxDynamicSharedMemorySize, kOsP * (int)sizeof(float2));
  cudaFuncSetAttribute(k_eq_os_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, kOsP * (int)sizeof(float2));
  cudaFuncSetAttribute(k_eq_os_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (2 * kOsP + kOsM) * (int)sizeof(float2));
  cudaFuncSetAttribute(k_eq_os_du, cudaFuncAttributeMaxDynamicSharedMemorySize, kOsP * (int)sizeof(float2));
  cudaFuncSetAttribute(k_eq_dh_reduce, cudaFuncAttributeMaxDynamicSharedMemorySize, kOsP * (int)sizeof(float2));
}

}  // namespace mg

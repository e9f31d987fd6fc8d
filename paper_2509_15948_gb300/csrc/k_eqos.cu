// Equalizer (Sec. 3.3, Eqs. 7-8) by single-pass overlap-save in shared memory.
// The 2047-tap zero-phase FIR is short against an 8192-point FFT, so every block of output samples is
// computed by one CTA from its input segment without any global scratch:
//   forward:  segment [s0 - 1023, s0 + 6146 + 1023) -> FFT -> x H -> IFFT -> 6146 valid outputs, fused with the
//             dry/wet blend and the L_g energies;
//   backward: segment [s0 - 2046, s0 + 4100 + 2046) -> U; y_bar = IFFT(U H) on [s0 - 1023, s0 + 4100 + 1023);
//             dL/dy_bar = w dy + c1 y_bar_mid there; du = IFFT(H FFT(dL/dy_bar)) on the block (h is even, so the
//             correlation adjoint is the same convolution); dL/dh partial = Re IFFT(FFT(dL/dy_bar on the block)
//             conj(U)) at lags -1023..1023 (the real part of the packed product is the sum over both channels).
// H is real (h real and even); both channels travel packed as one complex signal.
#include "mg_fftp.cuh"

namespace mg {

namespace {
constexpr int kOsLog = 13;
constexpr int kOsM = 1 << kOsLog;
constexpr int kOsThreads = 512;
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
  fft_p<false>(sm, kOsLog, 1, kOsP, c.tab.tw);
  for (int k = threadIdx.x; k < kOsM; k += blockDim.x) P.hspec[k] = sm[pidx(k)].x;
}

// item = (node, block): outputs [s0, s0 + 6146).
__global__ void __launch_bounds__(kOsThreads, 2) k_eq_os_fwd(LaunchCtx c, const Item* __restrict__ items) {
  extern __shared__ float2 sm[];
  __shared__ float red[2 * 32];
  const Item it = items[blockIdx.x];
  const ProcDev& P = c.procs[it.proc];
  constexpr int B = kOsM - 2 * kEqHalf;
  const int s0 = it.idx * B;
  for (int j = threadIdx.x; j < kOsM; j += blockDim.x) {
    const int s = s0 - kEqHalf + j;
    sm[pidx(j)] = (s >= 0 && s < P.L) ? make_float2(P.u[s], P.u[P.ld + s]) : make_float2(0.f, 0.f);
  }
  __syncthreads();
  fft_p<false>(sm, kOsLog, 1, kOsP, c.tab.tw);
  for (int k = threadIdx.x; k < kOsM; k += blockDim.x) sm[pidx(k)] = cscale(sm[pidx(k)], P.hspec[k]);
  __syncthreads();
  fft_p<true>(sm, kOsLog, 1, kOsP, c.tab.tw);
  const float w = dry_wet_w(c, P.qidx), wd = dry_wet_d(c, P.qidx);
  const float inv = 1.f / kOsM;
  float acc[2] = {0.f, 0.f};
  for (int t = threadIdx.x; t < B; t += blockDim.x) {
    const int s = s0 + t;
    if (s >= P.L) break;
    const float2 yb = cscale(sm[pidx(kEqHalf + t)], inv);
    const float ul = P.u[s], ur = P.u[P.ld + s];
    P.y[s] = w * yb.x + wd * ul;
    P.y[P.ld + s] = w * yb.y + wd * ur;
    const float ym = yb.x + yb.y, um = ul + ur;
    acc[0] += ym * ym;
    acc[1] += um * um;
  }
  float out[2];
  block_sum<2>(acc, red, out);
  if (threadIdx.x == 0) {
    P.fpart[it.idx * kNPart + 0] = out[0];
    P.fpart[it.idx * kNPart + 1] = out[1];
  }
}

// item = (node, block): block [s0, s0 + 4100).  Three padded 8192-point buffers in shared memory (204 KB).
__global__ void __launch_bounds__(kOsThreads) k_eq_os_bwd(LaunchCtx c, const Item* __restrict__ items) {
  extern __shared__ float2 sm[];
  __shared__ float red[32];
  float2* A = sm;                 // spectrum of the u segment
  float2* Bf = sm + kOsP;         // y_bar, then dL/dy_bar and du
  float2* C = sm + 2 * kOsP;      // dL/dy_bar restricted to the block, then the correlation
  const Item it = items[blockIdx.x];
  const ProcDev& P = c.procs[it.proc];
  constexpr int H2 = 2 * kEqHalf;              // 2046
  constexpr int B = kOsM - 2 * H2;             // 4100
  const int s0 = it.idx * B;
  const int segbeg = s0 - H2;
  for (int j = threadIdx.x; j < kOsM; j += blockDim.x) {
    const int s = segbeg + j;
    A[pidx(j)] = (s >= 0 && s < P.L) ? make_float2(P.u[s], P.u[P.ld + s]) : make_float2(0.f, 0.f);
  }
  __syncthreads();
  fft_p<false>(A, kOsLog, 1, kOsP, c.tab.tw);
  for (int k = threadIdx.x; k < kOsM; k += blockDim.x) Bf[pidx(k)] = cscale(A[pidx(k)], P.hspec[k]);
  __syncthreads();
  fft_p<true>(Bf, kOsLog, 1, kOsP, c.tab.tw);
  const float w = dry_wet_w(c, P.qidx), wd = dry_wet_d(c, P.qidx);
  const float c1 = P.stats[2], c2 = P.stats[3];
  const float inv = 1.f / kOsM;
  float acc[1] = {0.f};
  for (int j = threadIdx.x; j < kOsM; j += blockDim.x) {
    const int s = segbeg + j;
    float2 d = make_float2(0.f, 0.f), dblk = d;
    if (j >= kEqHalf && j < kOsM - kEqHalf && s >= 0 && s < P.L) {
      const float2 yb = cscale(Bf[pidx(j)], inv);
      const float gl = P.dy[s], gr = P.dy[P.ld + s];
      const float gm = c1 * (yb.x + yb.y);
      d = make_float2(w * gl + gm, w * gr + gm);
      if (j >= H2 && j < H2 + B) {
        dblk = d;
        acc[0] += gl * (yb.x - P.u[s]) + gr * (yb.y - P.u[P.ld + s]);
      }
    }
    Bf[pidx(j)] = d;
    C[pidx(j)] = dblk;
  }
  float out[1];
  block_sum<1>(acc, red, out);    // barrier before the transforms
  if (threadIdx.x == 0) P.bpart[it.idx * kNPart] = out[0];
  fft_p<false>(Bf, kOsLog, 1, kOsP, c.tab.tw);
  fft_p<false>(C, kOsLog, 1, kOsP, c.tab.tw);
  for (int k = threadIdx.x; k < kOsM; k += blockDim.x) {
    const int e = pidx(k);
    Bf[e] = cscale(Bf[e], P.hspec[k]);
    C[e] = cmulc(C[e], A[e]);
  }
  __syncthreads();
  fft_p<true>(Bf, kOsLog, 1, kOsP, c.tab.tw);
  fft_p<true>(C, kOsLog, 1, kOsP, c.tab.tw);
  for (int t = threadIdx.x; t < B; t += blockDim.x) {
    const int s = s0 + t;
    if (s >= P.L) break;
    const float2 dw = cscale(Bf[pidx(H2 + t)], inv);
    const float um = c2 * (P.u[s] + P.u[P.ld + s]);
    P.du[s] = wd * P.dy[s] + dw.x + um;
    P.du[P.ld + s] = wd * P.dy[P.ld + s] + dw.y + um;
  }
  // lags n = -1023..1023 sit at circular positions n mod M; partial row of this block
  float* dst = P.dhpart + (size_t)it.idx * kEqTaps;
  for (int j = threadIdx.x; j < kEqTaps; j += blockDim.x) {
    const int n = j - kEqHalf;
    dst[j] = C[pidx(n & (kOsM - 1))].x * inv;
  }
}

// dL/dh (both channels summed into row 0, row 1 zero) from the per-block partials, fixed order.
__global__ void __launch_bounds__(256) k_eq_dh_reduce(LaunchCtx c, const int* __restrict__ procs) {
  const ProcDev& P = c.procs[procs[blockIdx.x]];
  for (int j = threadIdx.x; j < kEqTaps; j += blockDim.x) {
    float s = 0.f;
    for (int b = 0; b < P.nbpart; ++b) s += P.dhpart[(size_t)b * kEqTaps + j];
    P.dtaps[j] = s;
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
  if (n) k_eq_os_bwd<<<n, kOsThreads, 3 * kOsP * sizeof(float2), c.stream>>>(c, items);
}
void launch_eq_dh_reduce(const LaunchCtx& c, const int* procs, int n) {
  if (n) k_eq_dh_reduce<<<n, 256, 0, c.stream>>>(c, procs);
}
void init_eqos_attributes() {
  cudaFuncSetAttribute(k_eq_spec, cudaFuncAttributeMaxDynamicSharedMemorySize, kOsP * (int)sizeof(float2));
  cudaFuncSetAttribute(k_eq_os_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, kOsP * (int)sizeof(float2));
  cudaFuncSetAttribute(k_eq_os_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, 3 * kOsP * (int)sizeof(float2));
}

}  // namespace mg

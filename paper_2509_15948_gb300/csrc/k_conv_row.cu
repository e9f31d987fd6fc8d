// Row passes of the four-step FFT convolution (see k_conv_common.cuh).
#include "k_conv_common.cuh"

namespace mg {

namespace {

// Row pass of the filter spectrum: forward N1-point FFTs of rows a and b = N2 - a of Hz, in place.
__global__ void __launch_bounds__(kRowThreads, 2) k_row_fwd_hz(LaunchCtx c, const Item* __restrict__ items) {
  extern __shared__ float2 sm[];
  const Item it = items[blockIdx.x];
  const ProcDev& P = c.procs[it.proc];
  const int N1 = rows_len(P), N2 = 1 << P.logN2, rs = pstride(N1);
  const int a = it.idx, b = (N2 - it.idx) & (N2 - 1);
  const int nr = a == b ? 1 : 2;
  float2* ha = P.Hz + (int64_t)a * N1;
  float2* hb = P.Hz + (int64_t)b * N1;
  // global in, global out: the first pass reads the rows, the last writes them (the passes between hold
  // barriers, so every read precedes every write)
  row_fft<false>(sm, P, nr, rs, c.tab, [=](int slot, int k1) { return (slot ? hb : ha)[k1]; },
                 [=](int slot, int k1, float2 v) { (slot ? hb : ha)[k1] = v; });
}

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

}  // namespace

void init_kernel_attributes() {
  init_col_attributes();
  init_dyn_attributes();
  cudaFuncSetAttribute(k_row_fwd_hz, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * pstride(kMaxRow) * (int)sizeof(float2));
  cudaFuncSetAttribute(k_row_conv<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * pstride(kMaxRow) * (int)sizeof(float2));
  cudaFuncSetAttribute(k_row_conv<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * pstride(kMaxRow) * (int)sizeof(float2));
  init_row_bwd_attributes();
}


void launch_row_fwd_hz(const LaunchCtx& c, const Item* items, int n, int maxN1) {
  if (n) k_row_fwd_hz<<<n, row_threads(maxN1), (size_t)2 * pstride(maxN1) * sizeof(float2), c.stream>>>(c, items);
}

void launch_row_conv_fwd(const LaunchCtx& c, const Item* items, int n, int maxN1, bool keep) {
  if (!n) return;
  const size_t smem = (size_t)2 * pstride(maxN1) * sizeof(float2);
  if (keep) k_row_conv<true><<<n, row_threads(maxN1), smem, c.stream>>>(c, items);
  else k_row_conv<false><<<n, row_threads(maxN1), smem, c.stream>>>(c, items);
}


}  // namespace mg

// Backward row pass of the four-step FFT convolution (see k_conv_common.cuh).
#include "k_conv_common.cuh"

namespace mg {

namespace {

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
  // the dH rows written to T1 become visible to the whole block at the barrier that opens the second inverse
  // transform, which reads them back from T1 in its first pass
  const float2* ta = P.T1 + (int64_t)a * N1;
  const float2* tb = P.T1 + (int64_t)b * N1;
  inv_rows_store(s, P.T1, a, b, P, c.tab, tt, [=](int slot, int k1) { return (slot ? tb : ta)[k1]; });
}

}  // namespace

void init_row_bwd_attributes() {
  cudaFuncSetAttribute(k_row_bwd2, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * pstride(kMaxRow) * (int)sizeof(float2));
}

void launch_row_bwd2(const LaunchCtx& c, const Item* items, int n, int maxN1) {
  if (!n) return;
  const size_t smem = (size_t)2 * pstride(maxN1) * sizeof(float2);
  k_row_bwd2<<<n, row_threads(maxN1), smem, c.stream>>>(c, items);
}

}  // namespace mg

// Elementwise processors (gain/panning Eq. 4, stereo imager Eqs. 5-6) fused with the dry/wet blend
// (Eq. 2b), their adjoints, the mix / output sums (Eq. 3) and source ingest (input node i).
// HBM-bound: one read of u and one write of y per sample in the forward pass; one read of dy and u
// and one write of du in the backward pass; float4 accesses on 256-byte aligned planar rows.
#include "mg_fft.cuh"

namespace mg {

__global__ void __launch_bounds__(256) k_gs_fwd(LaunchCtx c, const Item* __restrict__ items) {
  const Item it = items[blockIdx.x];
  const ProcDev& P = c.procs[it.proc];
  const float w = dry_wet_w(c, P.qidx), wd = dry_wet_d(c, P.qidx);
  const float4* ul = reinterpret_cast<const float4*>(P.u);
  const float4* ur = reinterpret_cast<const float4*>(P.u + P.ld);
  float4* yl = reinterpret_cast<float4*>(P.y);
  float4* yr = reinterpret_cast<float4*>(P.y + P.ld);
  const int v0 = it.idx * (c.elem_tile / 4);
  const int vend = min(v0 + c.elem_tile / 4, (P.L + 3) >> 2);
  if (P.type == T_G) {
    const float gl = expf(P.p[0]), gr = expf(P.p[1]);
    for (int v = v0 + threadIdx.x; v < vend; v += blockDim.x) {
      const float4 a = ul[v], b = ur[v];
      float4 oa, ob;
      oa.x = w * (gl * a.x) + wd * a.x; oa.y = w * (gl * a.y) + wd * a.y;
      oa.z = w * (gl * a.z) + wd * a.z; oa.w = w * (gl * a.w) + wd * a.w;
      ob.x = w * (gr * b.x) + wd * b.x; ob.y = w * (gr * b.y) + wd * b.y;
      ob.z = w * (gr * b.z) + wd * b.z; ob.w = w * (gr * b.w) + wd * b.w;
      yl[v] = oa;
      yr[v] = ob;
    }
  } else {  // stereo imager
    const float e = expf(P.p[0]);
    for (int v = v0 + threadIdx.x; v < vend; v += blockDim.x) {
      const float4 a = ul[v], b = ur[v];
      float4 oa, ob;
#define MG_IMG(X)                                         \
  {                                                       \
    const float m = a.X + b.X, s = e * (a.X - b.X);       \
    oa.X = w * ((m + s) * 0.5f) + wd * a.X;        \
    ob.X = w * ((m - s) * 0.5f) + wd * b.X;        \
  }
      MG_IMG(x) MG_IMG(y) MG_IMG(z) MG_IMG(w)
#undef MG_IMG
      yl[v] = oa;
      yr[v] = ob;
    }
  }
}

// Adjoints.  g: du_c = (1-w) dy_c + w e^{p_c} dy_c; partials S_c = sum dy_c u_c give
// dp_c = w e^{p_c} S_c and dw = sum_c (e^{p_c} - 1) S_c.
// s: du from the transposed 2x2 mixing matrix; partial S = sum (u_l - u_r)(dy_l - dy_r) gives
// dp = w e^p S / 2 and dw = (e^p - 1) S / 2.
__global__ void __launch_bounds__(256) k_gs_bwd(LaunchCtx c, const Item* __restrict__ items) {
  __shared__ float red[2 * 32];
  const Item it = items[blockIdx.x];
  const ProcDev& P = c.procs[it.proc];
  const float w = dry_wet_w(c, P.qidx), wd = dry_wet_d(c, P.qidx);
  const float4* ul = reinterpret_cast<const float4*>(P.u);
  const float4* ur = reinterpret_cast<const float4*>(P.u + P.ld);
  const float4* gl4 = reinterpret_cast<const float4*>(P.dy);
  const float4* gr4 = reinterpret_cast<const float4*>(P.dy + P.ld);
  float4* dl = reinterpret_cast<float4*>(P.du);
  float4* dr = reinterpret_cast<float4*>(P.du + P.ld);
  const int v0 = it.idx * (c.elem_tile / 4);
  const int vend = min(v0 + c.elem_tile / 4, (P.L + 3) >> 2);
  float acc[2] = {0.f, 0.f};
  if (P.type == T_G) {
    const float kl = wd + w * expf(P.p[0]), kr = wd + w * expf(P.p[1]);
    for (int v = v0 + threadIdx.x; v < vend; v += blockDim.x) {
      const float4 a = ul[v], b = ur[v], ga = gl4[v], gb = gr4[v];
      acc[0] += ga.x * a.x + ga.y * a.y + ga.z * a.z + ga.w * a.w;
      acc[1] += gb.x * b.x + gb.y * b.y + gb.z * b.z + gb.w * b.w;
      dl[v] = make_float4(kl * ga.x, kl * ga.y, kl * ga.z, kl * ga.w);
      dr[v] = make_float4(kr * gb.x, kr * gb.y, kr * gb.z, kr * gb.w);
    }
  } else {
    const float e = expf(P.p[0]);
    for (int v = v0 + threadIdx.x; v < vend; v += blockDim.x) {
      const float4 a = ul[v], b = ur[v], ga = gl4[v], gb = gr4[v];
      float4 oa, ob;
#define MG_IMGB(X)                                                   \
  {                                                                  \
    const float bl = w * ga.X, br = w * gb.X;                        \
    const float sm = 0.5f * (bl + br), df = 0.5f * e * (bl - br);    \
    oa.X = wd * ga.X + sm + df;                               \
    ob.X = wd * gb.X + sm - df;                               \
    acc[0] += (a.X - b.X) * (ga.X - gb.X);                           \
  }
      MG_IMGB(x) MG_IMGB(y) MG_IMGB(z) MG_IMGB(w)
#undef MG_IMGB
      dl[v] = oa;
      dr[v] = ob;
    }
  }
  float out[2];
  block_sum<2>(acc, red, out);
  if (threadIdx.x == 0) {
    P.bpart[it.idx * kNPart + 0] = out[0];
    P.bpart[it.idx * kNPart + 1] = out[1];
  }
}

// Eq. (3) sums: out[s] = sum over its inputs (mix node m and output node o).
__global__ void __launch_bounds__(256) k_sum(float* const* outs, const float* const* ins, const int* in_beg,
                                             const int* Ls, const int* lds, const Item* items, int tile) {
  const Item it = items[blockIdx.x];
  const int s = it.proc, L = Ls[s], ld = lds[s];
  const int beg = in_beg[s], end = in_beg[s + 1];
  const int v0 = it.idx * (tile / 4);
  const int vend = min(v0 + tile / 4, (L + 3) >> 2);
  float4* ol = reinterpret_cast<float4*>(outs[s]);
  float4* orr = reinterpret_cast<float4*>(outs[s] + ld);
  for (int v = v0 + threadIdx.x; v < vend; v += blockDim.x) {
    float4 al = make_float4(0.f, 0.f, 0.f, 0.f), ar = al;
    for (int j = beg; j < end; ++j) {
      const float4 a = reinterpret_cast<const float4*>(ins[j])[v];
      const float4 b = reinterpret_cast<const float4*>(ins[j] + ld)[v];
      al.x += a.x; al.y += a.y; al.z += a.z; al.w += a.w;
      ar.x += b.x; ar.y += b.y; ar.z += b.z; ar.w += b.w;
    }
    ol[v] = al;
    orr[v] = ar;
  }
}

__global__ void k_ingest(const float* __restrict__ mono, float* __restrict__ st, int L, int ld) {
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < L; n += gridDim.x * blockDim.x) {
    const float x = mono[n];
    st[n] = x;
    st[ld + n] = x;
  }
}

// All K mono sources of one song ([K][L], device-readable: device memory or mapped pinned host memory) into
// both rows of their tracks' input buffers, one launch: blockIdx.y is the track.
__global__ void k_ingest_song(const float* __restrict__ mono, float* const* __restrict__ dst, int L, int ld) {
  const float* src = mono + (size_t)blockIdx.y * L;
  float* st = dst[blockIdx.y];
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < L; n += gridDim.x * blockDim.x) {
    const float x = src[n];
    st[n] = x;
    st[ld + n] = x;
  }
}

__global__ void k_copy_mix(const SongDev* songs, int nsongs, float* out, const int64_t* offs) {
  const int s = blockIdx.y;
  const SongDev& S = songs[s];
  float* o = out + offs[s];
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < S.L; n += gridDim.x * blockDim.x) {
    o[n] = S.mix[n];
    o[S.L + n] = S.mix[S.ld + n];
  }
}

void launch_gs_fwd(const LaunchCtx& c, const Item* items, int n) {
  if (n) k_gs_fwd<<<n, 256, 0, c.stream>>>(c, items);
}
void launch_gs_bwd(const LaunchCtx& c, const Item* items, int n) {
  if (n) k_gs_bwd<<<n, 256, 0, c.stream>>>(c, items);
}
void launch_sum(cudaStream_t st, float* const* outs, const float* const* ins, const int* in_beg, const int* L,
                const int* ld, const Item* items, int n, int tile) {
  if (n) k_sum<<<n, 256, 0, st>>>(outs, ins, in_beg, L, ld, items, tile);
}
void launch_ingest(cudaStream_t st, const float* mono, float* stereo, int L, int ld) {
  k_ingest<<<min(1024, (L + 255) / 256), 256, 0, st>>>(mono, stereo, L, ld);
}
void launch_ingest_song(cudaStream_t st, const float* mono, float* const* dst, int K, int L, int ld) {
  if (K > 0 && L > 0) k_ingest_song<<<dim3(std::min(256, (L + 255) / 256), K), 256, 0, st>>>(mono, dst, L, ld);
}
void launch_copy_mix(cudaStream_t st, const SongDev* songs, int nsongs, float* out, const int64_t* offs) {
  if (nsongs) k_copy_mix<<<dim3(256, nsongs), 256, 0, st>>>(songs, nsongs, out, offs);
}

}  // namespace mg

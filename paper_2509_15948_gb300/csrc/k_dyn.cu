// Compressor (Sec. 3.5) and noisegate (Sec. 3.6): the exact one-pole envelope recursion of Eq. (11),
// g[n] = alpha g[n-1] + (1 - alpha) x[n], x = (u_l + u_r)^2, evaluated as a chained single-pass scan over chunks
// of 4096 samples.  CTAs take chunks in list order from a launch-wide ticket, so the chunk a CTA depends on was
// taken earlier by a CTA that is running or finished.  A CTA
//   1. computes its chunk's zero-start end state (a warp-shuffle scan of the per-thread states, decay alpha^16
//      per thread),
//   2. waits (bounded) for the state entering its chunk, published by the CTA of the previous chunk, and
//      publishes the state entering the next chunk, g_next = A g_in + agg (A = alpha^4096); the stage's chunks are
//      listed in rounds across nodes, so that wait is normally over before it starts,
//   3. rescans its chunk from that state and applies the gain law (Eqs. 13-16) and Eq. (15), fused with the
//      dry/wet blend.  The forward's input arrives by TMA (a bulk tensor copy into shared memory, read by both
//      steps) when the node has a tensor map, else by plain loads with the rescan from L2.
// The adjoint runs the same way in reverse: lambda[n] = dL/dg[n] + alpha lambda[n+1], chunks in reverse order.
// Its first step also does the per-sample work that does not depend on lambda (the gain law, its partials,
// dL/dg and the lambda-free part of du), staged in global memory for the same CTA's last step.  A wait that
// runs out (about half a second) sets a host-visible error word and continues with a zero state.
#include "mg_fft.cuh"

namespace mg {

namespace {

constexpr int kPer = 16;   // samples per thread
constexpr int kThreads = kDynChunk / kPer;

struct DynParams {
  float alpha, beta, lna, T, W, R, Rm1;   // Rm1 = R - 1 = exp(p3)   // beta = 1 - alpha, evaluated as sigmoid(-p0) (no cancellation near 1)
  float invR, invR2, inv2W, inv4W;        // 1/R, 1/R^2, 1/(2W), 1/(4W): the gain laws multiply instead of dividing
  bool gate;
};

__device__ __forceinline__ DynParams dyn_params(const ProcDev& P) {
  DynParams d;
  const float p0 = P.p[0];
  d.alpha = 1.f / (1.f + expf(-p0));
  d.beta = 1.f / (1.f + expf(p0));
  d.lna = -log1pf(expf(-p0));          // ln sigmoid(p0)
  if (p0 < -20.f) d.lna = p0;          // log1p(exp(-p0)) = -p0 + log1p(exp(p0))
  d.T = P.p[1];
  d.W = expf(P.p[2]);
  d.Rm1 = expf(P.p[3]);
  d.R = 1.f + d.Rm1;
  d.invR = 1.f / d.R;
  d.invR2 = d.invR * d.invR;
  d.inv2W = 0.5f / d.W;
  d.inv4W = 0.25f / d.W;
  d.gate = P.type == T_N;
  return d;
}

// Gain laws (Eqs. 13-14 compressor, Eq. 16 noisegate) with their partial derivatives; t = q / (2W) in the knees.
__device__ __forceinline__ float gain_law(const DynParams& d, float G, float& dG, float& dT, float& dW, float& dR) {
  const float T = d.T, W = d.W, R = d.R, Rm1 = d.Rm1;
  if (!d.gate) {
    if (G >= T + W) {
      dG = d.invR; dT = Rm1 * d.invR; dW = 0.f; dR = -(G - T) * d.invR2;
      return T + (G - T) * d.invR;
    }
    if (G >= T - W) {
      const float q = G - T + W, k = -Rm1 * d.invR, t = q * d.inv2W, qq = q * q * d.inv4W;
      dG = 1.f + k * t; dT = -k * t;
      dW = k * (t - t * t); dR = -qq * d.invR2;
      return G + k * qq;
    }
    dG = 1.f; dT = 0.f; dW = 0.f; dR = 0.f;
    return G;
  }
  if (G >= T + W) {
    dG = 1.f; dT = 0.f; dW = 0.f; dR = 0.f;
    return G;
  }
  if (G >= T - W) {
    const float q = G - T - W, k = -Rm1, t = q * d.inv2W, qq = q * q * d.inv4W;
    dG = 1.f + k * t; dT = -k * t;
    dW = k * (-t - t * t); dR = -qq;
    return G + k * qq;
  }
  dG = R; dT = -Rm1; dW = 0.f; dR = G - T;
  return T + R * (G - T);
}

__device__ __forceinline__ float gain_law_v(const DynParams& d, float G) {
  float a, b, cc, e;
  return gain_law(d, G, a, b, cc, e);
}

// Samples of a quad at and beyond L are zeroed on load and skipped on store, so nothing depends on what the
// padding of a [2][ld] buffer holds.
__device__ __forceinline__ float4 tail_zero(float4 a, int n, int L) {
  if (n + 1 >= L) a.y = 0.f;
  if (n + 2 >= L) a.z = 0.f;
  if (n + 3 >= L) a.w = 0.f;
  return a;
}

__device__ __forceinline__ void store_quad(float* p, int n, int L, float x, float y, float z, float w) {
  if (n + 4 <= L) {
    *reinterpret_cast<float4*>(p + n) = make_float4(x, y, z, w);
    return;
  }
  p[n] = x;
  if (n + 1 < L) p[n + 1] = y;
  if (n + 2 < L) p[n + 2] = z;
}

// Decay powers of one node, computed once per CTA: dl[j] = alpha^(16 j) (j < 32, one thread's samples apart) and
// dw[j] = alpha^(512 j) (j < 8, one warp's samples apart), each expf(n ln alpha) of its exact exponent n.
constexpr int kDecay = 40;
__device__ __forceinline__ void init_decay(float* dec, float lna) {
  if (threadIdx.x < kDecay) {
    const int t = threadIdx.x;
    dec[t] = expf((float)(t < 32 ? kPer * t : kPer * 32 * (t - 32)) * lna);
  }
  __syncthreads();
}

// Exclusive forward scan over the block: returns the state entering this thread's first sample, given the
// per-thread zero-start end states s (each spanning 16 samples) and the chunk's entering state.
__device__ __forceinline__ float scan_fwd_excl(float s, const float* dl, const float* dw, float carry,
                                               float* sm /* >= 16 floats */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  float inc = s;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const float v = __shfl_up_sync(0xffffffffu, inc, off);
    if (lane >= off) inc += v * dl[off];
  }
  if (lane == 31) sm[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    float t = lane < kThreads / 32 ? sm[lane] : 0.f;
    float ti = t;
#pragma unroll
    for (int off = 1; off < kThreads / 32; off <<= 1) {
      const float v = __shfl_up_sync(0xffffffffu, ti, off);
      if (lane >= off) ti += v * dw[off];
    }
    // exclusive warp prefix, with the chunk carry folded in
    float ex = __shfl_up_sync(0xffffffffu, ti, 1);
    if (lane == 0) ex = 0.f;
    ex += carry * dw[lane & 7];
    if (lane < kThreads / 32) sm[8 + lane] = ex;
  }
  __syncthreads();
  const float win = sm[8 + wid];   // state entering the warp
  float ex = __shfl_up_sync(0xffffffffu, inc, 1);
  if (lane == 0) ex = 0.f;
  const float res = ex + win * dl[lane];
  __syncthreads();
  return res;
}

// Exclusive reverse scan: state entering this thread's last sample from the right.
__device__ __forceinline__ float scan_rev_excl(float r, const float* dl, const float* dw, float carry, float* sm) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int nw = kThreads / 32;
  float inc = r;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const float v = __shfl_down_sync(0xffffffffu, inc, off);
    if (lane + off < 32) inc += v * dl[off];
  }
  if (lane == 0) sm[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    // reverse scan over warps: warp w receives sum_{w' > w} total_{w'} decayed, plus the carry
    float t = lane < nw ? sm[lane] : 0.f;
    float ti = t;
#pragma unroll
    for (int off = 1; off < nw; off <<= 1) {
      const float v = __shfl_down_sync(0xffffffffu, ti, off);
      if (lane + off < nw) ti += v * dw[off];
    }
    float ex = __shfl_down_sync(0xffffffffu, ti, 1);
    if (lane >= nw - 1) ex = 0.f;
    ex += carry * dw[(nw - 1 - lane) & 7];
    if (lane < nw) sm[8 + lane] = ex;
  }
  __syncthreads();
  const float win = sm[8 + wid];
  float ex = __shfl_down_sync(0xffffffffu, inc, 1);
  if (lane == 31) ex = 0.f;
  const float res = ex + win * dl[31 - lane];
  __syncthreads();
  return res;
}

}  // namespace

constexpr long long kChainWaitCycles = 1000000000LL;   // about half a second at the SM clock

__global__ void k_chain_begin(unsigned* chain) {
  chain[0] += 1u;   // a new launch generation: flags of earlier launches no longer match
  chain[1] = 0u;    // the work ticket
}

// Work item of this CTA in ticket order (thread 0 draws, the block reads it after the barrier).
__device__ __forceinline__ Item take_item(const LaunchCtx& c, const Item* items, int* s_idx, unsigned* s_gen) {
  if (threadIdx.x == 0) {
    *s_idx = (int)atomicAdd(&c.chain[1], 1u);
    *s_gen = *(volatile unsigned*)&c.chain[0];
  }
  __syncthreads();
  return items[*s_idx];
}

// Thread 0: the state entering chunk k (0 for the first chunk of the direction), once the CTA of the neighbouring
// chunk has published it; then the state entering the next chunk, published for its CTA.  A published state is one
// 64-bit word, the launch generation in the high half and the float's bits in the low half, written and read as a
// whole: the value arrives with its flag, and no fence is needed between them.  keep (forward only) receives the
// state entering chunk k for the backward.
__device__ __forceinline__ float chain_link(const LaunchCtx& c, const ProcDev& P, int k, int next, bool first,
                                            float agg, float A, unsigned gen, bool hold, float* keep) {
  float in = 0.f;
  if (!first) {
    volatile unsigned long long* f = P.cflag + k;
    const long long t0 = clock64();
    unsigned long long w = *f;
    while ((unsigned)(w >> 32) != gen) {
      if (clock64() - t0 > kChainWaitCycles) {
        *(volatile int*)c.err = 1;
        w = 0ull;   // continue from a zero state
        break;
      }
      __nanosleep(32);
      w = *f;
    }
    in = __uint_as_float((unsigned)w);
  }
  if (next >= 0 && next < P.nchunks && !hold)
    *(volatile unsigned long long*)(P.cflag + next) =
        ((unsigned long long)gen << 32) | __float_as_uint(fmaf(A, in, agg));
  if (keep) keep[k] = in;
  return in;
}

__device__ __forceinline__ float q_at(const float4& v, int e) { return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w; }

// ---- TMA staging of a scan chunk ----
// With a tensor map of a node's [2][ld] buffer (its input u, or in the backward also its adjoint dL/dy: rows of
// 32 floats = 128 bytes, both channels: 2 ld / 32 rows), one thread stages the chunk's 128 rows of each channel
// into shared memory with two bulk tensor copies
// (cp.async.bulk.tensor, 128-byte swizzle) completing on an mbarrier.  Rows past the tensor read as zeros; rows of
// the left channel past its ld read the right channel's first rows, and every sample at or beyond L is masked
// anyway.  The swizzle stores the 16-byte chunk c of row r at chunk c ^ (r mod 8), so the quads a thread reads
// (row t / 2, chunks 4 (t mod 2) + j) fall on distinct bank groups within each quarter warp.
constexpr int kChanBytes = kDynChunk * 4;                  // one channel of a chunk, 16 KB
constexpr int kDynFwdSmem = 2 * kChanBytes + 1024;         // both channels + alignment slack of the swizzle
constexpr int kDynBwdSmem = 4 * kChanBytes + 1024;         // u and dL/dy, both channels

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void stage_init(unsigned long long* bar, unsigned bytes) {
  const unsigned b = smem_u32(bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
}

// Both channels of chunk idx of the buffer behind `map` ([2][ld] floats) into dst (left) and dst + 16 KB (right).
__device__ __forceinline__ void stage_copy(const void* map, int ld, int idx, float* dst, unsigned long long* bar) {
  const unsigned b = smem_u32(bar), d = smem_u32(dst);
  const unsigned long long m = reinterpret_cast<unsigned long long>(map);
  const int r0 = idx * (kDynChunk / 32), r1 = ld / 32 + r0;
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(d), "l"(m), "r"(0), "r"(r0), "r"(b) : "memory");
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(d + kChanBytes), "l"(m), "r"(0), "r"(r1), "r"(b) : "memory");
}

// Bounded wait for the staged chunk (phase 0 of the mbarrier): false when it did not arrive in time.
__device__ __forceinline__ bool stage_wait(const unsigned long long* bar) {
  const unsigned b = smem_u32(bar);
  const long long t0 = clock64();
  while (true) {
    unsigned ok;
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }"
                 : "=r"(ok) : "r"(b) : "memory");
    if (ok) return true;
    if (clock64() - t0 > kChainWaitCycles) return false;
  }
}

// Quad q of thread t's 16 samples of channel ch in a swizzled stage.
__device__ __forceinline__ float4* stage_at(float* stage, int ch, int t, int q) {
  const int row = t >> 1, chunk = ((t & 1) << 2) | q;
  return reinterpret_cast<float4*>(reinterpret_cast<char*>(stage) + ch * kChanBytes + row * 128 +
                                   ((chunk ^ (row & 7)) << 4));
}
__device__ __forceinline__ float4 stage_quad(const float* stage, int ch, int t, int q) {
  return *stage_at(const_cast<float*>(stage), ch, t, q);
}

__device__ __forceinline__ float4 mask_quad(float4 v, int n, int L) {
  return n < L ? tail_zero(v, n, L) : make_float4(0.f, 0.f, 0.f, 0.f);
}

// Forward: chunk aggregate, chained state, rescan with the gain law.  The chunk comes from the TMA stage when the
// node has a tensor map (read twice from shared memory), else from global memory (the rescan from L2).
__global__ void __launch_bounds__(kThreads, 4) k_dyn_fwd(LaunchCtx c, const Item* __restrict__ items) {
  extern __shared__ unsigned char dsm[];
  float* stage = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(dsm) + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) unsigned long long bar;
  __shared__ float red[32];
  __shared__ int s_idx;
  __shared__ unsigned s_gen;
  __shared__ float s_in;
  __shared__ float dec[kDecay];
  const Item it = take_item(c, items, &s_idx, &s_gen);
  const ProcDev& P = c.procs[it.proc];
  const bool tma = P.umap != nullptr;
  if (tma && threadIdx.x == 0) {
    stage_init(&bar, 2 * kChanBytes);
    stage_copy(P.umap, P.ld, it.idx, stage, &bar);
  }
  const DynParams d = dyn_params(P);
  init_decay(dec, d.lna);   // its barrier also publishes the mbarrier's initialisation
  const int t = threadIdx.x, n0 = it.idx * kDynChunk + t * kPer, L = P.L, ld = P.ld;
  if (tma) {
    const bool late = !stage_wait(&bar);
    if (__syncthreads_or(late)) {   // the copies did not arrive: report, let them land (bounded), skip the chunk
      if (t == 0) {
        *(volatile int*)c.err = 1;
        stage_wait(&bar);
      }
      __syncthreads();
      return;
    }
  }
  auto quad = [&](int ch, int q) {
    const int n = n0 + 4 * q;
    if (tma) return mask_quad(stage_quad(stage, ch, t, q), n, L);
    return n < L ? tail_zero(*reinterpret_cast<const float4*>(P.u + ch * ld + n), n, L) : make_float4(0.f, 0.f, 0.f, 0.f);
  };
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < kPer / 4; ++q) {
    const float4 a = quad(0, q), b = quad(1, q);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float m = q_at(a, e) + q_at(b, e);
      s = d.alpha * s + d.beta * (m * m);
    }
  }
  float v[1] = {s * (dec[31 - (t & 31)] * dec[32 + 7 - (t >> 5)])};   // alpha^(16 (255 - t))
  float out[1];
  block_sum<1>(v, red, out);
  if (t == 0) {
    const float A = expf((float)kDynChunk * d.lna);
    s_in = chain_link(c, P, it.idx, it.idx + 1, it.idx == 0, out[0], A, s_gen, c.chain_hold && s_idx == 0, P.carry);
  }
  __syncthreads();
  const float w = dry_wet_w(c, P.qidx), wd = dry_wet_d(c, P.qidx);
  float g = scan_fwd_excl(s, dec, dec + 32, s_in, red);
#pragma unroll
  for (int q = 0; q < kPer / 4; ++q) {
    const float4 a = quad(0, q), b = quad(1, q);   // again: shared memory, or L2
    float yl[4], yr[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float ul = q_at(a, e), ur = q_at(b, e), m = ul + ur;
      g = d.alpha * g + d.beta * (m * m);
      const float Gu = logf(g + kEnvEps);
      const float gain = expf(gain_law_v(d, Gu) - Gu);
      yl[e] = w * (gain * ul) + wd * ul;
      yr[e] = w * (gain * ur) + wd * ur;
    }
    const int n = n0 + 4 * q;
    if (n < L) {
      store_quad(P.y, n, L, yl[0], yl[1], yl[2], yl[3]);
      store_quad(P.y + ld, n, L, yr[0], yr[1], yr[2], yr[3]);
    }
  }
}

// dL/dg at one sample, plus accumulation of the gain-law parameter partials and dw.
struct DynAdj {
  float dT, dW, dR, dw;
};

__device__ __forceinline__ float dyn_dg(const DynParams& d, float w, float g, float ul, float ur, float gl, float gr,
                                        float& gain, DynAdj& acc) {
  const float Gu = logf(g + kEnvEps);
  float dG, dT, dW, dR;
  const float Gy = gain_law(d, Gu, dG, dT, dW, dR);
  gain = expf(Gy - Gu);
  const float bl = w * gl, br = w * gr;
  const float dE = (bl * ul + br * ur) * gain;
  acc.dT += dE * dT;
  acc.dW += dE * dW;
  acc.dR += dE * dR;
  acc.dw += gl * (gain * ul - ul) + gr * (gain * ur - ur);
  return dE * (dG - 1.f) * __frcp_rn(g + kEnvEps);
}

// One quad of a [2][ld] buffer's channel row at sample n (n a multiple of 4; zeros at and beyond L).
__device__ __forceinline__ float4 load_quad(const float* row, int n, int L) {
  return n < L ? tail_zero(*reinterpret_cast<const float4*>(row + n), n, L) : make_float4(0.f, 0.f, 0.f, 0.f);
}

// Backward.  Step 1, everything that does not depend on lambda: per sample dL/dg (to aux) and the part of du
// without the envelope term, the partials of dL/dT, dL/dW, dL/dR and dL/dw, and the chunk's zero-start lambda
// aggregate.  Step 2, the chained lambda state from the right.  Step 3: lambda[n] = dL/dg[n] + alpha lambda[n+1]
// from that state, du += 2 beta lambda m on both channels, and the partial of dL/dalpha =
// sum lambda[n] (g[n-1] - x[n]).  With tensor maps of u and dL/dy the chunk of both arrives by TMA: step 1 reads
// them from shared memory and leaves its part of du over dL/dy there, step 3 reads u and that part back from
// shared memory and dL/dg from L2, and du is written once.  Without maps u and dL/dy are read from global memory
// and step 1's part of du goes through global memory.  Both steps stream a quad at a time.
__global__ void __launch_bounds__(kThreads, 3) k_dyn_bwd(LaunchCtx c, const Item* __restrict__ items) {
  extern __shared__ unsigned char dsm[];
  float* stage = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(dsm) + 1023) & ~(uintptr_t)1023);
  float* dstage = stage + 2 * kDynChunk;   // dL/dy, then step 1's part of du
  __shared__ __align__(8) unsigned long long bar;
  __shared__ float sm[32 * 5];
  __shared__ int s_idx;
  __shared__ unsigned s_gen;
  __shared__ float s_in;
  __shared__ float dec[kDecay];
  const Item it = take_item(c, items, &s_idx, &s_gen);
  const ProcDev& P = c.procs[it.proc];
  const bool tma = P.umap != nullptr && P.dymap != nullptr;
  if (tma && threadIdx.x == 0) {
    stage_init(&bar, 4 * kChanBytes);
    stage_copy(P.umap, P.ld, it.idx, stage, &bar);
    stage_copy(P.dymap, P.ld, it.idx, dstage, &bar);
  }
  const DynParams d = dyn_params(P);
  init_decay(dec, d.lna);   // its barrier also publishes the mbarrier's initialisation
  const float w = dry_wet_w(c, P.qidx), wd = dry_wet_d(c, P.qidx);
  const int t = threadIdx.x, n0 = it.idx * kDynChunk + t * kPer, L = P.L, ld = P.ld;
  if (tma) {
    const bool late = !stage_wait(&bar);
    if (__syncthreads_or(late)) {   // the copies did not arrive: report, let them land (bounded), skip the chunk
      if (t == 0) {
        *(volatile int*)c.err = 1;
        stage_wait(&bar);
      }
      __syncthreads();
      return;
    }
  }
  auto uq = [&](int ch, int q) {
    const int n = n0 + 4 * q;
    return tma ? mask_quad(stage_quad(stage, ch, t, q), n, L) : load_quad(P.u + ch * ld, n, L);
  };
  {
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < kPer / 4; ++q) {
      const float4 a = uq(0, q), b = uq(1, q);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float m = q_at(a, e) + q_at(b, e);
        s = d.alpha * s + d.beta * (m * m);
      }
    }
    float g = scan_fwd_excl(s, dec, dec + 32, P.carry[it.idx], sm);
    DynAdj acc = {0.f, 0.f, 0.f, 0.f};
    float lam = 0.f, pw = 1.f;   // zero-start lambda entering the thread's first sample: sum_j alpha^j dL/dg[j]
#pragma unroll
    for (int q = 0; q < kPer / 4; ++q) {
      const int n = n0 + 4 * q;
      const float4 a = uq(0, q), b = uq(1, q);
      const float4 ga = tma ? mask_quad(stage_quad(dstage, 0, t, q), n, L) : load_quad(P.dy, n, L);
      const float4 gb = tma ? mask_quad(stage_quad(dstage, 1, t, q), n, L) : load_quad(P.dy + ld, n, L);
      float dl[4], dr[4], dgq[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float ul = q_at(a, e), ur = q_at(b, e), gl = q_at(ga, e), gr = q_at(gb, e);
        const float m = ul + ur;
        g = d.alpha * g + d.beta * (m * m);
        float gain;
        dgq[e] = dyn_dg(d, w, g, ul, ur, gl, gr, gain, acc);
        dl[e] = wd * gl + gain * (w * gl);
        dr[e] = wd * gr + gain * (w * gr);
        lam = fmaf(pw, dgq[e], lam);
        pw *= d.alpha;
      }
      if (tma) {
        *stage_at(dstage, 0, t, q) = make_float4(dl[0], dl[1], dl[2], dl[3]);
        *stage_at(dstage, 1, t, q) = make_float4(dr[0], dr[1], dr[2], dr[3]);
      }
      if (n < L) {
        if (!tma) {
          store_quad(P.du, n, L, dl[0], dl[1], dl[2], dl[3]);
          store_quad(P.du + ld, n, L, dr[0], dr[1], dr[2], dr[3]);
        }
        store_quad(P.aux, n, L, dgq[0], dgq[1], dgq[2], dgq[3]);
      }
    }
    float v[5] = {lam * (dec[t & 31] * dec[32 + (t >> 5)]), acc.dT, acc.dW, acc.dR, acc.dw};
    float out[5];
    block_sum<5>(v, sm, out);
    if (t == 0) {
      float* bp = P.bpart + (size_t)it.idx * kNPart;
#pragma unroll
      for (int j = 1; j < 5; ++j) bp[j] = out[j];
      const float A = expf((float)kDynChunk * d.lna);
      s_in = chain_link(c, P, it.idx, it.idx - 1, it.idx == P.nchunks - 1, out[0], A, s_gen,
                        c.chain_hold && s_idx == 0, nullptr);
    }
  }
  __syncthreads();   // this CTA's du and aux stores are visible to its own loads below
  float m[kPer], ex[kPer];
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < kPer / 4; ++q) {
    const float4 a = uq(0, q), b = uq(1, q);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      m[4 * q + e] = q_at(a, e) + q_at(b, e);
      s = d.alpha * s + d.beta * (m[4 * q + e] * m[4 * q + e]);
    }
  }
  float g = scan_fwd_excl(s, dec, dec + 32, P.carry[it.idx], sm);
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const float x = m[j] * m[j];
    ex[j] = g - x;
    g = d.alpha * g + d.beta * x;
  }
  float rl = 0.f;
#pragma unroll
  for (int q = kPer / 4 - 1; q >= 0; --q) {
    const float4 dg = load_quad(P.aux, n0 + 4 * q, L);
#pragma unroll
    for (int e = 3; e >= 0; --e) rl = q_at(dg, e) + d.alpha * rl;
  }
  float lam = scan_rev_excl(rl, dec, dec + 32, s_in, sm);   // lambda entering the last sample from the right
  float dalpha = 0.f;
#pragma unroll
  for (int q = kPer / 4 - 1; q >= 0; --q) {
    const int n = n0 + 4 * q;
    const float4 dg = load_quad(P.aux, n, L);
    const float4 a = tma ? stage_quad(dstage, 0, t, q) : load_quad(P.du, n, L);
    const float4 b = tma ? stage_quad(dstage, 1, t, q) : load_quad(P.du + ld, n, L);
    float dl[4] = {a.x, a.y, a.z, a.w}, dr[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int e = 3; e >= 0; --e) {
      const int j = 4 * q + e;
      lam = q_at(dg, e) + d.alpha * lam;
      dalpha += lam * ex[j];
      const float dx2m = d.beta * lam * 2.f * m[j];
      dl[e] += dx2m;
      dr[e] += dx2m;
    }
    if (n < L) {
      store_quad(P.du, n, L, dl[0], dl[1], dl[2], dl[3]);
      store_quad(P.du + ld, n, L, dr[0], dr[1], dr[2], dr[3]);
    }
  }
  float v[1] = {dalpha};
  float out[1];
  block_sum<1>(v, sm, out);
  if (t == 0) P.bpart[(size_t)it.idx * kNPart] = out[0];
}

void init_dyn_attributes() {
  cudaFuncSetAttribute(k_dyn_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynBwdSmem);
}

void launch_dyn_fwd(const LaunchCtx& c, const Item* items, int n) {
  if (!n) return;
  k_chain_begin<<<1, 1, 0, c.stream>>>(c.chain);
  k_dyn_fwd<<<n, kThreads, c.dyn_tma ? kDynFwdSmem : 0, c.stream>>>(c, items);   // no stage without maps
}
void launch_dyn_bwd(const LaunchCtx& c, const Item* items, int n) {
  if (!n) return;
  k_chain_begin<<<1, 1, 0, c.stream>>>(c.chain);
  k_dyn_bwd<<<n, kThreads, c.dyn_tma ? kDynBwdSmem : 0, c.stream>>>(c, items);
}

}  // namespace mg

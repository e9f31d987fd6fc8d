// Per-node reductions of the partial sums, the objective (Eqs. 20-23, 26), the final gradient assembly and
// Adam (Sec. 5.1).  All reductions run in a fixed order in double precision, so every song's result is
// independent of the batch it is computed in.
#include <algorithm>
#include "mg_fft.cuh"

namespace mg {

// One warp per processor: stats[0..1] = sums of the forward partials (LTI: E_ybar_mid, E_u_mid);
// stats[4..11] = sums of the backward partials.
__global__ void k_node_stats(LaunchCtx c, const int* __restrict__ procs, int n, int fwd) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= n) return;
  const ProcDev& P = c.procs[procs[w]];
  if (lane >= kNPart) return;
  const float* src = fwd ? P.fpart : P.bpart;
  const int rows = fwd ? P.nfpart : P.nbpart;
  if (src == nullptr) return;
  double s = 0.0;
  for (int r = 0; r < rows; ++r) s += (double)src[(size_t)r * kNPart + lane];
  if (fwd) {
    if (lane < 2) P.stats[lane] = (float)s;
  } else {
    P.stats[4 + lane] = (float)s;
  }
}

// One CTA per song.  mode 0: squared norms of the target spectrograms; mode 1: losses, backward
// coefficients and the gain-staging coefficients of every LTI node; mode 2: L_a only (pruning trials).
__global__ void __launch_bounds__(64) k_loss_finalize(LaunchCtx c, const SongDev* __restrict__ songs,
                                                      const LossRes* __restrict__ resv, int nres,
                                                      const float* __restrict__ alphas, int mode,
                                                      float* out_losses, float* out_la, int la_stride) {
  __shared__ double sums[3][6];
  const int si = blockIdx.x;
  const SongDev& S = songs[si];
  const int t = threadIdx.x;
  if (t < nres * 6) {
    const int r = t / 6, j = t % 6;
    double s = 0.0;
    for (int i = 0; i < S.litems[r]; ++i) s += (double)S.lpart[((size_t)r * S.lcap + i) * 6 + j];
    sums[r][j] = s;
  }
  __syncthreads();
  if (t != 0) return;
  if (mode == 0) {
    for (int r = 0; r < nres; ++r)
      for (int k = 0; k < 3; ++k) S.ynorm2[r * 3 + k] = sums[r][k];
    return;
  }
  double Lset[3] = {0.0, 0.0, 0.0};
  for (int r = 0; r < nres; ++r) {
    const int frames = S.nframes[r] - S.first_frame[r];
    if (frames <= 0) {
      for (int k = 0; k < 6; ++k) S.coef[r * 6 + k] = 0.f;
      continue;
    }
    for (int k = 0; k < 3; ++k) {
      const double cnt = (double)frames * resv[r].nbands * (k == 0 ? 2 : 1);
      const double yn = sqrt(S.ynorm2[r * 3 + k]);
      const double dn = sqrt(sums[r][2 * k + 1]);
      Lset[k] += sums[r][2 * k] / cnt + dn / yn;
      S.coef[r * 6 + 2 * k] = (float)(alphas[k] / cnt);
      S.coef[r * 6 + 2 * k + 1] = dn > 0.0 ? (float)(alphas[k] / (dn * yn)) : 0.f;
    }
  }
  const double La = alphas[0] * Lset[0] + alphas[1] * Lset[1] + alphas[2] * Lset[2];
  if (mode == 2) {
    out_la[si * la_stride] = (float)La;
    return;
  }
  double Lg = 0.0, Lp = 0.0;
  for (int i = S.pbeg; i < S.pend; ++i) {
    const ProcDev& P = c.procs[i];
    if (!P.present) continue;
    double w = 1.0 / (1.0 + exp(-(double)c.q[P.qidx]));
    if (c.mask) w *= (double)c.mask[P.qidx];
    Lp += w;
    if (P.type == T_E || P.type == T_R || P.type == T_D) {
      const double ey = P.stats[0], eu = P.stats[1];
      const double d = 0.5 * log(ey + 1e-12) - 0.5 * log(eu + 1e-12);
      Lg += fabs(d);
      const double sg = d > 0.0 ? 1.0 : (d < 0.0 ? -1.0 : 0.0);
      P.stats[2] = (float)(c.alpha_g * sg / (ey + 1e-12));
      P.stats[3] = (float)(-c.alpha_g * sg / (eu + 1e-12));
    }
  }
  const double ap = c.hyper[0];
  if (out_losses) {
    float* o = out_losses + si * 7;
    o[0] = (float)La;
    o[1] = (float)Lset[0];
    o[2] = (float)Lset[1];
    o[3] = (float)Lset[2];
    o[4] = (float)Lg;
    o[5] = (float)Lp;
    o[6] = (float)(La + c.alpha_g * Lg + ap * Lp);
  }
}

// Gradient assembly per processor from the backward sums (stats[4..]); dry/wet logit gradient
// dL/dq = (dL/dw + alpha_p) sigmoid'(q).
__global__ void k_grad_finalize(LaunchCtx c, const int* __restrict__ procs, int n, float* __restrict__ gq) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const ProcDev& P = c.procs[procs[i]];
  const float wr = 1.f / (1.f + expf(-c.q[P.qidx]));
  const float* s = P.stats + 4;
  float dw = 0.f;
  switch (P.type) {
    case T_G: {
      const float el = expf(P.p[0]), er = expf(P.p[1]);
      P.gp[0] = wr * el * s[0];
      P.gp[1] = wr * er * s[1];
      dw = (el - 1.f) * s[0] + (er - 1.f) * s[1];
      break;
    }
    case T_S: {
      const float e = expf(P.p[0]);
      P.gp[0] = wr * e * 0.5f * s[0];
      dw = (e - 1.f) * 0.5f * s[0];
      break;
    }
    case T_C:
    case T_N: {
      const float a = 1.f / (1.f + expf(-P.p[0])), b = 1.f / (1.f + expf(P.p[0]));   // sigmoid(p0), 1 - sigmoid(p0)
      P.gp[0] = s[0] * a * b;
      P.gp[1] = s[1];
      P.gp[2] = s[2] * expf(P.p[2]);
      P.gp[3] = s[3] * expf(P.p[3]);
      dw = s[4];
      break;
    }
    default:
      dw = s[0];   // LTI: dL/dw from the y_bar pass; FIR parameter gradients come from the adjoint kernels
  }
  gq[P.qidx] = (dw + c.hyper[0]) * wr / (1.f + expf(c.q[P.qidx]));   // w (1 - w), 1 - w = sigmoid(-q)
}

__global__ void k_adam(const float* __restrict__ hyper, const int* __restrict__ step, float* __restrict__ p,
                       const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v, int64_t n) {
  const float lr = hyper[1], b1 = hyper[2], b2 = hyper[3], eps = hyper[4], wd = hyper[5];
  const int t = *step + 1;
  const float bc1 = 1.f - powf(b1, (float)t), bc2 = 1.f - powf(b2, (float)t);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float pi = p[i];
    const float gi = g[i];
    pi -= lr * wd * pi;
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] = pi - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  }
}

__global__ void k_adam_tick(int* step) { *step += 1; }

__global__ void k_set_hyper(float* hyper, float a0, float a1, float a2, float a3, float a4, float a5, int which) {
  if (which == 0) {
    hyper[0] = a0;
  } else {
    hyper[1] = a1;
    hyper[2] = a2;
    hyper[3] = a3;
    hyper[4] = a4;
    hyper[5] = a5;
  }
}

void launch_node_stats(const LaunchCtx& c, const int* procs, int n, int fwd) {
  if (n) k_node_stats<<<(n * 32 + 255) / 256, 256, 0, c.stream>>>(c, procs, n, fwd);
}
void launch_loss_finalize_mode(const LaunchCtx& c, const SongDev* songs, int nsongs, const LossRes* res, int nres,
                               const float* alphas, int mode, float* out_losses, float* out_la, int la_stride) {
  if (nsongs) k_loss_finalize<<<nsongs, 64, 0, c.stream>>>(c, songs, res, nres, alphas, mode, out_losses, out_la, la_stride);
}
void launch_grad_finalize2(const LaunchCtx& c, const int* procs, int n, float* gq) {
  if (n) k_grad_finalize<<<(n + 127) / 128, 128, 0, c.stream>>>(c, procs, n, gq);
}
void launch_adam2(cudaStream_t st, const float* hyper, int* step, float* p, const float* g, float* m, float* v,
                  int64_t n) {
  if (n) {
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    k_adam<<<blocks, 256, 0, st>>>(hyper, step, p, g, m, v, n);
  }
  k_adam_tick<<<1, 1, 0, st>>>(step);
}
void launch_set_hyper(cudaStream_t st, float* hyper, float alpha_p, float lr, float b1, float b2, float eps, float wd,
                      int which) {
  k_set_hyper<<<1, 1, 0, st>>>(hyper, alpha_p, lr, b1, b2, eps, wd, which);
}

// Candidate scoring: the dry/wet logit of every forward-only node copy, gathered from the processor it copies
// (the copies carry their own mask values and index these by their own position).
__global__ void k_gather_q(const float* __restrict__ q, const int* __restrict__ src, float* __restrict__ dst, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = q[src[i]];
}
void launch_gather_q(cudaStream_t st, const float* q, const int* src, float* dst, int n) {
  if (n) k_gather_q<<<(n + 255) / 256, 256, 0, st>>>(q, src, dst, n);
}

// Candidate scoring: out[j][s] = L_a of the copy of song s that candidate j changed (map >= 0), else the song's
// L_a under the base mask.
__global__ void k_score_scatter(const int* __restrict__ map, const float* __restrict__ vla,
                                const float* __restrict__ base_la, float* __restrict__ out, int n, int nsongs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = map[i] >= 0 ? vla[map[i]] : base_la[i % nsongs];
}
void launch_score_scatter(cudaStream_t st, const int* map, const float* vla, const float* base_la, float* out, int n,
                          int nsongs) {
  if (n) k_score_scatter<<<(n + 255) / 256, 256, 0, st>>>(map, vla, base_la, out, n, nsongs);
}

}  // namespace mg

// Allocation-free equalizer forward for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside another framework's memory pool or allocator
// hooks, plug-in hosts that forbid device allocations on their audio threads, or work already recorded on a
// stream where an allocation would synchronise the device.  mg_eq_forward_noalloc gives them one processor
// of the console (the zero-phase FIR equalizer followed by the dry/wet blend) with no allocation at all: the
// FIR taps, the FFT scratch, the node table and the lookup tables live in one file-scope __device__ array of
// fixed size (about 3.3 MB) that every GPU which loads this library keeps until the process exits.  The
// console's four-step FFT convolution kernels (those of the reverb and delay stages) do the work.
#include <algorithm>
#include <mutex>

#include "../../include/mixgraph.h"
#include "mg_fftp.cuh"

namespace mg {
namespace {

constexpr int kNaLogN = 17;                  // largest FFT: 2^17 points
constexpr int kNaN = 1 << kNaLogN;
constexpr int kNaLogN1 = (kNaLogN + 1) / 2;  // 512 columns
constexpr int kNaLogN2 = kNaLogN / 2;        // 256 rows
constexpr int kNaMaxCol = (1 << kNaLogN1);   // column groups (at most N1 / G with G >= 1)
constexpr int kNaMaxRow = (1 << kNaLogN2);
// the FFT must hold the signal plus the 2047-tap FIR without wrap-around: L + 2047 + 1023 + 1 <= N
constexpr int64_t kNaMaxSamples = kNaN - kEqTaps - kEqHalf - 1;

struct NaLayout {
  float2 fft[3 * kNaN];                      // T1, T2, Hz
  float2 tw[kTwN];
  float2 twf[kTwN];                          // exp(-2 pi i j / 2^26): fine factor of the four-step twiddles
  float2 ptw[kPtwCount];                     // pass twiddles of the row and column FFTs
  float cos_eq[kEqTaps];
  float hann_eq[kEqTaps];
  float taps[2 * kEqTaps];
  float stats[kStatsFloats];                 // the channel scales stay 0 here: the transforms use scale 1
  float fpart[kNaMaxCol * kNPart];
  float hyper[8];
  ProcDev proc;
  int proc_list[4];
  Item col_items[kNaMaxCol];
  Item pair_items[kNaMaxRow / 2 + 1];
};

constexpr size_t kNaFloat2s = (sizeof(NaLayout) + sizeof(float2) - 1) / sizeof(float2);

// The scratch of mg_eq_forward_noalloc.  Host code must not use this name as an address (it is a host-side
// stand-in); it obtains the device address with cudaGetSymbolAddress.
static __device__ __align__(256) float2 g_noalloc_scratch[kNaFloat2s];

// Twiddles and cosine / window tables, computed once per device in double precision.
__global__ void k_na_tables() {
  NaLayout* S = reinterpret_cast<NaLayout*>(g_noalloc_scratch);
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  for (int j = t; j < kTwN; j += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * j / kTwN, &s, &c);
    S->tw[j] = make_float2((float)c, (float)-s);
    sincospi(2.0 * j / (double)(1 << kTwFineLog), &s, &c);
    S->twf[j] = make_float2((float)c, (float)-s);
  }
  for (int e = t; e < kPtwCount; e += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * ptw_source(e) / kTwN, &s, &c);
    S->ptw[e] = make_float2((float)c, (float)-s);
  }
  for (int m = t; m < kEqTaps; m += gridDim.x * blockDim.x) {
    S->cos_eq[m] = (float)cospi(2.0 * m / kEqTaps);
    S->hann_eq[m] = (float)(0.5 * (1.0 + cospi((double)(m - kEqHalf) / kEqHalf)));
  }
}

// Node table and work lists of one call, written on the device (no host-to-device copies).
__global__ void k_na_prep(const float* u, float* y, const float* params, int L, int logN, int logN1, int logN2, int G) {
  NaLayout* S = reinterpret_cast<NaLayout*>(g_noalloc_scratch);
  const int t = threadIdx.x;
  const int N1 = 1 << logN1, N2 = 1 << logN2;
  if (t == 0) {
    ProcDev d{};
    d.type = T_E;
    d.qidx = 0;
    d.present = 1;
    d.rev = -1;
    d.L = L;
    d.ld = L;
    d.u = u;
    d.y = y;
    d.p = params;
    d.stats = S->stats;
    d.fpart = S->fpart;
    d.nfpart = N1 / G;
    d.logN = logN;
    d.logN1 = logN1;
    d.logN2 = logN2;
    d.f = 1;
    d.colG = G;
    d.n0 = -kEqHalf;
    d.Nh = kEqTaps;
    d.T1 = S->fft;
    d.T2 = S->fft + ((size_t)1 << logN);
    d.Hz = S->fft + ((size_t)2 << logN);
    d.taps = S->taps;
    S->proc = d;
    S->proc_list[0] = 0;
  }
  for (int i = t; i < N1 / G; i += blockDim.x) S->col_items[i] = Item{0, i};
  for (int i = t; i <= N2 / 2; i += blockDim.x) S->pair_items[i] = Item{0, i};
}

struct DeviceScratch {
  NaLayout* ptr = nullptr;   // address the tables were built at (null: not built yet)
};
std::mutex g_na_mutex;
DeviceScratch g_na_dev[64];

}  // namespace
}  // namespace mg

using namespace mg;

extern "C" mg_status mg_eq_forward_noalloc(const float* d_u, float* d_y, int64_t num_samples, const float* d_params,
                                           cudaStream_t stream) {
  if (!d_u || !d_y || !d_params) return MG_ERR_INVALID;
  if (num_samples < 1 || num_samples > kNaMaxSamples) return MG_ERR_UNSUPPORTED;
  // An error left pending by earlier work on this thread would be indistinguishable from this call's own
  // launch errors below: refuse to launch, and leave it in place for its owner.
  if (cudaPeekAtLastError() != cudaSuccess) return MG_ERR_CUDA;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return MG_ERR_CUDA;
  NaLayout* S = nullptr;
  {
    // The symbol's device address is looked up on every call (the lookup allocates nothing): if the module was
    // reloaded (a device reset, a new context) the array may have moved and lost its tables, which are then
    // rebuilt.  Building them synchronises the stream, so the first call on a device comes before any capture.
    std::lock_guard<std::mutex> lock(g_na_mutex);
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return MG_ERR_CUDA;
    DeviceScratch& ds = g_na_dev[dev];
    if (ds.ptr != reinterpret_cast<NaLayout*>(p)) {
      ds.ptr = nullptr;
      init_kernel_attributes();
      k_na_tables<<<16, 256, 0, stream>>>();
      if (cudaGetLastError() != cudaSuccess) return MG_ERR_CUDA;
      if (cudaStreamSynchronize(stream) != cudaSuccess) return MG_ERR_CUDA;
      ds.ptr = reinterpret_cast<NaLayout*>(p);
    }
    S = ds.ptr;
  }
  const int L = (int)num_samples;
  int logN = 12;
  while (((int64_t)1 << logN) < (int64_t)L + kEqTaps + kEqHalf + 1) ++logN;
  const int logN1 = (logN + 1) / 2, logN2 = logN / 2;
  const int G = std::min(8, std::min(8192 >> logN2, 1 << logN1));
  const int N1 = 1 << logN1, N2 = 1 << logN2;
  k_na_prep<<<1, 256, 0, stream>>>(d_u, d_y, d_params, L, logN, logN1, logN2, G);

  LaunchCtx x{};
  x.stream = stream;
  x.procs = &S->proc;
  x.q = d_params + kEqParams;            // the dry/wet logit follows the 1024 log-magnitudes
  x.mask = nullptr;
  x.hyper = S->hyper;
  x.alpha_g = 0.f;
  x.fs = 0.0;
  x.tab.tw = S->tw;
  x.tab.twf = S->twf;
  x.tab.ptw = S->ptw;
  x.tab.cos_eq = S->cos_eq;
  x.tab.hann_eq = S->hann_eq;
  launch_eq_fir(x, S->proc_list, 1);
  launch_col_fwd_taps(x, S->col_items, N1 / G, N2 * G);
  launch_row_fwd_hz(x, S->pair_items, N2 / 2 + 1, N1);
  launch_col_fwd_audio(x, S->col_items, N1 / G, N2 * G);
  launch_row_conv_fwd(x, S->pair_items, N2 / 2 + 1, N1, false);
  launch_col_inv_out(x, S->col_items, N1 / G, N2 * G);
  // no error was pending on entry, so whatever is pending now came from these launches
  return cudaGetLastError() == cudaSuccess ? MG_OK : MG_ERR_CUDA;
}

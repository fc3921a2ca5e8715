// bte_peak.cu -- arithmetic peaks of the current GPU, measured by FMA loops.
//
// The FP64-mode sweep is measured against the FP64 pipe's rate and its
// double-float form against the FP32 pipe's rate; neither is in a vendor table
// one can trust for a given part and clock, so the library measures them:
// every thread runs kChains independent FMA chains (enough to cover the
// pipe's latency at the occupancy of 8 CTAs of 256 threads per SM), the
// kernel is timed with CUDA events, and the best of three launches is
// returned as flop/s (2 flop per FMA; a packed f32x2 FMA is two FMAs).  The
// result depends on the SM clock during the launches; the caller samples it.
#include "../../include/bte.h"
#include "bte_internal.h"

namespace bte {
namespace {

constexpr int kChains = 8;
static __device__ double g_peak_sink;  // keeps the loops' results alive without a device allocation

__global__ void dfma_loop_kernel(int n, double s) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = 1.0 + 1e-3 * (threadIdx.x + c);
  for (int i = 0; i < n; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], s, 0.5);
  double r = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) r += a[c];
  if (r == -1.0) g_peak_sink = r;  // never true for s in (0, 1): the sum stays positive
}

__global__ void ffma2_loop_kernel(int n, float s) {
  unsigned long long a[kChains];
  unsigned long long sv, hv;
  asm("mov.b64 %0, {%1, %1};" : "=l"(sv) : "f"(s));
  asm("mov.b64 %0, {%1, %1};" : "=l"(hv) : "f"(0.5f));
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    const float x = 1.0f + 1e-3f * (threadIdx.x + c);
    asm("mov.b64 %0, {%1, %1};" : "=l"(a[c]) : "f"(x));
  }
  for (int i = 0; i < n; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[c]) : "l"(sv), "l"(hv));
  float r = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    float x, y;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a[c]));
    r += x + y;
  }
  if (r == -1.0f) g_peak_sink = r;
}

}  // namespace
}  // namespace bte

using namespace bte;

extern "C" int bte_measure_peak(int kind, double* flops, double* ms) {
  if (!flops || (kind != BTE_PEAK_FP64_FMA && kind != BTE_PEAK_FP32X2_FMA)) return BTE_E_ARG;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess || sms <= 0) return BTE_E_CUDA;
  const int threads = 256, grid = 8 * sms;
  // about 30 ms per launch on a GB300-class part (FP64 FMA runs at 1/64 of the FP32 rate there)
  const int n = kind == BTE_PEAK_FP64_FMA ? 8192 : 262144;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first launch warms up, the best of the rest counts
    e = cudaEventRecord(e0, s);
    if (kind == BTE_PEAK_FP64_FMA) dfma_loop_kernel<<<grid, threads, 0, s>>>(n, 0.999);
    else ffma2_loop_kernel<<<grid, threads, 0, s>>>(n, 0.999f);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e == cudaSuccess && rep > 0 && t < best) best = t;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (e != cudaSuccess) return BTE_E_CUDA;
  const double fmas = (double)grid * threads * (double)n * kChains * (kind == BTE_PEAK_FP64_FMA ? 1.0 : 2.0);
  *flops = 2.0 * fmas / (best * 1e-3);
  if (ms) *ms = best;
  return BTE_OK;
}

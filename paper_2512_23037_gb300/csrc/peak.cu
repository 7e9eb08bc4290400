// peak.cu -- issue-rate peaks of the arithmetic pipes the shot kernels use, for
// their roofline denominators (the FP64 path is bound by GB300's narrow FP64
// pipe, for which no vendor figure is measured here).
//
// Each thread runs kChains independent dependency chains of one instruction
// kind (FP64 FMA, FP32 FMA, or a 32-bit three-input logic op), kUnroll steps
// per loop trip, with operands the compiler cannot fold; the chains' sum is
// stored only if it equals an impossible value, so nothing is dead code.
// A grid of 4 blocks of 256 threads per SM keeps every pipe's queue full.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "../../include/soft_peak.h"
#include "handles.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;

template <int Kind>
__global__ void __launch_bounds__(kThreads) pipe_kernel(uint32_t trips, double bd, double cd, float bf, float cf,
                                                        uint32_t bi, uint32_t ci, double *sink) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (Kind == SOFT_PEAK_FP64_FMA) {
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1e-9 * (double)t + (double)k;
#pragma unroll 1
    for (uint32_t it = 0; it < trips; ++it)
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], bd, cd);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == -12345.0) sink[0] = s;
  } else if (Kind == SOFT_PEAK_FP32_FMA) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1e-9f * (float)t + (float)k;
#pragma unroll 1
    for (uint32_t it = 0; it < trips; ++it)
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], bf, cf);
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == -12345.0f) sink[0] = (double)s;
  } else {
    uint32_t a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = t * 2654435761u + (uint32_t)k;
#pragma unroll 1
    for (uint32_t it = 0; it < trips; ++it)
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = (a[k] & bi) ^ (ci + (uint32_t)u);  // one three-input op
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s ^= a[k];
    if (s == 0x9E3779B9u && bi == 0u) sink[0] = (double)s;
  }
}

// loop trips per launch (a launch of a few to a few tens of milliseconds on GB300)
uint32_t trips_for(int kind) { return kind == SOFT_PEAK_FP64_FMA ? 512u : 16384u; }

}  // namespace

extern "C" int soft_peak_pipe_rate(int32_t kind, void *stream, double *ops_per_s, double *ms_per_launch) {
  if (!ops_per_s || kind < SOFT_PEAK_FP64_FMA || kind > SOFT_PEAK_INT32_LOGIC)
    return soft::set_error(SOFT_E_ARG, "bad argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return soft::set_error(SOFT_E_CUDA, cudaGetErrorString(e));
  const unsigned grid = (unsigned)(sms * kBlocksPerSm);
  const uint32_t trips = trips_for(kind);
  // the sink is written only on an impossible value: a null pointer is never dereferenced
  double *sink = nullptr;
  auto launch = [&]() {
    if (kind == SOFT_PEAK_FP64_FMA)
      pipe_kernel<SOFT_PEAK_FP64_FMA><<<grid, kThreads, 0, st>>>(trips, 0.999999, 1e-7, 0.f, 0.f, 0u, 0u, sink);
    else if (kind == SOFT_PEAK_FP32_FMA)
      pipe_kernel<SOFT_PEAK_FP32_FMA><<<grid, kThreads, 0, st>>>(trips, 0.0, 0.0, 0.9999f, 1e-4f, 0u, 0u, sink);
    else
      pipe_kernel<SOFT_PEAK_INT32_LOGIC><<<grid, kThreads, 0, st>>>(trips, 0.0, 0.0, 0.f, 0.f, 0x7FFFFFFFu,
                                                                      0x12345u, sink);
    return cudaGetLastError();
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return soft::set_error(SOFT_E_CUDA, cudaGetErrorString(e));
  }
  float best = 0.f;
  for (int r = 0; r < 7 && e == cudaSuccess; ++r) {  // two warm-up launches, then the best of five
    if ((e = cudaEventRecord(e0, st)) != cudaSuccess || (e = launch()) != cudaSuccess ||
        (e = cudaEventRecord(e1, st)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess)
      break;
    float f = 0.f;
    if ((e = cudaEventElapsedTime(&f, e0, e1)) != cudaSuccess) break;
    if (r >= 2 && (best == 0.f || f < best)) best = f;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return soft::set_error(SOFT_E_CUDA, cudaGetErrorString(e));
  const double per_op = kind == SOFT_PEAK_INT32_LOGIC ? 1.0 : 2.0;  // an FMA counts as two flops
  const double ops = per_op * (double)grid * kThreads * kChains * kUnroll * trips;
  *ops_per_s = ops / ((double)best * 1e-3);
  if (ms_per_launch) *ms_per_launch = (double)best;
  return SOFT_OK;
}

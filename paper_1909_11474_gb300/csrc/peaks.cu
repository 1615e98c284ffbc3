// peaks.cu -- arithmetic throughput microbenchmarks of the device: the denominators (and their
// cross-checks) of the roofline figures the benchmark reports. Each kernel runs independent dependency
// chains in every thread of a grid that fills every SM, long enough (milliseconds) for launch overhead
// to vanish, and is timed with CUDA events; the rate is (operations executed) / (elapsed time).
//  - FP32 FMA:  8 chains a = a * b + c per thread (one FFMA each), counted as 2 FLOP per FMA;
//  - FP32x2:    the packed two-lane FMA (__ffma2_rn), 4 FLOP per instruction;
//  - FP64 FMA:  8 chains of fma(double), 2 FLOP per FMA;
//  - FP64 add:  8 chains of double additions, 1 op each;
//  - XU:        8 chains x = 2^x * c on the special-function unit (ex2.approx), 1 op per ex2 (the FP32
//               multiply runs on the FMA pipe beside it);
//  - F32<->F64: 8 chains f = (float)(double)f (one conversion each way), 2 conversions per link.
// The values feed nothing but the measurement: each chain's end value is written out so that the
// compiler keeps the work.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "ctx.hpp"

namespace tsf {

constexpr int kPeakThreads = 256;
constexpr int kChains = 8;

enum PeakOp { kOpFfma = 0, kOpFfma2 = 1, kOpDfma = 2, kOpDadd = 3, kOpEx2 = 4, kOpCvt = 5 };

template <int OP>
__global__ void __launch_bounds__(kPeakThreads) peak_kernel(int iters, float fb, float fc, double *out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double sink = 0.0;
  if constexpr (OP == kOpFfma) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1.0f + 1e-3f * (float)(t + k);
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = __fmaf_rn(a[k], fb, fc);
#pragma unroll
    for (int k = 0; k < kChains; ++k) sink += a[k];
  } else if constexpr (OP == kOpFfma2) {
    float2 a[kChains];
    const float2 b = make_float2(fb, fb), c = make_float2(fc, fc);
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = make_float2(1.0f + 1e-3f * (float)(t + k), 1.0f - 1e-3f * (float)k);
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = __ffma2_rn(a[k], b, c);
#pragma unroll
    for (int k = 0; k < kChains; ++k) sink += a[k].x + a[k].y;
  } else if constexpr (OP == kOpDfma) {
    double a[kChains];
    const double b = fb, c = fc;
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1.0 + 1e-3 * (double)(t + k);
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
#pragma unroll
    for (int k = 0; k < kChains; ++k) sink += a[k];
  } else if constexpr (OP == kOpDadd) {
    double a[kChains];
    const double c = fc;
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1.0 + 1e-3 * (double)(t + k);
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = __dadd_rn(a[k], c);
#pragma unroll
    for (int k = 0; k < kChains; ++k) sink += a[k];
  } else if constexpr (OP == kOpEx2) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 0.5f + 1e-4f * (float)k;
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = ex2(a[k]) * fc;   // fc < 1/2 keeps the chain in (0, 1)
#pragma unroll
    for (int k = 0; k < kChains; ++k) sink += a[k];
  } else {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1.0f + 1e-3f * (float)(t + k);
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int k = 0; k < kChains; ++k) {
        double d;
        asm volatile("cvt.f64.f32 %0, %1;" : "=d"(d) : "f"(a[k]));
        asm volatile("cvt.rn.f32.f64 %0, %1;" : "=f"(a[k]) : "d"(d));
      }
#pragma unroll
    for (int k = 0; k < kChains; ++k) sink += a[k];
  }
  if (sink == 1234.5678) out[t] = sink;   // practically never true; keeps the chains live
}

// Runs one microbenchmark: returns operations per second (FLOP/s for the FMA kinds) or a negative
// value on a CUDA error.
template <int OP>
static double run_peak(int nsm, int iters, double ops_per_chain_link, double *sink) {
  const int blocks = nsm * (2048 / kPeakThreads);
  const float fb = 0.999999f, fc = OP == kOpEx2 ? 0.4f : 1e-6f;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -1.0;
  float best = 3.4e38f;
  bool ok = true;
  for (int r = 0; r < 4 && ok; ++r) {   // the first launch warms up
    ok = cudaEventRecord(e0) == cudaSuccess;
    peak_kernel<OP><<<blocks, kPeakThreads>>>(iters, fb, fc, sink);
    ok = ok && launched(1) == cudaSuccess && cudaEventRecord(e1) == cudaSuccess &&
         cudaEventSynchronize(e1) == cudaSuccess;
    float ms = 0.f;
    ok = ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    if (ok && r > 0) best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok) return -1.0;
  const double ops = (double)blocks * kPeakThreads * (double)iters * kChains * ops_per_chain_link;
  return ops / (1e-3 * (double)best);
}

}  // namespace tsf

extern "C" int tersoff_measure_peaks(int32_t device, double *out) {
  if (!out) return TERSOFF_E_ARG;
  int cur = 0, n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return TERSOFF_E_ARG;
  if (cudaGetDevice(&cur) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) return TERSOFF_E_CUDA;
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
  double *sink = nullptr;
  const int threads = nsm * 2048;
  int rc = TERSOFF_OK;
  if (cudaMalloc(&sink, (size_t)threads * sizeof(double)) != cudaSuccess) rc = TERSOFF_E_CUDA;
  if (rc == TERSOFF_OK) {
    out[0] = tsf::run_peak<tsf::kOpFfma>(nsm, 4096, 2.0, sink);
    out[1] = tsf::run_peak<tsf::kOpFfma2>(nsm, 2048, 4.0, sink);
    out[2] = tsf::run_peak<tsf::kOpDfma>(nsm, 64, 2.0, sink);
    out[3] = tsf::run_peak<tsf::kOpDadd>(nsm, 64, 1.0, sink);
    out[4] = tsf::run_peak<tsf::kOpEx2>(nsm, 1024, 1.0, sink);
    out[5] = tsf::run_peak<tsf::kOpCvt>(nsm, 64, 2.0, sink);
    for (int k = 0; k < 6; ++k)
      if (out[k] < 0.0) rc = TERSOFF_E_CUDA;
  }
  if (sink) cudaFree(sink);
  cudaSetDevice(cur);
  return rc;
}

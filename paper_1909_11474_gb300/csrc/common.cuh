// common.cuh -- device helpers shared by the kernels of the minimal-Tersoff library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tersoff.h"
#include "ctx.hpp"

namespace tsf {

constexpr int kWarp = 32;

// ---------------------------------------------------------------------------------------------
// Transcendentals. FP32 uses the SFU (MUFU) instructions directly through PTX; FP64 calls the
// CUDA math library. exp(x) = 2^(x log2 e) is formed by the callers, which fold log2 e into the
// per-parameter-set constants.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ double ex2(double x) { return exp2(x); }
__device__ __forceinline__ double lg2(double x) { return log2(x); }
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }

template <typename R>
struct Vec4;
template <>
struct Vec4<float> {
  using T = float4;
};
template <>
struct Vec4<double> {
  using T = dvec4;
};

__device__ __forceinline__ void set_status(unsigned *status, unsigned bit) {
  if (status) atomicOr(status, bit);
}

// Sums over the lanes of one warp that share `lane % PT` (the lanes handling the same parameter
// set): xor-shuffle over the atom-slot bits of the lane index.
template <int PT, typename T>
__device__ __forceinline__ T sum_over_atom_slots(T v) {
#pragma unroll
  for (int off = PT; off < kWarp; off <<= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

}  // namespace tsf

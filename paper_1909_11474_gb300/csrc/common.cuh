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

// Programmatic dependent launch: a kernel launched with programmatic stream serialization may start
// before its predecessor in the stream has finished; it waits here before reading that predecessor's
// results. The predecessor lets its dependents launch early with pdl_trigger. Both are no-ops for a
// kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ void set_status(unsigned *status, unsigned bit) {
  if (status) atomicOr(status, bit);
}

// Exact FP64 membership test of the neighbour sets (Eq. 2, 7):
//   d = (x_j - x_i) + ((n0 a + n1 b) + n2 c),  r^2 = (dx^2 + dy^2) + dz^2,
// every operation individually rounded (no contraction into FMA), so the decision r^2 < R2^2 is
// reproducible bit for bit by any FP64 implementation that evaluates the same expression.
struct ExactPair {
  double dx, dy, dz, r2;
};
__device__ __forceinline__ ExactPair exact_pair(double xjx, double xjy, double xjz, double xix,
                                                double xiy, double xiz, const double *H, int n0,
                                                int n1, int n2) {
  double f0 = (double)n0, f1 = (double)n1, f2 = (double)n2;
  double tx = __dadd_rn(__dadd_rn(__dmul_rn(f0, H[0]), __dmul_rn(f1, H[3])), __dmul_rn(f2, H[6]));
  double ty = __dadd_rn(__dadd_rn(__dmul_rn(f0, H[1]), __dmul_rn(f1, H[4])), __dmul_rn(f2, H[7]));
  double tz = __dadd_rn(__dadd_rn(__dmul_rn(f0, H[2]), __dmul_rn(f1, H[5])), __dmul_rn(f2, H[8]));
  ExactPair e;
  e.dx = __dadd_rn(__dsub_rn(xjx, xix), tx);
  e.dy = __dadd_rn(__dsub_rn(xjy, xiy), ty);
  e.dz = __dadd_rn(__dsub_rn(xjz, xiz), tz);
  e.r2 = __dadd_rn(__dadd_rn(__dmul_rn(e.dx, e.dx), __dmul_rn(e.dy, e.dy)), __dmul_rn(e.dz, e.dz));
  return e;
}


// FP32 -> FP64, exact, built from the IEEE-754 binary32 and binary64 layouts with integer operations
// (sign kept, exponent rebiased from 127 to 1023, significand shifted left by 29), so that the
// conversions of per-warp partial sums do not queue on the device's scarce FP64 unit. Zeros take the
// same path; subnormal, infinite and NaN inputs (which partial sums of finite terms do not produce in
// practice) are converted by the FP64 unit.
__device__ __forceinline__ double widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if ((e == 0u && (u << 1) != 0u) || e == 0xffu) return (double)f;
  const unsigned hi = (u & 0x80000000u) | (e == 0u ? 0u : ((e + 896u) << 20)) | ((u >> 3) & 0xfffffu);
  return __hiloint2double((int)hi, (int)(u << 29));
}
__device__ __forceinline__ double widen(double d) { return d; }

// Sums over the lanes of one warp that share `lane % PT` (the lanes handling the same parameter
// set): xor-shuffle over the atom-slot bits of the lane index.
template <int PT, typename T>
__device__ __forceinline__ T sum_over_atom_slots(T v) {
#pragma unroll
  for (int off = PT; off < kWarp; off <<= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

}  // namespace tsf

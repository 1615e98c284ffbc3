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


// x (FP64) as FP32 head + tail, by integer operations on the binary64 layout (the device's FP64 unit is
// slow): the head keeps the top 24 bits of the significand (truncated), the tail is the remaining 29
// bits converted to FP32 with one rounding, so |x - head - tail| <= 2^-48 |x|. |x| < 2^-60 gives
// head = tail = 0 (off by less than 2^-60). Returns false for |x| > 2^60 and non-finite x, which the
// caller takes through FP64 arithmetic.
__device__ __forceinline__ bool split_f64(double x, float &hi, float &lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ffu) - 1023;
  hi = 0.f;
  lo = 0.f;
  if (e < -60) return true;
  if (e > 60) return false;
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const unsigned long long mant = b & 0xfffffffffffffull;
  hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | (unsigned)(mant >> 29));
  const float scale = __uint_as_float((unsigned)(e - 52 + 127 + 64) << 23);   // 2^(e - 52 + 64)
  lo = __uint_as_float(__float_as_uint(__uint2float_rn((unsigned)(mant & 0x1fffffffu)) * scale) ^ sign) *
       0x1p-64f;
  return true;
}

// s + t = a + b exactly (FP32 two-sum, six additions).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &t) {
  s = a + b;
  const float bb = s - a;
  t = (a - (s - bb)) + (b - bb);
}

// Component k of the bond vector d = x_j - x_i + n H from FP32 head + tail pairs of the positions
// (split_f64) and of the box rows (H_a = h_a + l_a): the head difference and the head products n_a h_a
// (exact by FMA; n_a is a small integer) are summed by two-sum, every rounding error and tail goes to
// a running tail, and head + tail is rounded once at the end. The result is within ~2^-45 of
// max(|x|, |n H|) of the exact value, so it equals the FP64 vector rounded to FP32 except where that
// value lies within this distance of a rounding boundary.
__device__ __forceinline__ float bond_component(float xjh, float xjl, float xih, float xil, float n0, float n1,
                                                float n2, float h0, float l0, float h1, float l1, float h2,
                                                float l2) {
  float s, t;
  two_sum(xjh, -xih, s, t);
  float lo = t + (xjl - xil);
  const float n[3] = {n0, n1, n2}, h[3] = {h0, h1, h2}, l[3] = {l0, l1, l2};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float p = n[a] * h[a];
    const float e = __fmaf_rn(n[a], h[a], -p);
    two_sum(s, p, s, t);
    lo += (t + e) + n[a] * l[a];
  }
  return s + lo;
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

// Sum of N FP32 values rounded once to FP64, by integer arithmetic (the device's FP64 unit does one
// conversion): each value becomes a 64-bit fixed-point integer aligned to the largest exponent (its
// leading bit at bit 57, so N <= 16 values cannot overflow), the integers are added exactly, and the
// sum is converted and rescaled by a power of two. The result is the exact sum rounded to FP64,
// except that bits of a value lying more than 2^34 below the largest value's last bit are dropped
// (an error below 2^-57 of the largest value) -- at least as accurate as FP64 recursive summation,
// which rounds at every step. Subnormal values take part; an infinite or NaN value makes the sum an
// FP64 sum of the widened values, which propagates it.
template <int N>
__device__ __forceinline__ double exact_sum(const float (&x)[N]) {
  static_assert(N >= 1 && N <= 16, "fixed-point headroom");
  unsigned u[N];
  int emax = 1;
  bool special = false;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    u[k] = __float_as_uint(x[k]);
    const int e = (int)((u[k] >> 23) & 0xffu);
    special = special || e == 0xff;
    emax = max(emax, e);
  }
  if (special) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < N; ++k) s += (double)x[k];
    return s;
  }
  long long acc = 0;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    int e = (int)((u[k] >> 23) & 0xffu);
    unsigned m = u[k] & 0x7fffffu;
    if (e != 0) m |= 0x800000u;
    else e = 1;                                   // subnormal: no implicit bit, exponent 1
    const int sh = emax - e;
    const unsigned long long v = sh >= 64 ? 0ull : ((unsigned long long)m << 34) >> sh;
    acc += (u[k] >> 31) ? -(long long)v : (long long)v;
  }
  if (acc == 0) return 0.0;
  // acc * 2^(emax - 127 - 23 - 34): the power of two added to the exponent field (no overflow or
  // underflow: |acc| < 2^62 and emax is in [1, 254])
  const long long bits = __double_as_longlong(__ll2double_rn(acc)) + ((long long)(emax - 184) << 52);
  return __longlong_as_double(bits);
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

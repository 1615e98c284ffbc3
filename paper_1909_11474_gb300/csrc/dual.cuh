// dual.cuh -- forward-mode dual numbers for the parameter gradient: a value and K tangents, with the
// arithmetic and the transcendentals (2^x, log2 x, 1/x) used by the per-atom core of the potential.
#pragma once

#include "common.cuh"

namespace tsf {

template <int K, typename R>
struct Dual {
  R v;
  R d[K];
  __device__ __forceinline__ Dual() {}
  __device__ __forceinline__ Dual(R x) : v(x) {
#pragma unroll
    for (int k = 0; k < K; ++k) d[k] = R(0);
  }
};

#define TSF_DUAL template <int K, typename R> __device__ __forceinline__

TSF_DUAL Dual<K, R> operator+(const Dual<K, R> &a, const Dual<K, R> &b) {
  Dual<K, R> o;
  o.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < K; ++k) o.d[k] = a.d[k] + b.d[k];
  return o;
}
TSF_DUAL Dual<K, R> operator-(const Dual<K, R> &a, const Dual<K, R> &b) {
  Dual<K, R> o;
  o.v = a.v - b.v;
#pragma unroll
  for (int k = 0; k < K; ++k) o.d[k] = a.d[k] - b.d[k];
  return o;
}
TSF_DUAL Dual<K, R> operator-(const Dual<K, R> &a) {
  Dual<K, R> o;
  o.v = -a.v;
#pragma unroll
  for (int k = 0; k < K; ++k) o.d[k] = -a.d[k];
  return o;
}
TSF_DUAL Dual<K, R> operator*(const Dual<K, R> &a, const Dual<K, R> &b) {
  Dual<K, R> o;
  o.v = a.v * b.v;
#pragma unroll
  for (int k = 0; k < K; ++k) o.d[k] = a.d[k] * b.v + a.v * b.d[k];
  return o;
}
TSF_DUAL Dual<K, R> operator*(const Dual<K, R> &a, R s) {
  Dual<K, R> o;
  o.v = a.v * s;
#pragma unroll
  for (int k = 0; k < K; ++k) o.d[k] = a.d[k] * s;
  return o;
}
TSF_DUAL Dual<K, R> operator*(R s, const Dual<K, R> &a) { return a * s; }
TSF_DUAL Dual<K, R> operator+(const Dual<K, R> &a, R s) {
  Dual<K, R> o = a;
  o.v += s;
  return o;
}
TSF_DUAL Dual<K, R> operator+(R s, const Dual<K, R> &a) { return a + s; }
TSF_DUAL Dual<K, R> operator-(const Dual<K, R> &a, R s) {
  Dual<K, R> o = a;
  o.v -= s;
  return o;
}
TSF_DUAL Dual<K, R> operator-(R s, const Dual<K, R> &a) { return (-a) + s; }
TSF_DUAL Dual<K, R> &operator+=(Dual<K, R> &a, const Dual<K, R> &b) {
  a = a + b;
  return a;
}
TSF_DUAL Dual<K, R> &operator-=(Dual<K, R> &a, const Dual<K, R> &b) {
  a = a - b;
  return a;
}
TSF_DUAL bool operator>(const Dual<K, R> &a, const Dual<K, R> &b) { return a.v > b.v; }

// d(2^x) = 2^x ln2 dx;  d(log2 x) = dx / (x ln2);  d(1/x) = -dx / x^2
TSF_DUAL Dual<K, R> ex2(const Dual<K, R> &a) {
  Dual<K, R> o;
  o.v = ex2(a.v);
  const R f = o.v * R(0.6931471805599453);
#pragma unroll
  for (int k = 0; k < K; ++k) o.d[k] = f * a.d[k];
  return o;
}
TSF_DUAL Dual<K, R> lg2(const Dual<K, R> &a) {
  Dual<K, R> o;
  o.v = lg2(a.v);
  const R f = rcp(a.v) * R(1.4426950408889634);
#pragma unroll
  for (int k = 0; k < K; ++k) o.d[k] = f * a.d[k];
  return o;
}
TSF_DUAL Dual<K, R> rcp(const Dual<K, R> &a) {
  Dual<K, R> o;
  o.v = rcp(a.v);
  const R f = -o.v * o.v;
#pragma unroll
  for (int k = 0; k < K; ++k) o.d[k] = f * a.d[k];
  return o;
}

#undef TSF_DUAL

}  // namespace tsf

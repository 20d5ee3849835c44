// sve_dual.cuh -- forward-mode dual numbers for the discrete adjoint.
//
// A Dual<N> carries a value and N directional derivatives.  The templated
// projection, celerities, Newton and fan code of sve_device.cuh run on it
// unchanged, so the adjoint differentiates exactly the arithmetic the step
// performs (each operator applies the chain rule to the derivative parts).
// Branches (max of the celerity bounds, the sign tests of the wave speeds,
// |.|) follow the value, i.e. the derivative of the active branch.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace sve {

template <int N>
struct Dual {
  double v;
  double d[N];
  __device__ __forceinline__ Dual() {}
  __device__ __forceinline__ Dual(double x) : v(x) {
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = 0.0;
  }
};

template <int N> __device__ __forceinline__ Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <int N> __device__ __forceinline__ Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <int N> __device__ __forceinline__ Dual<N> operator-(const Dual<N>& a) {
  Dual<N> r; r.v = -a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
template <int N> __device__ __forceinline__ Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <int N> __device__ __forceinline__ Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v / b.v;
  const double ib = 1.0 / b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
  return r;
}
template <int N> __device__ __forceinline__ Dual<N> tdiv(const Dual<N>& a, const Dual<N>& b) { return a / b; }
template <int N> __device__ __forceinline__ bool operator<(const Dual<N>& a, const Dual<N>& b) { return a.v < b.v; }
template <int N> __device__ __forceinline__ bool operator>(const Dual<N>& a, const Dual<N>& b) { return a.v > b.v; }
template <int N> __device__ __forceinline__ bool operator<=(const Dual<N>& a, const Dual<N>& b) { return a.v <= b.v; }
template <int N> __device__ __forceinline__ bool operator>=(const Dual<N>& a, const Dual<N>& b) { return a.v >= b.v; }
template <int N> __device__ __forceinline__ bool operator==(const Dual<N>& a, const Dual<N>& b) { return a.v == b.v; }

template <int N> __device__ __forceinline__ Dual<N> tsqrt(const Dual<N>& a) {
  Dual<N> r; r.v = sqrt(a.v);
  const double k = r.v > 0.0 ? 0.5 / r.v : 0.0;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = k * a.d[i];
  return r;
}
// a^b with both parts dual (a > 0)
template <int N> __device__ __forceinline__ Dual<N> tpow(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = pow(a.v, b.v);
  const double la = log(a.v);
  const double kb = r.v * b.v / a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = r.v * la * b.d[i] + kb * a.d[i];
  return r;
}
// a^(-1/3)
template <int N> __device__ __forceinline__ Dual<N> rcbrt64(const Dual<N>& a) {
  Dual<N> r; r.v = 1.0 / cbrt(a.v);
  const double k = -r.v / (3.0 * a.v);
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = k * a.d[i];
  return r;
}
template <int N> __device__ __forceinline__ Dual<N> nnmax(const Dual<N>& a, const Dual<N>& b) { return a.v >= b.v ? a : b; }
template <int N> __device__ __forceinline__ Dual<N> tmax(const Dual<N>& a, const Dual<N>& b) { return a.v >= b.v ? a : b; }
template <int N> __device__ __forceinline__ Dual<N> absbits(const Dual<N>& a) { return a.v < 0.0 ? -a : a; }
template <int N> __device__ __forceinline__ bool positive(const Dual<N>& a) { return a.v > 0.0; }
template <int N> __device__ __forceinline__ bool negative(const Dual<N>& a) { return a.v < 0.0; }
template <int N> __device__ __forceinline__ bool tfinite(const Dual<N>& a) { return isfinite(a.v); }

}  // namespace sve

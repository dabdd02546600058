// Forward-mode dual numbers with 8 tangents (d/du of the 8 cell unknowns),
// used by the property kernel to carry exact derivatives through the
// correlations of Sec. 2.2.
#pragma once

#include <cuda_runtime.h>

namespace isc {

struct D8 {
  double v;
  double d[8];
};

__device__ __forceinline__ D8 dc(double c) {
  D8 r;
  r.v = c;
#pragma unroll
  for (int k = 0; k < 8; ++k) r.d[k] = 0.0;
  return r;
}

__device__ __forceinline__ D8 dvar(double v, int idx) {
  D8 r = dc(v);
#pragma unroll
  for (int k = 0; k < 8; ++k) r.d[k] = (k == idx) ? 1.0 : 0.0;
  return r;
}

// r = f(a) with f'(a) = g
__device__ __forceinline__ D8 dchain(const D8& a, double f, double g) {
  D8 r;
  r.v = f;
#pragma unroll
  for (int k = 0; k < 8; ++k) r.d[k] = g * a.d[k];
  return r;
}

__device__ __forceinline__ D8 operator+(const D8& a, const D8& b) {
  D8 r;
  r.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < 8; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
__device__ __forceinline__ D8 operator-(const D8& a, const D8& b) {
  D8 r;
  r.v = a.v - b.v;
#pragma unroll
  for (int k = 0; k < 8; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
__device__ __forceinline__ D8 operator-(const D8& a) {
  D8 r;
  r.v = -a.v;
#pragma unroll
  for (int k = 0; k < 8; ++k) r.d[k] = -a.d[k];
  return r;
}
__device__ __forceinline__ D8 operator+(const D8& a, double b) {
  D8 r = a;
  r.v = a.v + b;
  return r;
}
__device__ __forceinline__ D8 operator+(double b, const D8& a) { return a + b; }
__device__ __forceinline__ D8 operator-(const D8& a, double b) {
  D8 r = a;
  r.v = a.v - b;
  return r;
}
__device__ __forceinline__ D8 operator-(double b, const D8& a) {
  D8 r;
  r.v = b - a.v;
#pragma unroll
  for (int k = 0; k < 8; ++k) r.d[k] = -a.d[k];
  return r;
}
__device__ __forceinline__ D8 operator*(const D8& a, const D8& b) {
  D8 r;
  r.v = a.v * b.v;
#pragma unroll
  for (int k = 0; k < 8; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
  return r;
}
__device__ __forceinline__ D8 operator*(const D8& a, double b) {
  D8 r;
  r.v = a.v * b;
#pragma unroll
  for (int k = 0; k < 8; ++k) r.d[k] = a.d[k] * b;
  return r;
}
__device__ __forceinline__ D8 operator*(double b, const D8& a) { return a * b; }
__device__ __forceinline__ D8 operator/(const D8& a, const D8& b) {
  D8 r;
  double ib = 1.0 / b.v;
  r.v = a.v * ib;
#pragma unroll
  for (int k = 0; k < 8; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
  return r;
}
__device__ __forceinline__ D8 operator/(const D8& a, double b) {
  D8 r;
  double ib = 1.0 / b;
  r.v = a.v * ib;
#pragma unroll
  for (int k = 0; k < 8; ++k) r.d[k] = a.d[k] * ib;
  return r;
}
__device__ __forceinline__ D8 operator/(double a, const D8& b) {
  double ib = 1.0 / b.v;
  double v = a * ib;
  return dchain(b, v, -v * ib);
}
__device__ __forceinline__ D8 dexp(const D8& a) {
  double e = exp(a.v);
  return dchain(a, e, e);
}
__device__ __forceinline__ D8 dlog(const D8& a) { return dchain(a, log(a.v), 1.0 / a.v); }
__device__ __forceinline__ D8 dsqrt(const D8& a) {
  double s = sqrt(a.v);
  return dchain(a, s, 0.5 / s);
}
// a^e for a > 0, real exponent
__device__ __forceinline__ D8 dpow(const D8& a, double e) {
  double p = pow(a.v, e);
  return dchain(a, p, e * p / a.v);
}
// fused a*b + c
__device__ __forceinline__ D8 dfma(const D8& a, const D8& b, const D8& c) {
  D8 r;
  r.v = fma(a.v, b.v, c.v);
#pragma unroll
  for (int k = 0; k < 8; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k] + c.d[k];
  return r;
}

}  // namespace isc

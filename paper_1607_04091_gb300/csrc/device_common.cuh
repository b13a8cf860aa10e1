// Device helpers shared by the NFFT translation units: complex arithmetic on
// float2 / double2 and the Kaiser-Bessel window.
#pragma once

#include "gs_internal.h"

namespace gs {
namespace dev {

template <typename R> __device__ inline C<R> mk(R a, R b);
template <> __device__ inline float2 mk<float>(float a, float b) { return make_float2(a, b); }
template <> __device__ inline double2 mk<double>(double a, double b) { return make_double2(a, b); }

template <typename T> __device__ inline T cmul(T a, T b) {
  T r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename T> __device__ inline T cmulc(T a, T b) {  // a * conj(b)
  T r;
  r.x = a.x * b.x + a.y * b.y;
  r.y = a.y * b.x - a.x * b.y;
  return r;
}
template <typename T> __device__ inline T cadd(T a, T b) {
  a.x += b.x;
  a.y += b.y;
  return a;
}
template <typename T, typename R> __device__ inline T cscale(T a, R s) {
  a.x *= s;
  a.y *= s;
  return a;
}

__device__ inline float kb_window(float d, int m, float beta) {
  float s2 = (float)(m * m) - d * d;
  if (s2 <= 0.0f) return beta * 0.318309886183790672f;
  float s = sqrtf(s2);
  return sinhf(beta * s) / (3.14159265358979323846f * s);
}
__device__ inline double kb_window(double d, int m, double beta) {
  double s2 = (double)(m * m) - d * d;
  if (s2 <= 0.0) return beta / M_PI;
  double s = sqrt(s2);
  return sinh(beta * s) / (M_PI * s);
}


template <typename R> __device__ inline R shfl(R v, int src) { return __shfl_sync(0xffffffffu, v, src); }

}  // namespace dev
}  // namespace gs

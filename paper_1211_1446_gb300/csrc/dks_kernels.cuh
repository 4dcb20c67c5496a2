// Complex helpers shared by the device code of this library (double2 / float2).
#pragma once
#include <cuda_runtime.h>

namespace dks {

template <typename V> struct RealOf;
template <> struct RealOf<double2> { using T = double; };
template <> struct RealOf<float2> { using T = float; };

template <typename V>
__device__ __host__ __forceinline__ V cadd(V a, V b) { return V{a.x + b.x, a.y + b.y}; }
template <typename V>
__device__ __host__ __forceinline__ V csub(V a, V b) { return V{a.x - b.x, a.y - b.y}; }
template <typename V>
__device__ __host__ __forceinline__ V cmul(V a, V b) {
  return V{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// conj(a) * b
template <typename V>
__device__ __host__ __forceinline__ V cmulc(V a, V b) {
  return V{a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x};
}
template <typename V>
__device__ __forceinline__ V mul_i(V a) { return V{-a.y, a.x}; }
template <typename V>
__device__ __forceinline__ V mul_mi(V a) { return V{a.y, -a.x}; }
template <typename V, typename T>
__device__ __forceinline__ V cscale(V a, T s) { return V{a.x * s, a.y * s}; }

// tw[t] = exp(+2 pi i t / N); forward transforms use the conjugate
template <typename V>
__device__ __forceinline__ V twiddle(const V* __restrict__ tw, int t, bool fwd) {
  V w = __ldg(tw + t);
  if (fwd) w.y = -w.y;
  return w;
}

__device__ __forceinline__ double2 to_d2(double2 v) { return v; }
__device__ __forceinline__ double2 to_d2(float2 v) { return double2{(double)v.x, (double)v.y}; }
template <typename V> __device__ __forceinline__ V from_d2(double2 v);
template <> __device__ __forceinline__ double2 from_d2<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 from_d2<float2>(double2 v) {
  return float2{(float)v.x, (float)v.y};
}

}  // namespace dks

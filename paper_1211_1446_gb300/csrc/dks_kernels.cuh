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
// c + a b and c + conj(a) b as four fused multiply-adds
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
  return float2{fmaf(-a.y, b.y, fmaf(a.x, b.x, c.x)), fmaf(a.y, b.x, fmaf(a.x, b.y, c.y))};
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
  return double2{fma(-a.y, b.y, fma(a.x, b.x, c.x)), fma(a.y, b.x, fma(a.x, b.y, c.y))};
}
__device__ __forceinline__ float2 cfmac(float2 a, float2 b, float2 c) {
  return float2{fmaf(a.y, b.y, fmaf(a.x, b.x, c.x)), fmaf(-a.y, b.x, fmaf(a.x, b.y, c.y))};
}
__device__ __forceinline__ double2 cfmac(double2 a, double2 b, double2 c) {
  return double2{fma(a.y, b.y, fma(a.x, b.x, c.x)), fma(-a.y, b.x, fma(a.x, b.y, c.y))};
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

namespace dks {

// ---------------------------------------------------------------- double-float arithmetic
// A value is the unevaluated sum h + l of two floats (about 48 significant bits).  Sums use
// Knuth's two-sum and products Dekker's exact product via fma, each followed by a fast
// renormalisation; all of it runs on the FP32 units.
struct dfl {
  float h, l;
};
__device__ __forceinline__ dfl df_from(double x) {
  const float h = (float)x;
  return dfl{h, (float)(x - (double)h)};
}
__device__ __forceinline__ double df_val(dfl a) { return (double)a.h + (double)a.l; }
// double -> (h, l) with integer operations (no FP64 unit): h = x with the mantissa truncated to
// 24 bits, l = the remaining 29 bits converted to FP32 (rounded), h + l = x to 2^-47 relative.
// Zero and magnitudes outside [2^-74, 2^127) take the FP64 conversions.  For bulk splits
// (k_split_df, shared-memory staging).
__device__ __forceinline__ dfl df_from_bits(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned hi32 = (unsigned)(u >> 32), lo32 = (unsigned)u;
  const int e = (int)((hi32 >> 20) & 0x7ffu);
  if (e < 949 || e > 1149) return df_from(x);
  const unsigned sign = hi32 & 0x80000000u;
  const float h = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | ((hi32 & 0xfffffu) << 3) | (lo32 >> 29));
  const float lv = __uint2float_rn(lo32 & 0x1fffffffu) * __uint_as_float((unsigned)(e - 948) << 23);
  return dfl{h, sign ? -lv : lv};
}
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  const float s = a.h + b.h;
  const float bb = s - a.h;
  float e = (a.h - (s - bb)) + (b.h - bb);
  e += a.l + b.l;
  const float h = s + e;
  return dfl{h, e - (h - s)};
}
__device__ __forceinline__ dfl df_neg(dfl a) { return dfl{-a.h, -a.l}; }
// a + x for a float x (two-sum of the leading parts, then a fast renormalisation)
__device__ __forceinline__ dfl df_add_f(dfl a, float x) {
  const float s = a.h + x;
  const float bb = s - a.h;
  const float e = ((a.h - (s - bb)) + (x - bb)) + a.l;
  const float h = s + e;
  return dfl{h, e - (h - s)};
}
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  const float h = p + e;
  return dfl{h, e - (h - p)};
}

// complex double-float (16 bytes, the size of a double2)
struct cdf {
  dfl re, im;
};
__device__ __forceinline__ cdf cadd(cdf a, cdf b) { return cdf{df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ cdf csub(cdf a, cdf b) {
  return cdf{df_add(a.re, df_neg(b.re)), df_add(a.im, df_neg(b.im))};
}
__device__ __forceinline__ cdf cmul(cdf a, cdf b) {
  return cdf{df_add(df_mul(a.re, b.re), df_neg(df_mul(a.im, b.im))), df_add(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}
__device__ __forceinline__ cdf mul_i(cdf a) { return cdf{df_neg(a.im), a.re}; }
__device__ __forceinline__ cdf mul_mi(cdf a) { return cdf{a.im, df_neg(a.re)}; }
__device__ __forceinline__ cdf cscale(cdf a, dfl s) { return cdf{df_mul(a.re, s), df_mul(a.im, s)}; }
__device__ __forceinline__ cdf twiddle(const cdf* __restrict__ tw, int t, bool fwd) {
  cdf w = tw[t];
  if (fwd) w.im = df_neg(w.im);
  return w;
}
__device__ __forceinline__ double2 to_d2(cdf v) { return double2{df_val(v.re), df_val(v.im)}; }
template <> __device__ __forceinline__ cdf from_d2<cdf>(double2 v) { return cdf{df_from(v.x), df_from(v.y)}; }
template <> struct RealOf<cdf> { using T = dfl; };

// conversions between the storage type in global memory and the compute type in shared memory
template <typename Vs> __device__ __forceinline__ Vs to_s(double2 v) { return from_d2<Vs>(v); }
template <typename Vs> __device__ __forceinline__ Vs to_s(float2 v) { return v; }
__device__ __forceinline__ double2 to_g(double2 v) { return v; }
__device__ __forceinline__ float2 to_g(float2 v) { return v; }
__device__ __forceinline__ double2 to_g(cdf v) { return to_d2(v); }

// Index checks of the debug build (-DDKS_DEBUG, libdks_debug.so): a failed check records its code
// in its translation unit's status word (the first failure is kept) and the caller skips the
// access.  In the product build the check is `true` and the comparisons compile away.
#ifdef DKS_DEBUG
static __device__ unsigned int g_dks_check = 0u;
__device__ __forceinline__ bool dks_ok(bool ok, unsigned code) {
  if (!ok) atomicCAS(&g_dks_check, 0u, code);
  return ok;
}
#else
__device__ __forceinline__ bool dks_ok(bool, unsigned) { return true; }
#endif
// check codes: kernel in the top byte, the failing item's low 24 bits below it
constexpr unsigned kChkStickInverse = 1u << 24, kChkStickForward = 2u << 24, kChkStickForwardKs = 3u << 24,
                   kChkPlane = 4u << 24, kChkPlaneDensity = 5u << 24, kChkUnpermute = 6u << 24;

}  // namespace dks

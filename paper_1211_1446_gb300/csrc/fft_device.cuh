// Mixed-radix FFT passes over lines held in shared memory (radices 2, 3, 4, 5, 6, 7, 8).
//
// A pass of radix R over a block length L (sub-length S = L / R) combines the R elements
// j, j + S, ..., j + (R-1) S of every length-L block.  The decimation-in-frequency (DIF) pass
// applies the small DFT and then multiplies output m by w^(j m N/L); the decimation-in-time
// (DIT) pass multiplies input r by w^(j r N/L) first.  Running the DIF passes with L = N, N/R0,
// ... leaves the spectrum in mixed-radix digit-reversed order, and the DIT passes in the
// opposite order take that order back to natural order, so a DIF inverse transform followed by
// a DIT forward transform needs no permutation at all.
//
// The small DFTs use fixed butterflies with the roots of unity as compile-time constants: the
// odd radices pair inputs r and R-r (R=3, 5, 7), radices 6 and 8 are a two-factor split
// (2x3, 2x4) with constant inner twiddles.  Only the inter-pass twiddles come from a table
// (tw[t] = exp(+2 pi i t / N); the forward direction uses the conjugate).
//
// Thread mapping: consecutive threads take consecutive lines (same butterfly position), so a
// warp touches addresses one line stride apart; callers give lines an odd stride (contiguous
// lines) or a unit stride (strided lines), which keeps shared-memory accesses free of bank
// conflicts for 8- and 16-byte elements.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "dks_kernels.cuh"

namespace dks {

// ------------------------------------------------------------------ constants
// cos(2 pi k / R), sin(2 pi k / R) for the k the butterflies need (first half of the circle)
__host__ __device__ constexpr double root_cos(int R, int k) {
  return R == 3 ? -0.5
       : R == 5 ? (k == 1 ? 0.3090169943749474241023 : -0.8090169943749474241023)
       : R == 7 ? (k == 1 ? 0.6234898018587335305250 : k == 2 ? -0.2225209339563144042889 : -0.9009688679024191262361)
       : R == 6 ? (k == 1 ? 0.5 : -0.5)
       : /* R == 8 */ (k == 1 ? 0.7071067811865475244008 : k == 2 ? 0.0 : -0.7071067811865475244008);
}
__host__ __device__ constexpr double root_sin(int R, int k) {
  return R == 3 ? 0.8660254037844386467637
       : R == 5 ? (k == 1 ? 0.9510565162951535721164 : 0.5877852522924731291687)
       : R == 7 ? (k == 1 ? 0.7818314824680298087084 : k == 2 ? 0.9749279121818236070181 : 0.4338837391175581204758)
       : R == 6 ? 0.8660254037844386467637
       : /* R == 8 */ (k == 2 ? 1.0 : 0.7071067811865475244008);
}

// a real constant in the three arithmetic types: double, float, and a double-float pair
struct RK {
  double d;
  float h, l;
};
__host__ __device__ constexpr RK rk(double x) { return RK{x, (float)x, (float)(x - (double)(float)x)}; }

__device__ __forceinline__ float2 rmul(float2 a, RK c) { return float2{a.x * c.h, a.y * c.h}; }
__device__ __forceinline__ double2 rmul(double2 a, RK c) { return double2{a.x * c.d, a.y * c.d}; }
__device__ __forceinline__ cdf rmul(cdf a, RK c) {
  const dfl k{c.h, c.l};
  return cdf{df_mul(a.re, k), df_mul(a.im, k)};
}
__device__ __forceinline__ float2 cneg(float2 a) { return float2{-a.x, -a.y}; }
__device__ __forceinline__ double2 cneg(double2 a) { return double2{-a.x, -a.y}; }
__device__ __forceinline__ cdf cneg(cdf a) { return cdf{df_neg(a.re), df_neg(a.im)}; }

// a * exp(i sg 2 pi k / R), sg = -1 for the forward direction
template <int R, int K, bool fwd, typename V>
__device__ __forceinline__ V mul_root(V a) {
  if constexpr (K == 0) {
    return a;
  } else if constexpr (4 * K == R) {
    return fwd ? mul_mi(a) : mul_i(a);
  } else {
    constexpr RK c = rk(root_cos(R, K)), s = rk(root_sin(R, K));
    const V ac = rmul(a, c), as = rmul(a, s);
    return cadd(ac, fwd ? mul_mi(as) : mul_i(as));
  }
}

// compile-time loop
template <int I, int N, typename F>
__device__ __forceinline__ void sfor(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    sfor<I + 1, N>(f);
  }
}

// ------------------------------------------------------------------ small DFTs, y = DFT_R(x)
template <typename V, int R, bool fwd>
__device__ __forceinline__ void dft(const V* x, V* y);

// odd R: pairs a_r = x_r + x_{R-r}, b_r = x_r - x_{R-r};
// y_m, y_{R-m} = x_0 + sum_r a_r cos(2 pi r m / R) +- i sg sum_r b_r sin(2 pi r m / R)
template <typename V, int R, bool fwd>
__device__ __forceinline__ void dft_odd(const V* x, V* y) {
  constexpr int H = (R - 1) / 2;
  V a[H], b[H];
  V y0 = x[0];
  sfor<1, H + 1>([&](auto rc) {
    constexpr int r = decltype(rc)::value;
    a[r - 1] = cadd(x[r], x[R - r]);
    b[r - 1] = csub(x[r], x[R - r]);
    y0 = cadd(y0, a[r - 1]);
  });
  sfor<1, H + 1>([&](auto mc) {
    constexpr int m = decltype(mc)::value;
    V re = x[0], im;
    sfor<1, H + 1>([&](auto rc) {
      constexpr int r = decltype(rc)::value;
      constexpr int k = (r * m) % R;
      constexpr int kk = k <= H ? k : R - k;
      constexpr RK c = rk(root_cos(R, kk)), s = rk(root_sin(R, kk));
      re = cadd(re, rmul(a[r - 1], c));
      const V t = rmul(b[r - 1], s);
      if constexpr (r == 1) {
        im = k <= H ? t : cneg(t);
      } else {
        im = k <= H ? cadd(im, t) : csub(im, t);
      }
    });
    const V ti = fwd ? mul_mi(im) : mul_i(im);
    y[m] = cadd(re, ti);
    y[R - m] = csub(re, ti);
  });
  y[0] = y0;
}

// R = P Q, n = Q n1 + n2, k = k1 + P k2:
// y[k1 + P k2] = sum_n2 w_Q^(n2 k2) [ w_R^(n2 k1) sum_n1 x[Q n1 + n2] w_P^(n1 k1) ]
template <typename V, int P, int Q, bool fwd>
__device__ __forceinline__ void dft_split(const V* x, V* y) {
  constexpr int R = P * Q;
  V a[Q][P];
  sfor<0, Q>([&](auto n2c) {
    constexpr int n2 = decltype(n2c)::value;
    V in[P];
    sfor<0, P>([&](auto n1c) { in[decltype(n1c)::value] = x[Q * decltype(n1c)::value + n2]; });
    dft<V, P, fwd>(in, a[n2]);
    sfor<1, P>([&](auto k1c) {
      constexpr int k1 = decltype(k1c)::value;
      a[n2][k1] = mul_root<R, n2 * k1, fwd>(a[n2][k1]);
    });
  });
  sfor<0, P>([&](auto k1c) {
    constexpr int k1 = decltype(k1c)::value;
    V in[Q], out[Q];
    sfor<0, Q>([&](auto n2c) { in[decltype(n2c)::value] = a[decltype(n2c)::value][k1]; });
    dft<V, Q, fwd>(in, out);
    sfor<0, Q>([&](auto k2c) { y[k1 + P * decltype(k2c)::value] = out[decltype(k2c)::value]; });
  });
}

template <typename V, int R, bool fwd>
__device__ __forceinline__ void dft(const V* x, V* y) {
  if constexpr (R == 1) {
    y[0] = x[0];
  } else if constexpr (R == 2) {
    y[0] = cadd(x[0], x[1]);
    y[1] = csub(x[0], x[1]);
  } else if constexpr (R == 4) {
    const V a = cadd(x[0], x[2]), b = csub(x[0], x[2]);
    const V c = cadd(x[1], x[3]), d = csub(x[1], x[3]);
    const V di = fwd ? mul_mi(d) : mul_i(d);
    y[0] = cadd(a, c);
    y[2] = csub(a, c);
    y[1] = cadd(b, di);
    y[3] = csub(b, di);
  } else if constexpr (R == 6) {
    dft_split<V, 2, 3, fwd>(x, y);
  } else if constexpr (R == 8) {
    dft_split<V, 2, 4, fwd>(x, y);
  } else {
    static_assert(R == 3 || R == 5 || R == 7, "unsupported radix");
    dft_odd<V, R, fwd>(x, y);
  }
}

// ------------------------------------------------------------------ passes
// a / b for 0 <= a < 2^24 and 1 <= b, with rb ~ 1/b: the float quotient is off by at most one
__device__ __forceinline__ int qdiv(int a, int b, float rb) {
  int q = __float2int_rz(__int2float_rn(a) * rb);
  const int r = a - q * b;
  q += (r >= b) - (r < 0);
  return q;
}

template <typename V, int R, bool DIT, bool fwd>
__device__ __forceinline__ void fft_pass(V* buf, int nlines, int lstride, int estride, int n, int L,
                                         const V* __restrict__ tw) {
  const int S = L / R;
  const int per_line = n / R;
  const int total = nlines * per_line;
  const int tstep = n / L;
  const int es = S * estride;
  const float rl = __fdividef(1.0f, (float)nlines), rs = __fdividef(1.0f, (float)S);
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int u = qdiv(t, nlines, rl);
    const int line = t - u * nlines;
    const int blk = qdiv(u, S, rs);
    const int j = u - blk * S;
    V* base = buf + line * lstride + (blk * L + j) * estride;
    V x[R], y[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = base[r * es];
    if (DIT && j) {
#pragma unroll
      for (int r = 1; r < R; ++r) x[r] = cmul(x[r], twiddle(tw, j * r * tstep, fwd));
    }
    dft<V, R, fwd>(x, y);
    if (!DIT && j) {
#pragma unroll
      for (int m = 1; m < R; ++m) y[m] = cmul(y[m], twiddle(tw, j * m * tstep, fwd));
    }
#pragma unroll
    for (int m = 0; m < R; ++m) base[m * es] = y[m];
  }
}

// all passes of one axis over nlines lines (element i of line l at buf[l*lstride + i*estride]);
// DIF passes in plan order, DIT passes in reverse order
template <typename V, bool DIT, bool fwd>
__device__ void fft_lines(V* buf, int nlines, int lstride, int estride, const AxisPlan& p,
                          const V* __restrict__ tw) {
  for (int i = 0; i < p.nst; ++i) {
    const int s = DIT ? (p.nst - 1 - i) : i;
    const int L = p.blk[s];
    switch (p.radix[s]) {
      case 2: fft_pass<V, 2, DIT, fwd>(buf, nlines, lstride, estride, p.n, L, tw); break;
      case 3: fft_pass<V, 3, DIT, fwd>(buf, nlines, lstride, estride, p.n, L, tw); break;
      case 4: fft_pass<V, 4, DIT, fwd>(buf, nlines, lstride, estride, p.n, L, tw); break;
      case 5: fft_pass<V, 5, DIT, fwd>(buf, nlines, lstride, estride, p.n, L, tw); break;
      case 6: fft_pass<V, 6, DIT, fwd>(buf, nlines, lstride, estride, p.n, L, tw); break;
      case 7: fft_pass<V, 7, DIT, fwd>(buf, nlines, lstride, estride, p.n, L, tw); break;
      default: fft_pass<V, 8, DIT, fwd>(buf, nlines, lstride, estride, p.n, L, tw); break;
    }
    __syncthreads();
  }
}

}  // namespace dks

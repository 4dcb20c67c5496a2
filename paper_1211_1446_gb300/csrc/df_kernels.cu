// Double-float ("float-float") versions of the two tall-skinny complex contractions, for the
// FP64 refinement phase of the mixed mode.
//
// GB300 issues FP64 at about 1/60 of its FP32 rate, and the FP64 Gram and rotation kernels run
// with the FP64 pipe ~88% busy while the FP32 FMA pipe is idle.  Here every FP64 operand is
// split on load into hi = fl32(x) and lo = fl32(x - hi) (48 significant bits), products use the
// error-free transformation p = hi_a*hi_b, e = fma(hi_a, hi_b, -p) plus the two cross terms, and
// sums are kept as unevaluated pairs with Knuth's two-sum followed by a fast renormalisation
// (Dekker / Knuth error-free transformations).  The fast renormalisation of an accumulator runs
// after every 8 of its updates instead of after each: a real multiply-add costs 12 FP32
// instructions plus 3/8, about 5x the FP64 rate on this part, with rounding at the 2^-46..2^-48
// level relative to the accumulated sums (FP64: 2^-53).  Inputs and outputs stay complex128.
#include <cuda_runtime.h>

#include <algorithm>

#include "dks_internal.h"
#include "dks_kernels.cuh"

namespace dks {

struct gdf {   // unevaluated sum hi + lo
  float hi, lo;
};

__device__ __forceinline__ gdf df_split(double x) {
  const float h = (float)x;
  return gdf{h, (float)(x - (double)h)};
}

// s += a * b without the final renormalisation: the leading part takes the exact two-sum, the
// error terms collect in s.lo; callers renormalise every few updates (df_renorm), which keeps
// |s.lo| within a few ulps of s.hi
__device__ __forceinline__ void df_mac_nr(gdf& s, const gdf a, const gdf b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const float t = s.hi + p;
  const float bb = t - s.hi;
  s.lo += ((s.hi - (t - bb)) + (p - bb)) + e;
  s.hi = t;
}
__device__ __forceinline__ void df_renorm(gdf& s) {
  const float h = s.hi + s.lo;
  s.lo = s.lo - (h - s.hi);
  s.hi = h;
}

__device__ __forceinline__ gdf df_neg(gdf a) { return gdf{-a.hi, -a.lo}; }
__device__ __forceinline__ double df_to_d(gdf a) { return (double)a.hi + (double)a.lo; }

struct gcdf {   // complex double-float
  gdf re, im;
};

__device__ __forceinline__ gcdf gcdf_split(double2 v) { return gcdf{df_split(v.x), df_split(v.y)}; }
// operand element as double-float: split a complex128 value, or take a pre-split (re hi, re lo,
// im hi, im lo) quadruple as it is
__device__ __forceinline__ gcdf ld_df(const double2* p, size_t i) {
  const double2 v = p[i];
  const dfl re = df_from_bits(v.x), im = df_from_bits(v.y);
  return gcdf{{re.h, re.l}, {im.h, im.l}};
}
__device__ __forceinline__ gcdf ld_df(const float4* p, size_t i) {
  const float4 v = p[i];
  return gcdf{{v.x, v.y}, {v.z, v.w}};
}
template <typename T> __device__ __forceinline__ gcdf zero_df() { return gcdf{{0.f, 0.f}, {0.f, 0.f}}; }

// acc += conj(a) * b  (unnormalised, see df_mac_nr)
__device__ __forceinline__ void cdf_macc(gcdf& acc, const gcdf& a, const gcdf& b) {
  df_mac_nr(acc.re, a.re, b.re);
  df_mac_nr(acc.re, a.im, b.im);
  df_mac_nr(acc.im, a.re, b.im);
  df_mac_nr(acc.im, df_neg(a.im), b.re);
}
// acc += a * b  (unnormalised)
__device__ __forceinline__ void cdf_mac(gcdf& acc, const gcdf& a, const gcdf& b) {
  df_mac_nr(acc.re, a.re, b.re);
  df_mac_nr(acc.re, df_neg(a.im), b.im);
  df_mac_nr(acc.im, a.re, b.im);
  df_mac_nr(acc.im, a.im, b.re);
}
__device__ __forceinline__ void cdf_renorm(gcdf& acc) {
  df_renorm(acc.re);
  df_renorm(acc.im);
}

// ---------------------------------------------------------------- C += A^H B
constexpr int DHN_T = 32;

// RM = 2: 32 x 32 tiles of C; RM = 3: 48 x 32 tiles (less padding when m is just above 32)
template <typename TA, typename TB, int RM>
__global__ void __launch_bounds__(256) k_gemm_hn_df(const TA* __restrict__ a, int lda,
                                                    const TB* __restrict__ b, int ldb, int k, int m, int n,
                                                    int mt, int kchunk, double2* __restrict__ c, int ldc,
                                                    int lower) {
  constexpr int TM = 16 * RM;
  __shared__ gcdf as[DHN_T][TM + 1];
  __shared__ gcdf bs[DHN_T][DHN_T + 1];
  int tm, tn;
  if (lower) {
    const int t = blockIdx.x;
    tm = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
    while ((tm + 1) * (tm + 2) / 2 <= t) ++tm;
    while (tm * (tm + 1) / 2 > t) --tm;
    tn = t - tm * (tm + 1) / 2;
  } else {
    tm = blockIdx.x % mt;
    tn = blockIdx.x / mt;
  }
  const int m0 = tm * TM, n0 = tn * DHN_T;
  const int kb = blockIdx.y * kchunk;
  const int ke = min(k, kb + kchunk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  gcdf acc[RM][2];
#pragma unroll
  for (int i = 0; i < RM; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j] = gcdf{{0.f, 0.f}, {0.f, 0.f}};
  for (int k0 = kb; k0 < ke; k0 += DHN_T) {
    for (int e = threadIdx.x; e < DHN_T * TM; e += 256) {
      const int kq = e & (DHN_T - 1), q = e >> 5;
      const int gk = k0 + kq;
      gcdf va = zero_df<TA>();
      if (gk < ke && m0 + q < m) va = ld_df(a, (size_t)(m0 + q) * lda + gk);
      as[kq][q] = va;
    }
    for (int e = threadIdx.x; e < DHN_T * DHN_T; e += 256) {
      const int kq = e & (DHN_T - 1), q = e >> 5;
      const int gk = k0 + kq;
      gcdf vb = zero_df<TB>();
      if (gk < ke && n0 + q < n) vb = ld_df(b, (size_t)(n0 + q) * ldb + gk);
      bs[kq][q] = vb;
    }
    __syncthreads();
    for (int kq0 = 0; kq0 < DHN_T; kq0 += 4) {
#pragma unroll
      for (int kq = kq0; kq < kq0 + 4; ++kq) {
        const gcdf b0 = bs[kq][tx], b1 = bs[kq][tx + 16];
#pragma unroll
        for (int i = 0; i < RM; ++i) {
          const gcdf ai = as[kq][ty + 16 * i];
          cdf_macc(acc[i][0], ai, b0);
          cdf_macc(acc[i][1], ai, b1);
        }
      }
#pragma unroll
      for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) cdf_renorm(acc[i][j]);   // every 8 updates of each part
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < RM; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int mm = m0 + ty + 16 * i, nn = n0 + tx + 16 * j;
      if (mm < m && nn < n) {
        atomicAdd(&c[(size_t)nn * ldc + mm].x, df_to_d(acc[i][j].re));
        atomicAdd(&c[(size_t)nn * ldc + mm].y, df_to_d(acc[i][j].im));
      }
    }
}

// Both Gram matrices from double-float copies in one pass: S = Z^H Z and A = Z^H HZ, block lower
// triangles of 32 x 32 tiles; the Z tile of the row block serves both products.
constexpr int DG_K = 16;

__global__ void __launch_bounds__(256) k_gram_df(const float4* __restrict__ z, const float4* __restrict__ hz,
                                                 int ld, int k, int m, int kchunk, double2* __restrict__ a,
                                                 double2* __restrict__ s) {
  __shared__ gcdf zs[DG_K][DHN_T + 1];
  __shared__ gcdf zb[DG_K][DHN_T + 1];
  __shared__ gcdf hb[DG_K][DHN_T + 1];
  const int t = blockIdx.x;
  int tm = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
  while ((tm + 1) * (tm + 2) / 2 <= t) ++tm;
  while (tm * (tm + 1) / 2 > t) --tm;
  const int tn = t - tm * (tm + 1) / 2;
  const int m0 = tm * DHN_T, n0 = tn * DHN_T;
  const int kb = blockIdx.y * kchunk;
  const int ke = min(k, kb + kchunk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  gcdf as_[2][2], aa[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) as_[i][j] = aa[i][j] = gcdf{{0.f, 0.f}, {0.f, 0.f}};
  for (int k0 = kb; k0 < ke; k0 += DG_K) {
    for (int e = threadIdx.x; e < DG_K * DHN_T; e += 256) {
      const int kq = e & (DG_K - 1), q = e >> 4;
      const int gk = k0 + kq;
      gcdf vz = zero_df<float4>(), vb = zero_df<float4>(), vh = zero_df<float4>();
      if (gk < ke) {
        if (m0 + q < m) vz = ld_df(z, (size_t)(m0 + q) * ld + gk);
        if (n0 + q < m) {
          vb = ld_df(z, (size_t)(n0 + q) * ld + gk);
          vh = ld_df(hz, (size_t)(n0 + q) * ld + gk);
        }
      }
      zs[kq][q] = vz;
      zb[kq][q] = vb;
      hb[kq][q] = vh;
    }
    __syncthreads();
    for (int kq0 = 0; kq0 < DG_K; kq0 += 4) {
#pragma unroll
      for (int kq = kq0; kq < kq0 + 4; ++kq) {
        const gcdf a0 = zs[kq][ty], a1 = zs[kq][ty + 16];
        const gcdf b0 = zb[kq][tx], b1 = zb[kq][tx + 16];
        const gcdf h0 = hb[kq][tx], h1 = hb[kq][tx + 16];
        cdf_macc(as_[0][0], a0, b0);
        cdf_macc(as_[0][1], a0, b1);
        cdf_macc(as_[1][0], a1, b0);
        cdf_macc(as_[1][1], a1, b1);
        cdf_macc(aa[0][0], a0, h0);
        cdf_macc(aa[0][1], a0, h1);
        cdf_macc(aa[1][0], a1, h0);
        cdf_macc(aa[1][1], a1, h1);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          cdf_renorm(as_[i][j]);   // every 8 updates of each part
          cdf_renorm(aa[i][j]);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int mm = m0 + ty + 16 * i, nn = n0 + tx + 16 * j;
      if (mm < m && nn < m) {
        atomicAdd(&s[(size_t)nn * m + mm].x, df_to_d(as_[i][j].re));
        atomicAdd(&s[(size_t)nn * m + mm].y, df_to_d(as_[i][j].im));
        atomicAdd(&a[(size_t)nn * m + mm].x, df_to_d(aa[i][j].re));
        atomicAdd(&a[(size_t)nn * m + mm].y, df_to_d(aa[i][j].im));
      }
    }
}

static int df_num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

template <typename TA, typename TB>
static int gemm_hn_df_t(const TA* a, int lda, const TB* b, int ldb, int k, int m, int n, double2* c,
                        cudaStream_t st, int cat, int ldc, bool lower) {
  if (m <= 0 || n <= 0 || k <= 0) return DKS_OK;
  if (ldc <= 0) ldc = m;
  if (lower && m != n) return fail(DKS_ERR_INVALID_ARG, "gemm_hn_df: lower-triangle mode needs a square result");
  const bool rm3 = !lower && (m + 47) / 48 * 48 < (m + 31) / 32 * 32;
  const int tmr = rm3 ? 48 : DHN_T;
  const int mt = (m + tmr - 1) / tmr, nt = (n + DHN_T - 1) / DHN_T;
  const int tiles = lower ? mt * (mt + 1) / 2 : mt * nt;
  const int ktiles = (k + DHN_T - 1) / DHN_T;
  int splits = std::max(1, (4 * df_num_sms()) / tiles);
  splits = std::min(splits, ktiles);
  const int kchunk = ((ktiles + splits - 1) / splits) * DHN_T;
  splits = (k + kchunk - 1) / kchunk;
  dim3 grid(tiles, splits);
  const bool same = (const void*)a == (const void*)b;
  Prof pr(cat, st, (same ? (double)m : (double)(m + n)) * k * 16.0 + 16.0 * m * n,
          (lower ? 4.0 * m * (m + 1.0) : 8.0 * m * n) * (double)k);
  if (rm3)
    k_gemm_hn_df<TA, TB, 3><<<grid, 256, 0, st>>>(a, lda, b, ldb, k, m, n, mt, kchunk, c, ldc, lower ? 1 : 0);
  else
    k_gemm_hn_df<TA, TB, 2><<<grid, 256, 0, st>>>(a, lda, b, ldb, k, m, n, mt, kchunk, c, ldc, lower ? 1 : 0);
  DKS_CUDA_TRY(cudaGetLastError());
  return DKS_OK;
}

int gemm_hn_df(const double2* a, int lda, const double2* b, int ldb, int k, int m, int n, double2* c,
               cudaStream_t st, int cat, int ldc, bool lower) {
  return gemm_hn_df_t(a, lda, b, ldb, k, m, n, c, st, cat, ldc, lower);
}
int gemm_hn_df(const float4* a, int lda, const float4* b, int ldb, int k, int m, int n, double2* c,
               cudaStream_t st, int cat, int ldc, bool lower) {
  return gemm_hn_df_t(a, lda, b, ldb, k, m, n, c, st, cat, ldc, lower);
}
int gemm_hn_df(const float4* a, int lda, const double2* b, int ldb, int k, int m, int n, double2* c,
               cudaStream_t st, int cat, int ldc, bool lower) {
  return gemm_hn_df_t(a, lda, b, ldb, k, m, n, c, st, cat, ldc, lower);
}

// ---------------------------------------------------------------- OUT = alpha A diag(ws) W + beta OUT
// 64 rows x (8 * ncg) columns per CTA (ncg <= 5 column groups, sized to the number of output
// columns), one row x 8 columns per thread, two CTAs per SM.
constexpr int DNN_RPT = 1, DNN_R = 64 * DNN_RPT, DNN_GMAX = 5, DNN_CMAX = 8 * DNN_GMAX, DNN_M = 16;

template <typename TA>
__global__ void __launch_bounds__(64 * DNN_GMAX, 2) k_gemm_nn_df(const TA* __restrict__ a, int lda, int k, int m,
                                                       const double2* __restrict__ w, int ldw,
                                                       const double* __restrict__ ws, int n,
                                                       double2* __restrict__ out, int ldo, double alpha, double beta) {
  __shared__ gcdf as[DNN_M][DNN_R];
  __shared__ gcdf wsm[DNN_M][DNN_CMAX];
  const int ncols = (blockDim.x >> 6) * 8;
  const int r0 = blockIdx.x * DNN_R, c0 = blockIdx.y * ncols;
  const int rg = threadIdx.x & 63, cg = threadIdx.x >> 6;
  gcdf acc[DNN_RPT][8];
#pragma unroll
  for (int i = 0; i < DNN_RPT; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = gcdf{{0.f, 0.f}, {0.f, 0.f}};
  for (int m0 = 0; m0 < m; m0 += DNN_M) {
    for (int e = threadIdx.x; e < DNN_M * DNN_R; e += blockDim.x) {
      const int mm = e / DNN_R, rr = e - mm * DNN_R;
      gcdf v = zero_df<TA>();
      if (m0 + mm < m && r0 + rr < k) v = ld_df(a, (size_t)(m0 + mm) * lda + r0 + rr);
      as[mm][rr] = v;
    }
    for (int e = threadIdx.x; e < DNN_M * ncols; e += blockDim.x) {
      const int mm = e / ncols, cc = e - mm * ncols;
      double2 v{0, 0};
      if (m0 + mm < m && c0 + cc < n) {
        v = w[(size_t)(c0 + cc) * ldw + m0 + mm];
        const double s = (ws ? ws[m0 + mm] : 1.0) * alpha;
        v.x *= s;
        v.y *= s;
      }
      wsm[mm][cc] = gcdf_split(v);
    }
    __syncthreads();
    for (int mm0 = 0; mm0 < DNN_M; mm0 += 4) {
#pragma unroll 2
      for (int mm = mm0; mm < mm0 + 4; ++mm) {
        gcdf av[DNN_RPT];
#pragma unroll
        for (int i = 0; i < DNN_RPT; ++i) av[i] = as[mm][rg + 64 * i];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const gcdf wv = wsm[mm][cg * 8 + j];
#pragma unroll
          for (int i = 0; i < DNN_RPT; ++i) cdf_mac(acc[i][j], av[i], wv);
        }
      }
#pragma unroll
      for (int i = 0; i < DNN_RPT; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) cdf_renorm(acc[i][j]);   // every 8 updates of each part
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < DNN_RPT; ++i) {
    const int row = r0 + rg + 64 * i;
    if (row >= k) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int cc = c0 + cg * 8 + j;
      if (cc < n) {
        double2* o = out + (size_t)cc * ldo + row;
        double2 r{df_to_d(acc[i][j].re), df_to_d(acc[i][j].im)};
        if (beta != 0.0) {
          const double2 old = *o;
          r.x += beta * old.x;
          r.y += beta * old.y;
        }
        *o = r;
      }
    }
  }
}

// The same product for pre-split (float4) A in two shared-memory stages: the A chunk of the
// next 16 inner indices is copied with cp.async (16 bytes per element) while the current one is
// multiplied; W is split into double-float pairs after the multiply.
constexpr size_t DNN_SMEM = 2 * (size_t)DNN_M * DNN_R * sizeof(gcdf) + 2 * (size_t)DNN_M * DNN_CMAX * sizeof(gcdf);

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src));
}

__global__ void __launch_bounds__(64 * DNN_GMAX, 2) k_gemm_nn_df4(const float4* __restrict__ a, int lda, int k, int m,
                                                        const double2* __restrict__ w, int ldw,
                                                        const double* __restrict__ ws, int n,
                                                        double2* __restrict__ out, int ldo, double alpha, double beta) {
  extern __shared__ __align__(16) unsigned char dn_smem[];
  gcdf* as_base = reinterpret_cast<gcdf*>(dn_smem);          // [2][DNN_M][DNN_R]
  gcdf* ws_base = as_base + 2 * DNN_M * DNN_R;                // [2][DNN_M][DNN_CMAX]
  const int ncols = (blockDim.x >> 6) * 8;
  const int r0 = blockIdx.x * DNN_R, c0 = blockIdx.y * ncols;
  const int rg = threadIdx.x & 63, cg = threadIdx.x >> 6;
  gcdf acc[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) acc[j] = gcdf{{0.f, 0.f}, {0.f, 0.f}};
  auto load_a = [&](int buf, int m0) {
    gcdf* dst = as_base + (size_t)buf * DNN_M * DNN_R;
    for (int e = threadIdx.x; e < DNN_M * DNN_R; e += blockDim.x) {
      const int mm = e / DNN_R, rr = e - mm * DNN_R;
      if (m0 + mm < m && r0 + rr < k) cp_async16(dst + e, a + (size_t)(m0 + mm) * lda + r0 + rr);
      else dst[e] = gcdf{{0.f, 0.f}, {0.f, 0.f}};
    }
    asm volatile("cp.async.commit_group;\n" ::);
  };
  auto load_w = [&](int buf, int m0) {
    gcdf* dst = ws_base + (size_t)buf * DNN_M * DNN_CMAX;
    for (int e = threadIdx.x; e < DNN_M * ncols; e += blockDim.x) {
      const int mm = e / ncols, cc = e - mm * ncols;
      double2 v{0, 0};
      if (m0 + mm < m && c0 + cc < n) {
        v = w[(size_t)(c0 + cc) * ldw + m0 + mm];
        const double sc = (ws ? ws[m0 + mm] : 1.0) * alpha;
        v.x *= sc;
        v.y *= sc;
      }
      dst[mm * DNN_CMAX + cc] = gcdf_split(v);
    }
  };
  const int nch = (m + DNN_M - 1) / DNN_M;
  load_a(0, 0);
  load_w(0, 0);
  for (int ch = 0; ch < nch; ++ch) {
    const int cur = ch & 1;
    const bool more = ch + 1 < nch;
    if (more) {
      load_a(cur ^ 1, (ch + 1) * DNN_M);
      asm volatile("cp.async.wait_group 1;\n" ::);
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::);
    }
    __syncthreads();
    const gcdf* as = as_base + (size_t)cur * DNN_M * DNN_R;
    const gcdf* wsm = ws_base + (size_t)cur * DNN_M * DNN_CMAX;
    for (int mm0 = 0; mm0 < DNN_M; mm0 += 4) {
#pragma unroll 2
      for (int mm = mm0; mm < mm0 + 4; ++mm) {
        const gcdf av = as[mm * DNN_R + rg];
#pragma unroll
        for (int j = 0; j < 8; ++j) cdf_mac(acc[j], av, wsm[mm * DNN_CMAX + cg * 8 + j]);
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) cdf_renorm(acc[j]);   // every 8 updates of each part
    }
    if (more) load_w(cur ^ 1, (ch + 1) * DNN_M);
    __syncthreads();
  }
  const int row = r0 + rg;
  if (row >= k) return;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int cc = c0 + cg * 8 + j;
    if (cc < n) {
      double2* o = out + (size_t)cc * ldo + row;
      double2 r{df_to_d(acc[j].re), df_to_d(acc[j].im)};
      if (beta != 0.0) {
        const double2 old = *o;
        r.x += beta * old.x;
        r.y += beta * old.y;
      }
      *o = r;
    }
  }
}

template <typename TA>
static int gemm_nn_df_t(const TA* a, int lda, int k, int m, const double2* w, int ldw, const double* wscale,
                        int n, double2* out, int ldo, double beta, cudaStream_t st, double alpha, int cat) {
  if (k <= 0 || n <= 0) return DKS_OK;
  // column groups of 8 per CTA: the fewest CTAs along n, then the smallest tile covering them
  const int tiles = (n + 8 * DNN_GMAX - 1) / (8 * DNN_GMAX);
  const int g = std::max(1, ((n + tiles - 1) / tiles + 7) / 8);
  dim3 grid((k + DNN_R - 1) / DNN_R, tiles);
  Prof pr(cat, st, (double)m * k * 16.0 + (beta != 0.0 ? 2.0 : 1.0) * n * k * 16.0 + 16.0 * m * n,
          8.0 * (double)k * m * n);
  if constexpr (std::is_same<TA, float4>::value) {
    static bool attr = false;
    if (!attr) {
      DKS_CUDA_TRY(cudaFuncSetAttribute((const void*)k_gemm_nn_df4, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)DNN_SMEM));
      attr = true;
    }
    k_gemm_nn_df4<<<grid, 64 * g, DNN_SMEM, st>>>(a, lda, k, m, w, ldw, wscale, n, out, ldo, alpha, beta);
  } else {
    k_gemm_nn_df<TA><<<grid, 64 * g, 0, st>>>(a, lda, k, m, w, ldw, wscale, n, out, ldo, alpha, beta);
  }
  DKS_CUDA_TRY(cudaGetLastError());
  return DKS_OK;
}

int gemm_nn_df(const double2* a, int lda, int k, int m, const double2* w, int ldw, const double* wscale, int n,
               double2* out, int ldo, double beta, cudaStream_t st, double alpha, int cat) {
  return gemm_nn_df_t(a, lda, k, m, w, ldw, wscale, n, out, ldo, beta, st, alpha, cat);
}

int gram_df(const float4* z, const float4* hz, int ld, int k, int m, double2* a, double2* s, cudaStream_t st) {
  if (m <= 0 || k <= 0) return DKS_OK;
  const int mt = (m + DHN_T - 1) / DHN_T;
  const int tiles = mt * (mt + 1) / 2;
  const int ktiles = (k + DG_K - 1) / DG_K;
  int splits = std::min(std::max(1, (4 * df_num_sms()) / tiles), ktiles);
  const int kchunk = ((ktiles + splits - 1) / splits) * DG_K;
  splits = (k + kchunk - 1) / kchunk;
  Prof pr(P_GRAM, st, 2.0 * m * 16.0 * k + 32.0 * m * m, 8.0 * m * (m + 1.0) * (double)k);
  k_gram_df<<<dim3(tiles, splits), 256, 0, st>>>(z, hz, ld, k, m, kchunk, a, s);
  DKS_CUDA_TRY(cudaGetLastError());
  return DKS_OK;
}
int gemm_nn_df(const float4* a, int lda, int k, int m, const double2* w, int ldw, const double* wscale, int n,
               double2* out, int ldo, double beta, cudaStream_t st, double alpha, int cat) {
  return gemm_nn_df_t(a, lda, k, m, w, ldw, wscale, n, out, ldo, beta, st, alpha, cat);
}

// ---------------------------------------------------------------- split complex128 -> double-float
// df_from_bits (integer operations); a block is split once and then read by every contraction
// of the iteration.
__global__ void k_split_df(const double2* __restrict__ in, float4* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double2 v = in[i];
    const dfl re = df_from_bits(v.x), im = df_from_bits(v.y);
    out[i] = float4{re.h, re.l, im.h, im.l};
  }
}

int split_df(const double2* in, float4* out, size_t n, cudaStream_t st) {
  if (!n) return DKS_OK;
  Prof pr(P_MISC, st, 32.0 * n, 0.0);
  const int blocks = (int)std::min<size_t>((n + 255) / 256, (size_t)df_num_sms() * 16);
  k_split_df<<<blocks, 256, 0, st>>>(in, out, n);
  DKS_CUDA_TRY(cudaGetLastError());
  return DKS_OK;
}

}  // namespace dks

// Block linear algebra of Algorithm 1 on tall-skinny complex blocks.
//
//  gemm_hn   C (m x n) += A^H B   A: k x m, B: k x n (k = 4 npw or 2 npw, huge; m, n small)
//            Gram matrices of the projected pencil and the projector coefficients B^H x~.
//            Split over k across the grid; each CTA reduces a 32x32 tile of C over its
//            k-range in registers and adds it to C with FP64 atomics.  With FP32 operands
//            each 32-deep k-tile is summed in FP32 and folded into a double-float total.
//  gemm_nn   OUT (k x n) = alpha A (k x m) diag(ws) W (m x n) + beta OUT
//            Rotations X <- Z V, P <- [0,Y,P] V and the projector
//            update x~ += B (D Z).  W (FP64, from the small solve) is staged in shared
//            memory in the working precision.
//  col_stats per column: ||hx - lam x||^2, ||x||^2 and sum_G |k+G|^2/2 |x|^2 (FP64 column sums)
//  precond   Y = K(x_G) (HX - lam X) on the active columns (residual and Teter factor fused)
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "dks_internal.h"
#include "dks_kernels.cuh"

namespace dks {

namespace cg = cooperative_groups;

// accumulation type: FP64 as soon as one operand is FP64
template <typename A, typename B> struct AccOf { using T = double2; };
template <> struct AccOf<float2, float2> { using T = float2; };
template <typename T> __device__ __forceinline__ T cvt(double2 v);
template <> __device__ __forceinline__ double2 cvt<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 cvt<float2>(double2 v) { return float2{(float)v.x, (float)v.y}; }
template <typename T> __device__ __forceinline__ T cvt(float2 v);
template <> __device__ __forceinline__ double2 cvt<double2>(float2 v) { return double2{v.x, v.y}; }
template <> __device__ __forceinline__ float2 cvt<float2>(float2 v) { return v; }

// ---------------------------------------------------------------- gemm_hn
constexpr int HN_T = 32;

// asynchronous global -> shared copies (cp.async, 8 bytes) for the multi-stage tile loops
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// RM = 2: 32 x 32 tiles of C; RM = 3: 48 x 32 tiles (less padding when m is just above 32)
template <typename Va, typename Vb, typename A, int RM>
__global__ void __launch_bounds__(256) k_gemm_hn(const Va* __restrict__ a, int lda, const Vb* __restrict__ b,
                                                 int ldb, int k, int m, int n, int mt, int kchunk,
                                                 double2* __restrict__ c, int ldc, int lower) {
  constexpr int TM = 16 * RM;
  __shared__ A as[HN_T][TM + 1];
  __shared__ A bs[HN_T][HN_T + 1];
  int tm, tn;
  if (lower) {   // only tiles with tn <= tm (the block lower triangle of a Hermitian result)
    const int t = blockIdx.x;
    tm = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while ((tm + 1) * (tm + 2) / 2 <= t) ++tm;
    while (tm * (tm + 1) / 2 > t) --tm;
    tn = t - tm * (tm + 1) / 2;
  } else {
    tm = blockIdx.x % mt;
    tn = blockIdx.x / mt;
  }
  const int m0 = tm * TM, n0 = tn * HN_T;
  const int kb = blockIdx.y * kchunk;
  const int ke = min(k, kb + kchunk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  A acc[RM][2];
#pragma unroll
  for (int i = 0; i < RM; ++i) acc[i][0] = acc[i][1] = A{0, 0};
  // FP32 arithmetic: each k-tile is summed in FP32 and folded into a double-float total, so
  // FP32 rounding accumulates over 32 terms instead of the whole k-range of the CTA
  constexpr bool fold = std::is_same<A, float2>::value;
  dfl tot[RM][2][2] = {};
  for (int k0 = kb; k0 < ke; k0 += HN_T) {
    for (int e = threadIdx.x; e < HN_T * TM; e += 256) {
      const int kq = e & (HN_T - 1), q = e >> 5;
      const int gk = k0 + kq;
      A va{0, 0};
      if (gk < ke && m0 + q < m) va = cvt<A>(a[(size_t)(m0 + q) * lda + gk]);
      as[kq][q] = va;
    }
    for (int e = threadIdx.x; e < HN_T * HN_T; e += 256) {
      const int kq = e & (HN_T - 1), q = e >> 5;
      const int gk = k0 + kq;
      A vb{0, 0};
      if (gk < ke && n0 + q < n) vb = cvt<A>(b[(size_t)(n0 + q) * ldb + gk]);
      bs[kq][q] = vb;
    }
    __syncthreads();
#pragma unroll 8
    for (int kq = 0; kq < HN_T; ++kq) {
      const A b0 = bs[kq][tx], b1 = bs[kq][tx + 16];
#pragma unroll
      for (int i = 0; i < RM; ++i) {
        const A ai = as[kq][ty + 16 * i];
        acc[i][0] = cfmac(ai, b0, acc[i][0]);
        acc[i][1] = cfmac(ai, b1, acc[i][1]);
      }
    }
    if constexpr (fold) {
#pragma unroll
      for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          tot[i][j][0] = df_add_f(tot[i][j][0], acc[i][j].x);
          tot[i][j][1] = df_add_f(tot[i][j][1], acc[i][j].y);
          acc[i][j] = A{0, 0};
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < RM; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int mm = m0 + ty + 16 * i, nn = n0 + tx + 16 * j;
      if (mm < m && nn < n) {
        const double vx = fold ? df_val(tot[i][j][0]) : (double)acc[i][j].x;
        const double vy = fold ? df_val(tot[i][j][1]) : (double)acc[i][j].y;
        atomicAdd(&c[(size_t)nn * ldc + mm].x, vx);
        atomicAdd(&c[(size_t)nn * ldc + mm].y, vy);
      }
    }
}

// The FP32 case of k_gemm_hn (complex64 operands, FP32 k-tiles folded into double-float totals)
// with two shared-memory stages: the next 32-deep k-tile of A and B is copied with cp.async
// while the current one is multiplied.
template <int RM>
constexpr size_t hn32_smem() {
  return 2 * ((size_t)HN_T * (16 * RM + 1) + (size_t)HN_T * (HN_T + 1)) * sizeof(float2);
}

template <int RM>
__global__ void __launch_bounds__(256) k_gemm_hn_f32p(const float2* __restrict__ a, int lda,
                                                      const float2* __restrict__ b, int ldb, int k, int m, int n,
                                                      int mt, int kchunk, double2* __restrict__ c, int ldc,
                                                      int lower) {
  constexpr int TM = 16 * RM;
  constexpr int AS = HN_T * (TM + 1), BS = HN_T * (HN_T + 1);
  extern __shared__ __align__(16) unsigned char h32_smem[];
  float2* stage = reinterpret_cast<float2*>(h32_smem);   // [2][as | bs]
  int tm, tn;
  if (lower) {
    const int t = blockIdx.x;
    tm = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while ((tm + 1) * (tm + 2) / 2 <= t) ++tm;
    while (tm * (tm + 1) / 2 > t) --tm;
    tn = t - tm * (tm + 1) / 2;
  } else {
    tm = blockIdx.x % mt;
    tn = blockIdx.x / mt;
  }
  const int m0 = tm * TM, n0 = tn * HN_T;
  const int kb = blockIdx.y * kchunk;
  const int ke = min(k, kb + kchunk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float2 acc[RM][2];
#pragma unroll
  for (int i = 0; i < RM; ++i) acc[i][0] = acc[i][1] = float2{0.f, 0.f};
  dfl tot[RM][2][2] = {};
  auto load = [&](int buf, int k0) {
    float2* as = stage + (size_t)buf * (AS + BS);
    float2* bs = as + AS;
    for (int e = threadIdx.x; e < HN_T * TM; e += 256) {
      const int kq = e & (HN_T - 1), q = e >> 5;
      const int gk = k0 + kq;
      float2* d = as + kq * (TM + 1) + q;
      if (gk < ke && m0 + q < m) cp_async8(d, a + (size_t)(m0 + q) * lda + gk);
      else *d = float2{0.f, 0.f};
    }
    for (int e = threadIdx.x; e < HN_T * HN_T; e += 256) {
      const int kq = e & (HN_T - 1), q = e >> 5;
      const int gk = k0 + kq;
      float2* d = bs + kq * (HN_T + 1) + q;
      if (gk < ke && n0 + q < n) cp_async8(d, b + (size_t)(n0 + q) * ldb + gk);
      else *d = float2{0.f, 0.f};
    }
    cp_async_commit();
  };
  if (kb < ke) load(0, kb);
  for (int k0 = kb, it = 0; k0 < ke; k0 += HN_T, ++it) {
    const int cur = it & 1;
    if (k0 + HN_T < ke) {
      load(cur ^ 1, k0 + HN_T);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const float2* as = stage + (size_t)cur * (AS + BS);
    const float2* bs = as + AS;
#pragma unroll 8
    for (int kq = 0; kq < HN_T; ++kq) {
      const float2 b0 = bs[kq * (HN_T + 1) + tx], b1 = bs[kq * (HN_T + 1) + tx + 16];
#pragma unroll
      for (int i = 0; i < RM; ++i) {
        const float2 ai = as[kq * (TM + 1) + ty + 16 * i];
        acc[i][0] = cfmac(ai, b0, acc[i][0]);
        acc[i][1] = cfmac(ai, b1, acc[i][1]);
      }
    }
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        tot[i][j][0] = df_add_f(tot[i][j][0], acc[i][j].x);
        tot[i][j][1] = df_add_f(tot[i][j][1], acc[i][j].y);
        acc[i][j] = float2{0.f, 0.f};
      }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < RM; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int mm = m0 + ty + 16 * i, nn = n0 + tx + 16 * j;
      if (mm < m && nn < n) {
        atomicAdd(&c[(size_t)nn * ldc + mm].x, df_val(tot[i][j][0]));
        atomicAdd(&c[(size_t)nn * ldc + mm].y, df_val(tot[i][j][1]));
      }
    }
}

// Both Gram matrices of Algorithm 1 from FP32 blocks in one pass: S = Z^H Z and A = Z^H HZ, block
// lower triangles of 32 x 32 tiles.  The Z tile of the row block serves both products; each of
// the 128 threads holds 4 x 2 outputs of S and of A, so per k step its 8 shared-memory loads
// (four Z row values, two Z and two HZ column values) feed 16 complex multiply-adds; FP32 within
// a 32-deep k-tile, folded into double-float totals.
// two shared-memory stages of (Z rows of the tile's row block, Z and HZ rows of its column block):
// the next 32-deep k-tile is copied with cp.async while the current one is multiplied
constexpr int GF_TILE = HN_T * (HN_T + 1);   // one padded 32 x 33 tile, float2
constexpr size_t GF_SMEM = 2 * 3 * (size_t)GF_TILE * sizeof(float2);
constexpr int GF_THREADS = 128;

__global__ void __launch_bounds__(GF_THREADS, 4) k_gram_f32(const float2* __restrict__ z, const float2* __restrict__ hz,
                                                  int ld, int k, int m, int kchunk, double2* __restrict__ a,
                                                  double2* __restrict__ s) {
  extern __shared__ __align__(16) unsigned char gf_smem[];
  float2* stage = reinterpret_cast<float2*>(gf_smem);   // [2][zs | zb | hb], each [HN_T][HN_T + 1]
  const int t = blockIdx.x;
  int tm = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
  while ((tm + 1) * (tm + 2) / 2 <= t) ++tm;
  while (tm * (tm + 1) / 2 > t) --tm;
  const int tn = t - tm * (tm + 1) / 2;
  const int m0 = tm * HN_T, n0 = tn * HN_T;
  const int kb = blockIdx.y * kchunk;
  const int ke = min(k, kb + kchunk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // rows ty + 8 i, columns tx + 16 j
  float2 as_[4][2], aa[4][2];
  dfl ts[4][2][2] = {}, ta[4][2][2] = {};
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) as_[i][j] = aa[i][j] = float2{0.f, 0.f};
  auto load = [&](int buf, int k0) {
    float2* zs = stage + (size_t)buf * 3 * GF_TILE;
    float2* zb = zs + GF_TILE;
    float2* hb = zb + GF_TILE;
    for (int e = threadIdx.x; e < HN_T * HN_T; e += GF_THREADS) {
      const int kq = e & (HN_T - 1), q = e >> 5;
      const int gk = k0 + kq;
      const int o = kq * (HN_T + 1) + q;
      const bool kin = gk < ke;
      if (kin && m0 + q < m) cp_async8(zs + o, z + (size_t)(m0 + q) * ld + gk);
      else zs[o] = float2{0.f, 0.f};
      if (kin && n0 + q < m) {
        cp_async8(zb + o, z + (size_t)(n0 + q) * ld + gk);
        cp_async8(hb + o, hz + (size_t)(n0 + q) * ld + gk);
      } else {
        zb[o] = float2{0.f, 0.f};
        hb[o] = float2{0.f, 0.f};
      }
    }
    cp_async_commit();
  };
  if (kb < ke) load(0, kb);
  for (int k0 = kb, it = 0; k0 < ke; k0 += HN_T, ++it) {
    const int cur = it & 1;
    if (k0 + HN_T < ke) {
      load(cur ^ 1, k0 + HN_T);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const float2* zs = stage + (size_t)cur * 3 * GF_TILE;
    const float2* zb = zs + GF_TILE;
    const float2* hb = zb + GF_TILE;
#pragma unroll 8
    for (int kq = 0; kq < HN_T; ++kq) {
      const float2* zr = zs + kq * (HN_T + 1);
      const float2* br = zb + kq * (HN_T + 1);
      const float2* hr = hb + kq * (HN_T + 1);
      const float2 b[2] = {br[tx], br[tx + 16]};
      const float2 h[2] = {hr[tx], hr[tx + 16]};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float2 ai = zr[ty + 8 * i];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          as_[i][j] = cfmac(ai, b[j], as_[i][j]);
          aa[i][j] = cfmac(ai, h[j], aa[i][j]);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        ts[i][j][0] = df_add_f(ts[i][j][0], as_[i][j].x);
        ts[i][j][1] = df_add_f(ts[i][j][1], as_[i][j].y);
        ta[i][j][0] = df_add_f(ta[i][j][0], aa[i][j].x);
        ta[i][j][1] = df_add_f(ta[i][j][1], aa[i][j].y);
        as_[i][j] = aa[i][j] = float2{0.f, 0.f};
      }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int mm = m0 + ty + 8 * i, nn = n0 + tx + 16 * j;
      if (mm < m && nn < m) {
        atomicAdd(&s[(size_t)nn * m + mm].x, df_val(ts[i][j][0]));
        atomicAdd(&s[(size_t)nn * m + mm].y, df_val(ts[i][j][1]));
        atomicAdd(&a[(size_t)nn * m + mm].x, df_val(ta[i][j][0]));
        atomicAdd(&a[(size_t)nn * m + mm].y, df_val(ta[i][j][1]));
      }
    }
}

static int g_num_sms = 0;
static int num_sms() {
  if (!g_num_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  return g_num_sms;
}

template <typename Va, typename Vb, bool Acc64>
int gemm_hn(const Va* a, int lda, const Vb* b, int ldb, int k, int m, int n, double2* c, cudaStream_t st,
            int cat, int ldc, bool lower, int tc) {
  if (m <= 0 || n <= 0 || k <= 0) return DKS_OK;
  if (ldc <= 0) ldc = m;
  if (lower && m != n) return fail(DKS_ERR_INVALID_ARG, "gemm_hn: lower-triangle mode needs a square result");
  if constexpr (std::is_same<Va, float2>::value && std::is_same<Vb, float2>::value && !Acc64) {
    // tensor cores: the result is written, which equals the accumulation into the zeroed c the
    // callers provide.  Projector coefficients: a side of at most 64 columns goes along the MMA's
    // 128 rows in the packed form (A and i A together); otherwise the wider block runs along
    // them, forming (x~^H B)^H when x~ is the wider one.
    const int bit = cat == P_PROJ_HN ? TC_PROJ_HN : TC_GRAM;
    const bool use = tc < 0 ? tc_enabled(bit) : (tc == 1 && tc_device());
    if (!lower && use && tc_hn_supported(a, lda, b, ldb, k)) {
      Prof pr(cat + kProf32, st, ((double)m * sizeof(Va) + (double)n * sizeof(Vb)) * k + 16.0 * m * n,
              8.0 * m * n * (double)k);
      pr.count(1);
      if (cat == P_PROJ_HN && m > 64 && (n <= 64 || n > m))
        return tc_gemm_hn(b, ldb, a, lda, k, n, m, c, ldc, true, st, num_sms());
      return tc_gemm_hn(a, lda, b, ldb, k, m, n, c, ldc, false, st, num_sms());
    }
  }
  // 48-row tiles when they pad m less than 32-row tiles (not for the square lower-triangle mode)
  const bool rm3 = !lower && (m + 47) / 48 * 48 < (m + 31) / 32 * 32;
  const int tmr = rm3 ? 48 : HN_T;
  const int mt = (m + tmr - 1) / tmr, nt = (n + HN_T - 1) / HN_T;
  const int tiles = lower ? mt * (mt + 1) / 2 : mt * nt;
  const int ktiles = (k + HN_T - 1) / HN_T;
  int splits = std::max(1, (4 * num_sms()) / tiles);
  splits = std::min(splits, ktiles);
  const int kchunk = ((ktiles + splits - 1) / splits) * HN_T;
  splits = (k + kchunk - 1) / kchunk;
  dim3 grid(tiles, splits);
  const bool same = (const void*)a == (const void*)b;
  const bool f32 = sizeof(Va) == sizeof(float2) && sizeof(Vb) == sizeof(float2) && !Acc64;
  Prof pr(f32 && cat < P_RR ? cat + kProf32 : cat, st, (same ? (double)m * sizeof(Va) : (double)m * sizeof(Va) + (double)n * sizeof(Vb)) * k +
                       16.0 * m * n,
          (lower ? 4.0 * m * (m + 1.0) : 8.0 * m * n) * (double)k);
  using A = typename std::conditional<Acc64, double2, typename AccOf<Va, Vb>::T>::type;
  if constexpr (std::is_same<A, float2>::value && std::is_same<Va, float2>::value &&
                std::is_same<Vb, float2>::value) {
    static bool attr = false;
    if (!attr) {
      DKS_CUDA_TRY(cudaFuncSetAttribute((const void*)k_gemm_hn_f32p<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)hn32_smem<3>()));
      DKS_CUDA_TRY(cudaFuncSetAttribute((const void*)k_gemm_hn_f32p<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)hn32_smem<2>()));
      attr = true;
    }
    if (rm3)
      k_gemm_hn_f32p<3><<<grid, 256, hn32_smem<3>(), st>>>(a, lda, b, ldb, k, m, n, mt, kchunk, c, ldc, lower ? 1 : 0);
    else
      k_gemm_hn_f32p<2><<<grid, 256, hn32_smem<2>(), st>>>(a, lda, b, ldb, k, m, n, mt, kchunk, c, ldc, lower ? 1 : 0);
  } else if (rm3) {
    k_gemm_hn<Va, Vb, A, 3><<<grid, 256, 0, st>>>(a, lda, b, ldb, k, m, n, mt, kchunk, c, ldc, lower ? 1 : 0);
  } else {
    k_gemm_hn<Va, Vb, A, 2><<<grid, 256, 0, st>>>(a, lda, b, ldb, k, m, n, mt, kchunk, c, ldc, lower ? 1 : 0);
  }
  DKS_CUDA_TRY(cudaGetLastError());
  return DKS_OK;
}

int gram_f32(const float2* z, const float2* hz, int ld, int k, int m, double2* a, double2* s, cudaStream_t st) {
  if (m <= 0 || k <= 0) return DKS_OK;
  if (tc_enabled(TC_GRAM) && tc_hn_supported(z, ld, hz, ld, k) && tc_hn_supported(z, ld, z, ld, k))
    return tc_gram(z, hz, ld, k, m, a, s, st, num_sms());
  const int mt = (m + HN_T - 1) / HN_T;
  const int tiles = mt * (mt + 1) / 2;
  const int ktiles = (k + HN_T - 1) / HN_T;
  int splits = std::min(std::max(1, (4 * num_sms()) / tiles), ktiles);
  const int kchunk = ((ktiles + splits - 1) / splits) * HN_T;
  splits = (k + kchunk - 1) / kchunk;
  Prof pr(P_GRAM + kProf32, st, 2.0 * m * 8.0 * k + 32.0 * m * m, 8.0 * m * (m + 1.0) * (double)k);
  static bool attr = false;
  if (!attr) {
    DKS_CUDA_TRY(cudaFuncSetAttribute((const void*)k_gram_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)GF_SMEM));
    attr = true;
  }
  k_gram_f32<<<dim3(tiles, splits), GF_THREADS, GF_SMEM, st>>>(z, hz, ld, k, m, kchunk, a, s);
  DKS_CUDA_TRY(cudaGetLastError());
  return DKS_OK;
}

// a = diag(1, 2, ..., m) (m x m, column-major)
__global__ void k_set_diag_ramp(double2* __restrict__ a, int m) {
  const int total = m * m;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int i = e % m, j = e / m;
    a[e] = double2{i == j ? (double)(i + 1) : 0.0, 0.0};
  }
}

int set_diag_ramp(double2* a, int m, cudaStream_t st) {
  if (m <= 0) return DKS_OK;
  Prof pr(P_MISC, st, 16.0 * m * m, 0.0);
  k_set_diag_ramp<<<std::min(1024, (m * m + 255) / 256), 256, 0, st>>>(a, m);
  DKS_CUDA_TRY(cudaGetLastError());
  return DKS_OK;
}

// upper triangle of a Hermitian m x m matrix from its lower triangle
__global__ void k_mirror_lower(double2* __restrict__ c, int m) {
  const int total = m * m;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int i = e % m, j = e / m;
    if (i < j) {
      const double2 v = c[(size_t)i * m + j];
      c[e] = double2{v.x, -v.y};
    }
  }
}

int mirror_lower(double2* c, int m, cudaStream_t st) {
  if (m <= 1) return DKS_OK;
  Prof pr(P_MISC, st, 16.0 * m * m, 0.0);
  k_mirror_lower<<<std::min(1024, (m * m + 255) / 256), 256, 0, st>>>(c, m);
  DKS_CUDA_TRY(cudaGetLastError());
  return DKS_OK;
}

// ---------------------------------------------------------------- gemm_nn
constexpr int NN_R = 64, NN_C = 32, NN_M = 16;

template <typename Va, typename Vo>
__global__ void __launch_bounds__(256) k_gemm_nn(const Va* __restrict__ a, int lda, int k, int m,
                                                 const double2* __restrict__ w, int ldw,
                                                 const double* __restrict__ ws, int n, Vo* __restrict__ out,
                                                 int ldo, double alpha, double beta) {
  using A = typename AccOf<Va, Vo>::T;
  __shared__ A as[NN_M][NN_R];
  __shared__ A wsm[NN_M][NN_C];
  const int r0 = blockIdx.x * NN_R, c0 = blockIdx.y * NN_C;
  const int row = threadIdx.x & (NN_R - 1), cg = threadIdx.x >> 6;
  A acc[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) acc[j] = A{0, 0};
  for (int m0 = 0; m0 < m; m0 += NN_M) {
    for (int e = threadIdx.x; e < NN_M * NN_R; e += 256) {
      const int rr = e & (NN_R - 1), mm = e >> 6;
      A v{0, 0};
      if (m0 + mm < m && r0 + rr < k) v = cvt<A>(a[(size_t)(m0 + mm) * lda + r0 + rr]);
      as[mm][rr] = v;
    }
    for (int e = threadIdx.x; e < NN_M * NN_C; e += 256) {
      const int cc = e & (NN_C - 1), mm = e >> 5;
      double2 v{0, 0};
      if (m0 + mm < m && c0 + cc < n) {
        v = w[(size_t)(c0 + cc) * ldw + m0 + mm];
        const double s = (ws ? ws[m0 + mm] : 1.0) * alpha;
        v.x *= s;
        v.y *= s;
      }
      wsm[mm][cc] = cvt<A>(v);
    }
    __syncthreads();
#pragma unroll 4
    for (int mm = 0; mm < NN_M; ++mm) {
      const A av = as[mm][row];
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j] = cfma(av, wsm[mm][cg * 8 + j], acc[j]);
    }
    __syncthreads();
  }
  if (r0 + row < k) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int cc = c0 + cg * 8 + j;
      if (cc < n) {
        Vo* o = out + (size_t)cc * ldo + r0 + row;
        A r = acc[j];
        if (beta != 0.0) {
          const A old = cvt<A>(*o);
          r.x += (typename RealOf<A>::T)beta * old.x;
          r.y += (typename RealOf<A>::T)beta * old.y;
        }
        *o = from_d2<Vo>(to_d2(r));
      }
    }
  }
}

// FP32 operands and output: 256 rows x (8 * ncg) columns per CTA (ncg <= 5 column groups, sized
// to the number of output columns so that no column of the tile is padding), one thread per
// 4 rows (t, t+64, t+128, t+192) x 8 columns; the FP64 -> FP32 conversion of W is amortised
// over 256 rows and every shared-memory load of W feeds four complex multiply-adds.
constexpr int NF_R = 256, NF_GMAX = 5, NF_CMAX = 8 * NF_GMAX, NF_M = 16;

// Two shared-memory stages: the A chunk of the next 16 inner indices is copied with cp.async and
// the W chunk fetched into registers while the current chunk is multiplied.
constexpr size_t NF_SMEM = 2 * (size_t)NF_M * NF_R * sizeof(float2) + 2 * (size_t)NF_M * NF_CMAX * sizeof(float2);


__global__ void __launch_bounds__(64 * NF_GMAX, 2) k_gemm_nn_f32(const float2* __restrict__ a, int lda, int k, int m,
                                                     const double2* __restrict__ w, int ldw,
                                                     const double* __restrict__ ws, int n,
                                                     float2* __restrict__ out, int ldo, double alpha, float beta) {
  extern __shared__ __align__(16) unsigned char nf_smem[];
  float2* as_base = reinterpret_cast<float2*>(nf_smem);                          // [2][NF_M][NF_R]
  float2* ws_base = as_base + 2 * NF_M * NF_R;                                     // [2][NF_M][NF_CMAX]
  const int ncols = (blockDim.x >> 6) * 8;
  const int r0 = blockIdx.x * NF_R, c0 = blockIdx.y * ncols;
  const int rg = threadIdx.x & 63, cg = threadIdx.x >> 6;
  float2 acc[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = float2{0.f, 0.f};
  auto load_a = [&](int buf, int m0) {
    float2* dst = as_base + (size_t)buf * NF_M * NF_R;
    for (int e = threadIdx.x; e < NF_M * NF_R; e += blockDim.x) {
      const int rr = e & (NF_R - 1), mm = e >> 8;
      if (m0 + mm < m && r0 + rr < k) cp_async8(dst + e, a + (size_t)(m0 + mm) * lda + r0 + rr);
      else dst[e] = float2{0.f, 0.f};
    }
    cp_async_commit();
  };
  // W chunk: NF_M x ncols = 2 blockDim elements, two per thread, scaled and rounded to FP32
  auto fetch_w = [&](int m0, float2 (&wr)[2]) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int e = threadIdx.x + q * blockDim.x;
      const int mm = e / ncols, cc = e - mm * ncols;
      float2 v{0.f, 0.f};
      if (m0 + mm < m && c0 + cc < n) {
        const double2 wv = w[(size_t)(c0 + cc) * ldw + m0 + mm];
        const float s = (float)((ws ? ws[m0 + mm] : 1.0) * alpha);
        v = float2{(float)wv.x * s, (float)wv.y * s};
      }
      wr[q] = v;
    }
  };
  auto store_w = [&](int buf, const float2 (&wr)[2]) {
    float2* dst = ws_base + (size_t)buf * NF_M * NF_CMAX;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int e = threadIdx.x + q * blockDim.x;
      const int mm = e / ncols, cc = e - mm * ncols;
      dst[mm * NF_CMAX + cc] = wr[q];
    }
  };
  const int nch = (m + NF_M - 1) / NF_M;
  {
    float2 wr[2];
    load_a(0, 0);
    fetch_w(0, wr);
    store_w(0, wr);
  }
  for (int ch = 0; ch < nch; ++ch) {
    const int cur = ch & 1;
    const bool more = ch + 1 < nch;
    float2 wr[2];
    if (more) {
      load_a(cur ^ 1, (ch + 1) * NF_M);
      fetch_w((ch + 1) * NF_M, wr);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const float2* as = as_base + (size_t)cur * NF_M * NF_R;
    const float2* wsm = ws_base + (size_t)cur * NF_M * NF_CMAX;
#pragma unroll 2
    for (int mm = 0; mm < NF_M; ++mm) {
      float2 av[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = as[mm * NF_R + rg + 64 * i];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float2 wv = wsm[mm * NF_CMAX + cg * 8 + j];
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i][j] = cfma(av[i], wv, acc[i][j]);
      }
    }
    if (more) store_w(cur ^ 1, wr);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int row = r0 + rg + 64 * i;
    if (row >= k) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int cc = c0 + cg * 8 + j;
      if (cc < n) {
        float2* o = out + (size_t)cc * ldo + row;
        float2 r = acc[i][j];
        if (beta != 0.f) {
          const float2 old = *o;
          r.x += beta * old.x;
          r.y += beta * old.y;
        }
        *o = r;
      }
    }
  }
}

// column groups of 8 per CTA for n output columns: the fewest CTAs along n, then the
// smallest tile that covers n / (number of column tiles)
static int col_groups(int n, int maxg) {
  const int tiles = (n + 8 * maxg - 1) / (8 * maxg);
  const int per = (n + tiles - 1) / tiles;
  return std::max(1, (per + 7) / 8);
}

template <typename Va, typename Vo>
int gemm_nn(const Va* a, int lda, int k, int m, const double2* w, int ldw, const double* wscale, int n,
            Vo* out, int ldo, double beta, cudaStream_t st, double alpha, int cat, int tc) {
  if (k <= 0 || n <= 0) return DKS_OK;
  if constexpr (std::is_same<Va, float2>::value && std::is_same<Vo, float2>::value) {
    const int bit = cat == P_PROJ_NN ? TC_PROJ_NN : TC_ROTATE;
    const bool use = tc < 0 ? tc_enabled(bit) : (tc == 1 && tc_device());
    if (use && tc_nn_supported(a, lda, k, m, n)) {
      Prof pr(cat + kProf32, st, (double)m * k * sizeof(Va) + (beta != 0.0 ? 2.0 : 1.0) * n * k * sizeof(Vo) + 16.0 * m * n,
              8.0 * (double)k * m * n);
      return tc_gemm_nn(a, lda, k, m, w, ldw, wscale, n, out, ldo, beta, st, alpha, num_sms());
    }
  }
  const bool f32 = sizeof(Va) == sizeof(float2) && sizeof(Vo) == sizeof(float2);
  Prof pr(f32 && cat < P_RR ? cat + kProf32 : cat, st, (double)m * k * sizeof(Va) + (beta != 0.0 ? 2.0 : 1.0) * n * k * sizeof(Vo) + 16.0 * m * n,
          8.0 * (double)k * m * n);
  if constexpr (std::is_same<Va, float2>::value && std::is_same<Vo, float2>::value) {
    const int g = col_groups(n, NF_GMAX);
    dim3 grid((k + NF_R - 1) / NF_R, (n + NF_CMAX - 1) / NF_CMAX);
    static bool attr = false;
    if (!attr) {
      DKS_CUDA_TRY(cudaFuncSetAttribute((const void*)k_gemm_nn_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)NF_SMEM));
      attr = true;
    }
    k_gemm_nn_f32<<<grid, 64 * g, NF_SMEM, st>>>(a, lda, k, m, w, ldw, wscale, n, out, ldo, alpha, (float)beta);
  } else {
    dim3 grid((k + NN_R - 1) / NN_R, (n + NN_C - 1) / NN_C);
    k_gemm_nn<Va, Vo><<<grid, 256, 0, st>>>(a, lda, k, m, w, ldw, wscale, n, out, ldo, alpha, beta);
  }
  DKS_CUDA_TRY(cudaGetLastError());
  return DKS_OK;
}

// ---------------------------------------------------------------- column statistics
// One 8-CTA cluster per column: each CTA sums an eighth of the planewaves (all four
// components, so |k+G|^2/2 is read once per planewave), and CTA 0 of the cluster adds the
// eight partial sums from distributed shared memory in rank order (deterministic result).
constexpr int STATS_SPLIT = 8;

template <typename V, int NC>
__global__ void __cluster_dims__(STATS_SPLIT, 1, 1) __launch_bounds__(256)
    k_col_stats(const V* __restrict__ x, const V* __restrict__ hx, const double* __restrict__ lam,
                const double* __restrict__ ek, int npw, double* __restrict__ stats) {
  cg::cluster_group cl = cg::this_cluster();
  const int part = (int)cl.block_rank();
  const int j = blockIdx.y;
  const size_t rows = (size_t)NC * npw;
  const V* xj = x + (size_t)j * rows;
  const V* hj = hx ? hx + (size_t)j * rows : nullptr;
  const double l = lam ? lam[j] : 0.0;
  const int per = (npw + STATS_SPLIT - 1) / STATS_SPLIT;
  const int p0 = part * per, p1 = min(npw, p0 + per);
  // per-planewave sums in the working precision (the residual is formed in it), column sums in FP64
  using T = typename RealOf<V>::T;
  const T lt = (T)l;
  double s0 = 0, s1 = 0, s2 = 0;
  for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
    T ax = 0, rr = 0;
#pragma unroll
    for (int a = 0; a < NC; ++a) {
      const V xv = xj[(size_t)a * npw + p];
      ax = fma(xv.x, xv.x, fma(xv.y, xv.y, ax));
      if (hj) {
        const V hv = hj[(size_t)a * npw + p];
        const T rx = fma(-lt, xv.x, hv.x), ry = fma(-lt, xv.y, hv.y);
        rr = fma(rx, rx, fma(ry, ry, rr));
      }
    }
    s0 += (double)rr;
    s1 += (double)ax;
    s2 = fma(ek[p], (double)ax, s2);
  }
  __shared__ double red[3][8];
  __shared__ double part_sum[3];
  for (int off = 16; off; off >>= 1) {
    s0 += __shfl_down_sync(0xffffffffu, s0, off);
    s1 += __shfl_down_sync(0xffffffffu, s1, off);
    s2 += __shfl_down_sync(0xffffffffu, s2, off);
  }
  const int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
  if (ln == 0) {
    red[0][w] = s0;
    red[1][w] = s1;
    red[2][w] = s2;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[threadIdx.x][i];
    part_sum[threadIdx.x] = t;
  }
  cl.sync();
  if (part == 0 && threadIdx.x < 3) {
    double t = 0;
    for (int r = 0; r < STATS_SPLIT; ++r) t += *cl.map_shared_rank(&part_sum[threadIdx.x], r);
    stats[3 * j + threadIdx.x] = t;
  }
  cl.sync();   // the other CTAs keep their shared memory until rank 0 has read it
}

template <typename V>
int col_stats(const V* x, const V* hx, const double* lam, const double* ek, int npw, int n, double* stats,
              cudaStream_t st, int ncomp) {
  if (n <= 0) return DKS_OK;
  if (n > 65535) return fail(DKS_ERR_INVALID_ARG, "col_stats: too many columns");
  Prof pr(P_STATS, st, (hx ? 2.0 : 1.0) * n * ncomp * npw * sizeof(V) + 8.0 * npw, 12.0 * n * ncomp * npw);
  if (ncomp == 2)
    k_col_stats<V, 2><<<dim3(STATS_SPLIT, n), 256, 0, st>>>(x, hx, lam, ek, npw, stats);
  else
    k_col_stats<V, 4><<<dim3(STATS_SPLIT, n), 256, 0, st>>>(x, hx, lam, ek, npw, stats);
  DKS_CUDA_TRY(cudaGetLastError());
  return DKS_OK;
}

// ---------------------------------------------------------------- Teter preconditioner
// grid (planewave blocks, active columns): the per-column Teter scale 1/T_band is formed once
// per thread; each thread then takes planewaves p and all four components, so |k+G|^2/2 is read
// once per planewave and the Teter factor computed once for the four components
template <typename V, typename Vo, int NC>
__global__ void k_precond(const V* __restrict__ x, const V* __restrict__ hx, const double* __restrict__ lam,
                          const double* __restrict__ stats, const int* __restrict__ act,
                          const double* __restrict__ ek, int npw, int precond, Vo* __restrict__ y) {
  using T = typename RealOf<V>::T;
  const int i = blockIdx.y;
  const int j = act[i];
  const size_t rows = (size_t)NC * npw;
  const V* xj = x + (size_t)j * rows;
  const V* hj = hx + (size_t)j * rows;
  Vo* yi = y + (size_t)i * rows;
  const T l = (T)lam[j];
  const double tb = fmax(stats[3 * j + 2] / fmax(stats[3 * j + 1], 1e-300), 1e-12);
  const T itb = (T)(1.0 / tb);
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npw; p += gridDim.x * blockDim.x) {
    T kf = (T)1;
    if (precond == DKS_PRECOND_TETER) {
      const T xx = (T)ek[p] * itb;
      const T pp = (T)27 + xx * ((T)18 + xx * ((T)12 + xx * (T)8));
      const T x2 = xx * xx;
      kf = pp / (pp + (T)16 * x2 * x2);
    }
#pragma unroll
    for (int a = 0; a < NC; ++a) {
      const V xv = xj[(size_t)a * npw + p], hv = hj[(size_t)a * npw + p];
      const V r{kf * (hv.x - l * xv.x), kf * (hv.y - l * xv.y)};
      if constexpr (std::is_same<V, Vo>::value) {
        yi[(size_t)a * npw + p] = r;
      } else {
        yi[(size_t)a * npw + p] = from_d2<Vo>(to_d2(r));
      }
    }
  }
}

template <typename V, typename Vo>
int precond_apply(const V* x, const V* hx, const double* lam, const double* stats, const int* act, int nact,
                  const double* ek, int npw, int precond, Vo* y, cudaStream_t st, int ncomp) {
  if (nact <= 0) return DKS_OK;
  if (nact > 65535) return fail(DKS_ERR_INVALID_ARG, "precond: too many columns");
  const size_t total = (size_t)ncomp * npw * nact;
  const int bx = std::max(1, std::min((npw + 255) / 256, (num_sms() * 8 + nact - 1) / nact));
  Prof pr(P_PRECOND, st, 3.0 * total * sizeof(V) + 8.0 * npw, 20.0 * total);
  if (ncomp == 2)
    k_precond<V, Vo, 2><<<dim3(bx, nact), 256, 0, st>>>(x, hx, lam, stats, act, ek, npw, precond, y);
  else
    k_precond<V, Vo, 4><<<dim3(bx, nact), 256, 0, st>>>(x, hx, lam, stats, act, ek, npw, precond, y);
  DKS_CUDA_TRY(cudaGetLastError());
  return DKS_OK;
}

// ---------------------------------------------------------------- conversions and gathers
template <typename Vi, typename Vo>
__global__ void k_convert(const Vi* __restrict__ in, Vo* __restrict__ out, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    out[e] = from_d2<Vo>(to_d2(in[e]));
}

template <typename Vi, typename Vo>
int convert(const Vi* in, Vo* out, size_t n, cudaStream_t st) {
  if (!n) return DKS_OK;
  const int blocks = (int)std::min<size_t>((n + 255) / 256, (size_t)num_sms() * 16);
  Prof pr(P_MISC, st, (double)n * (sizeof(Vi) + sizeof(Vo)), 0.0);
  k_convert<Vi, Vo><<<blocks, 256, 0, st>>>(in, out, n);
  DKS_CUDA_TRY(cudaGetLastError());
  return DKS_OK;
}

__global__ void k_gather_cols(const double2* __restrict__ v, int ldv, int row0, int rows,
                              const int* __restrict__ act, int nact, double2* __restrict__ out) {
  const int total = rows * nact;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int i = e / rows, r = e - i * rows;
    out[e] = v[(size_t)act[i] * ldv + row0 + r];
  }
}

int gather_cols(const double2* v, int ldv, int row0, int rows, const int* act, int nact, double2* out,
                cudaStream_t st) {
  if (rows <= 0 || nact <= 0) return DKS_OK;
  const int total = rows * nact;
  Prof pr(P_MISC, st, 32.0 * total, 0.0);
  k_gather_cols<<<std::min((total + 255) / 256, 1024), 256, 0, st>>>(v, ldv, row0, rows, act, nact, out);
  DKS_CUDA_TRY(cudaGetLastError());
  return DKS_OK;
}

// explicit instantiations
#define DKS_INST_HN(TA, TB, ACC)                                                                        \
  template int gemm_hn<TA, TB, ACC>(const TA*, int, const TB*, int, int, int, int, double2*, cudaStream_t, int, \
                                    int, bool, int);
DKS_INST_HN(double2, double2, false)
DKS_INST_HN(float2, float2, false)
DKS_INST_HN(float2, float2, true)
DKS_INST_HN(double2, float2, false)
DKS_INST_HN(float2, double2, false)
template int gemm_nn<double2, double2>(const double2*, int, int, int, const double2*, int, const double*, int,
                                       double2*, int, double, cudaStream_t, double, int, int);
template int gemm_nn<float2, float2>(const float2*, int, int, int, const double2*, int, const double*, int,
                                     float2*, int, double, cudaStream_t, double, int, int);
template int gemm_nn<float2, double2>(const float2*, int, int, int, const double2*, int, const double*, int,
                                      double2*, int, double, cudaStream_t, double, int, int);
template int col_stats<double2>(const double2*, const double2*, const double*, const double*, int, int, double*,
                                cudaStream_t, int);
template int col_stats<float2>(const float2*, const float2*, const double*, const double*, int, int, double*,
                               cudaStream_t, int);
template int precond_apply<double2, double2>(const double2*, const double2*, const double*, const double*,
                                             const int*, int, const double*, int, int, double2*, cudaStream_t, int);
template int precond_apply<float2, float2>(const float2*, const float2*, const double*, const double*, const int*,
                                           int, const double*, int, int, float2*, cudaStream_t, int);
template int precond_apply<double2, float2>(const double2*, const double2*, const double*, const double*,
                                            const int*, int, const double*, int, int, float2*, cudaStream_t, int);
template int convert<double2, float2>(const double2*, float2*, size_t, cudaStream_t);
template int convert<float2, double2>(const float2*, double2*, size_t, cudaStream_t);
template int convert<double2, double2>(const double2*, double2*, size_t, cudaStream_t);

}  // namespace dks

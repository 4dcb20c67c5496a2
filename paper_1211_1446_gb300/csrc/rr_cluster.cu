// FP64 Rayleigh-Ritz on a thread-block cluster (Cholesky path of Algorithm 1's Rayleigh-Ritz steps).
//
// FP64 throughput on GB300 is about two FMAs per clock per SM, so the O(m^3) work of the
// small pencil is spread over the SMs of one cluster (16 CTAs when the device allows
// non-portable clusters, else 8).  Matrices stay in a global scratch area (L2-resident);
// the cluster barrier (release/acquire at cluster scope) orders the dependent steps.  Serial
// chains read their operands from shared memory: blocks of L and of the reflectors are staged
// there, since every dependent global load after a cluster barrier costs an L2 round trip.
//
//  1. A' = D A D, S' = D S D, D = diag(S)^-1/2                     (element-parallel)
//  2. S' = L L^H, right-looking, one barrier per column; if a pivot^2 falls below
//     chol_tol the kernel records it and returns -- the single-CTA kernel then runs
//     the SVQB path
//  3. W = L^-1 A' and C = L^-1 W^H = L^-1 A' L^-H: column-oriented forward substitution,
//     warp per right-hand side, no reductions
//  4. Householder reduction of C to a complex tridiagonal with the columns of C distributed
//     over the shared memories of the cluster (column j in CTA j % csize); reflectors and
//     p = tau C v travel through distributed shared memory; two barriers per column
//  5. real tridiagonal by a diagonal phase; the n lowest eigenvalues by 33-way
//     multisection of the Sturm count (warp per eigenvalue): FP32 counts, then
//     double-float counts
//  6. eigenvectors by inverse iteration on the tridiagonal (LU with partial pivoting in
//     shared memory, one lane per vector); vectors of a cluster of close eigenvalues are
//     computed by one lane in turn and orthogonalised against each other
//  7. y = Phi z, Householder back-transformation, V = D L^-H U    (warp per column)
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cstdio>

#include "dks_internal.h"
#include "dks_kernels.cuh"

namespace cg = cooperative_groups;

namespace dks {

constexpr int RRC_THREADS = 512;
constexpr int RRC_WARPS = RRC_THREADS / 32;
static_assert(RRC_THREADS >= kMaxRR - 1, "one Householder row per thread");

// Phase timer for development builds (-DDKS_RR_TIMING): CTA 0, thread 0 prints the
// nanoseconds spent between the marks of the algorithm steps.
#ifdef DKS_RR_TIMING
#define RR_MARK(i) \
  if (gtid == 0) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(tmark[i]))
// RR_LAP(i): SM cycles since the previous lap mark added to lap slot i (CTA 0, thread 0)
#define RR_LAP(i)                                          \
  if (gtid == 0) {                                         \
    const unsigned long long c_ = clock64();               \
    tlap[i] += c_ - tlast;                                 \
    tlast = c_;                                            \
  }
#else
#define RR_MARK(i)
#define RR_LAP(i)
#endif

// Reciprocal and square root for the serial chains: FP64 division and square root are long
// instruction sequences on this part, so they are replaced by Newton-Raphson iterations
// (x <- x + x (1 - a x) for 1/a, y <- y (3 - a y^2)/2 for 1/sqrt(a)) in FP64 FMAs, seeded by the
// FP32 approximations; each iteration squares the relative error, so two take the ~1e-7 seed
// below FP64 rounding.  Outside the FP32 normal range the exact operations are used.
__device__ __forceinline__ bool f32_range(double a) {
  const double m = fabs(a);
  return m > 1e-37 && m < 1e37;
}
__device__ __forceinline__ double nr_rcp(double a) {
  if (!f32_range(a)) return 1.0 / a;
  double x = (double)__frcp_rn((float)a);
  x = fma(x, fma(-a, x, 1.0), x);
  x = fma(x, fma(-a, x, 1.0), x);
  return x;
}
__device__ __forceinline__ double nr_rsqrt(double a) {
  if (!f32_range(a) || a < 0) return 1.0 / sqrt(a);
  double y = (double)rsqrtf((float)a);
  const double h = 0.5 * a;
  y = y * fma(-h * y, y, 1.5);
  y = y * fma(-h * y, y, 1.5);
  return y;
}
__device__ __forceinline__ double nr_sqrt(double a) { return a == 0.0 ? 0.0 : a * nr_rsqrt(a); }
// 1/a for a > 0, with the range test done on the FP32 value (fewer FP64 instructions)
__device__ __forceinline__ double rcp_pos(double a) {
  const float af = __double2float_rn(a);
  if (!(af > 1e-37f && af < 1e37f)) return 1.0 / a;
  double x = (double)__frcp_rn(af);
  x = fma(x, fma(-a, x, 1.0), x);
  return fma(x, fma(-a, x, 1.0), x);
}
__device__ __forceinline__ double nr_hypot(double x, double y) {
  const double s = fmax(fabs(x), fabs(y));
  if (s == 0.0) return 0.0;
  const double r = nr_rcp(s), xs = x * r, ys = y * r;
  return s * nr_sqrt(xs * xs + ys * ys);
}

__device__ __forceinline__ double2 warp_csum(double2 v) {
  for (int o = 16; o; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// double-float helpers for the distributed Householder steps
__device__ __forceinline__ dfl dd_fma(dfl x, dfl y, dfl acc) {   // acc + x y
  const float p = x.h * y.h;
  float e = fmaf(x.h, y.h, -p);
  e = fmaf(x.h, y.l, e);
  e = fmaf(x.l, y.h, e);
  const float t = acc.h + p;
  const float bb = t - acc.h;
  const float lo = ((acc.h - (t - bb)) + (p - bb)) + (acc.l + e);
  const float h = t + lo;
  return dfl{h, lo - (h - t)};
}
__device__ __forceinline__ cdf cdf0() { return cdf{{0.f, 0.f}, {0.f, 0.f}}; }
__device__ __forceinline__ cdf ucdf(float4 v) { return cdf{{v.x, v.y}, {v.z, v.w}}; }
__device__ __forceinline__ float4 c4(cdf c) { return float4{c.re.h, c.re.l, c.im.h, c.im.l}; }
__device__ __forceinline__ float4 c4(double2 v) { return c4(cdf{df_from(v.x), df_from(v.y)}); }
__device__ __forceinline__ cdf cdf_fmac(cdf a, cdf b, cdf acc) {   // acc + conj(a) b
  acc.re = dd_fma(a.re, b.re, acc.re);
  acc.re = dd_fma(a.im, b.im, acc.re);
  acc.im = dd_fma(a.re, b.im, acc.im);
  acc.im = dd_fma(df_neg(a.im), b.re, acc.im);
  return acc;
}
__device__ __forceinline__ dfl warp_dsum(dfl v) {
  for (int o = 16; o; o >>= 1)
    v = df_add(v, dfl{__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)});
  return v;
}
__device__ __forceinline__ cdf warp_cdsum(cdf v) {
  v.re = warp_dsum(v.re);
  v.im = warp_dsum(v.im);
  return v;
}

// number of eigenvalues of the real symmetric tridiagonal (d, e) below x (Sturm count): the
// negative pivots of the LDL^T factorisation of T - x I, each pivot kept away from zero
__device__ int sturm_count_f(const float* d, const float* e2, int m, float x, float pivmin) {
  int cnt = 0;
  float q = d[0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  cnt += q < 0.f;
  for (int j = 1; j < m; ++j) {
    q = d[j] - x - __fdividef(e2[j - 1], q);
    if (fabsf(q) < pivmin) q = -pivmin;
    cnt += q < 0.f;
  }
  return cnt;
}

// a / b in double-float: quotient of the leading parts, one correction from the exact
// remainder a - q1 b (Dekker)
__device__ __forceinline__ dfl df_div(dfl a, dfl b) {
  const float rb = __frcp_rn(b.h);
  const float q1 = a.h * rb;
  const float p = q1 * b.h;
  const float pe = fmaf(q1, b.h, -p);
  const float r = ((a.h - p) - pe) + (a.l - q1 * b.l);
  const float q2 = r * rb;
  const float h = q1 + q2;
  return dfl{h, q2 - (h - q1)};
}

// sqrt(a) in double-float, a >= 0: s0 = fl32(sqrt(a.h)), then one correction from the exact
// remainder a - s0^2 (for a correctly rounded s0, a.h - s0^2 is representable in FP32)
__device__ __forceinline__ dfl df_sqrt(dfl a) {
  if (!(a.h > 0.f)) return dfl{0.f, 0.f};
  const float s0 = sqrtf(a.h);
  const float r = fmaf(-s0, s0, a.h) + a.l;
  const float c = r * (0.5f * __frcp_rn(s0));
  const float h = s0 + c;
  return dfl{h, c - (h - s0)};
}

// Sturm count in double-float arithmetic (same recurrence as above)
__device__ int sturm_count_df(const dfl* d, const dfl* e2, int m, dfl x, float pivmin) {
  const dfl nx = df_neg(x);
  int cnt = 0;
  dfl q = df_add(d[0], nx);
  if (fabsf(q.h) < pivmin) q = dfl{-pivmin, 0.f};
  cnt += q.h < 0.f;
  for (int j = 1; j < m; ++j) {
    q = df_add(df_add(d[j], nx), df_neg(df_div(e2[j - 1], q)));
    if (fabsf(q.h) < pivmin) q = dfl{-pivmin, 0.f};
    cnt += q.h < 0.f;
  }
  return cnt;
}

// deterministic start vector in (-1, 1)
__device__ __forceinline__ float start_val(int i, int v) {
  unsigned h = (unsigned)(i * 2654435761u) ^ (unsigned)(v * 40503u + 12345u);
  h ^= h >> 13;
  h *= 0x5bd1e995u;
  h ^= h >> 15;
  return (float)(h & 0xffffff) * (1.0f / 8388608.0f) - 1.0f;   // exact in FP32
}

// Inverse iteration on the real tridiagonal: solve (T - lam I) x = b in place (x holds b on
// entry) with the factors of tridiagonal Gaussian elimination with partial pivoting.  Rows are
// processed top-down; at step i the pivot is the larger of the current diagonal and the
// subdiagonal below it.
// The elimination and solve run in double-float arithmetic on the FP32 lanes (one lane runs a
// whole vector, so every step is a dependent chain: a double-float step is a few FP32
// instructions deep, an FP64 step a whole FP64-unit warp instruction).  f: 5m double-float
// slots (U diagonal reciprocals, two superdiagonals, multipliers, pivot flags).
__device__ void tri_factor_df(const dfl* d, const dfl* e, int m, dfl lam, float tiny, dfl* f) {
  dfl* u0 = f;
  dfl* u1 = f + m;
  dfl* u2 = f + 2 * m;
  dfl* l = f + 3 * m;
  dfl* piv = f + 4 * m;
  const dfl zero{0.f, 0.f}, nl = df_neg(lam);
  dfl a = df_add(d[0], nl);
  dfl b = m > 1 ? e[0] : zero;
  for (int i = 0; i < m - 1; ++i) {
    const dfl c = e[i];
    const dfl dn = df_add(d[i + 1], nl);
    const dfl bn = i + 1 < m - 1 ? e[i + 1] : zero;
    if (fabsf(a.h) >= fabsf(c.h)) {
      piv[i] = zero;
      if (a.h == 0.f) a = dfl{tiny, 0.f};
      const dfl mult = df_div(c, a);
      l[i] = mult;
      u0[i] = a;
      u1[i] = b;
      u2[i] = zero;
      a = dd_fma(df_neg(mult), b, dn);
      b = bn;
    } else {
      piv[i] = dfl{1.f, 0.f};
      const dfl mult = df_div(a, c);
      l[i] = mult;
      u0[i] = c;
      u1[i] = dn;
      u2[i] = bn;
      a = dd_fma(df_neg(mult), dn, b);
      b = df_neg(df_mul(mult, bn));
    }
  }
  if (a.h == 0.f) a = dfl{tiny, 0.f};
  u0[m - 1] = a;
  u1[m - 1] = zero;
  u2[m - 1] = zero;
  for (int i = 0; i < m; ++i) u0[i] = df_div(dfl{1.f, 0.f}, u0[i]);
}

__device__ void tri_solve_df(int m, const dfl* f, dfl* x) {
  const dfl* u0 = f;
  const dfl* u1 = f + m;
  const dfl* u2 = f + 2 * m;
  const dfl* l = f + 3 * m;
  const dfl* piv = f + 4 * m;
  for (int i = 0; i < m - 1; ++i) {
    if (piv[i].h != 0.f) {
      const dfl t = x[i];
      x[i] = x[i + 1];
      x[i + 1] = dd_fma(df_neg(l[i]), x[i], t);
    } else {
      x[i + 1] = dd_fma(df_neg(l[i]), x[i], x[i + 1]);
    }
  }
  x[m - 1] = df_mul(x[m - 1], u0[m - 1]);
  if (m > 1) x[m - 2] = df_mul(dd_fma(df_neg(u1[m - 2]), x[m - 1], x[m - 2]), u0[m - 2]);
  for (int i = m - 3; i >= 0; --i)
    x[i] = df_mul(dd_fma(df_neg(u2[i]), x[i + 2], dd_fma(df_neg(u1[i]), x[i + 1], x[i])), u0[i]);
}

// x <- x / |x| in double-float: scaled by a power of two first (exact), so that the squares stay
// inside the FP32 range whatever the growth of the inverse-iteration solve
__device__ void df_normalize(int m, dfl* x) {
  float amax = 0.f;
  for (int i = 0; i < m; ++i) amax = fmaxf(amax, fabsf(x[i].h));
  if (!(amax > 0.f) || !(amax < INFINITY)) return;
  int ex;
  frexpf(amax, &ex);
  const float sc = ldexpf(1.f, -ex);
  dfl a0{0.f, 0.f}, a1{0.f, 0.f};   // two independent chains
  int i = 0;
  for (; i + 1 < m; i += 2) {
    const dfl y0{x[i].h * sc, x[i].l * sc}, y1{x[i + 1].h * sc, x[i + 1].l * sc};
    a0 = dd_fma(y0, y0, a0);
    a1 = dd_fma(y1, y1, a1);
  }
  if (i < m) {
    const dfl y0{x[i].h * sc, x[i].l * sc};
    a0 = dd_fma(y0, y0, a0);
  }
  const dfl nrm = df_add(a0, a1);
  const dfl r = df_div(dfl{sc, 0.f}, df_sqrt(nrm));
  for (int i = 0; i < m; ++i) x[i] = df_mul(x[i], r);
}

__host__ __device__ inline size_t rr_tri_smem_offset(int m) {
  const size_t vec = (size_t)RRC_WARPS * m * sizeof(double2);
  return vec > 48 * 1024 ? vec : 48 * 1024;
}
__host__ __device__ inline size_t rr_stage_offset(int m) {
  const size_t tri = rr_tri_smem_offset(m) + (size_t)m * (3 * sizeof(double) + 2 * sizeof(float) + 2 * sizeof(dfl)) + 64;
  return (tri + 15) / 16 * 16;
}
__host__ __device__ inline size_t rr_cluster_smem(int m, int scols) {
  return rr_stage_offset(m) + (size_t)scols * m * sizeof(double2) + (size_t)m * (3 * sizeof(double) + sizeof(double2));
}
constexpr size_t kRrSmemMax = 200 * 1024;

__global__ void __launch_bounds__(RRC_THREADS, 1) k_rr_cluster(const double2* __restrict__ A,
                                                            const double2* __restrict__ S, int m, int n,
                                                            double2* __restrict__ V, double* __restrict__ lam,
                                                            int* __restrict__ info, double2* __restrict__ scr,
                                                            double chol_tol, int scols, int phase) {
  extern __shared__ __align__(16) unsigned char rrc_smem[];
  cg::cluster_group cl = cg::this_cluster();
  const int crank = (int)cl.block_rank(), csize = (int)cl.num_blocks();
  const int tid = threadIdx.x, lane = tid & 31, wl = tid >> 5;
  const int gtid = crank * RRC_THREADS + tid, gnt = csize * RRC_THREADS;
  const int gw = crank * RRC_WARPS + wl, gnw = csize * RRC_WARPS;
  const size_t mm = (size_t)m * m;
#ifdef DKS_RR_TIMING
  unsigned long long tmark[10] = {0};
  unsigned long long tlap[8] = {0}, tlast = clock64(), town[3] = {0, 0, 0};
#endif
  RR_MARK(0);
  double2* am = scr;           // A' (full Hermitian)
  double2* lm = am + mm;       // working copy for the Cholesky trailing updates
  double2* lf = lm + mm;       // L, column-major
  double2* lt = lf + mm;       // L, row-major (rows contiguous)
  double2* cm = lt + mm;       // W, then C (full), then Householder vectors
  double* dsc = reinterpret_cast<double*>(cm + mm);
  double* dd = dsc + m;
  double* ee = dd + m;
  double* e2 = ee + m;
  double* lamw = e2 + m;       // wanted eigenvalues
  // six m-length double arrays (one spare) keep the complex arrays below 16-byte aligned for odd m
  double2* tau = reinterpret_cast<double2*>(lamw + 2 * m);
  double2* ph = tau + m;
  double2* pv = ph + m;
  int* flag = reinterpret_cast<int*>(pv + m);
  double* zt = reinterpret_cast<double*>(lm);   // m x n real eigenvectors of T (after Cholesky)

  // staging area and per-index scalars in shared memory
  double2* stg = reinterpret_cast<double2*>(rrc_smem + rr_stage_offset(m));   // scols x m
  double2* sph = stg + (size_t)scols * m;              // complex arrays first: 16-byte aligned
  double* slinv = reinterpret_cast<double*>(sph + m);
  double* stau = slinv + m;
  double* sdsc = stau + m;

  double2* cc = lm;   // C = L^-1 A' L^-H from the second triangular solve (k_rr_trsm)
  if (phase == 0) {
  // 1. scaling (every CTA keeps D in shared memory)
  for (int i = tid; i < m; i += RRC_THREADS) {
    const double di = nr_rsqrt(fmax(S[(size_t)i * m + i].x, 1e-300));
    sdsc[i] = di;
    if (crank == 0) dsc[i] = di;
  }
  __syncthreads();
  // Distributed form when the owned columns fit in shared memory: column j of S' lives in
  // CTA j % csize.  Step j: every CTA copies the published column j (rows > j) and 1 / pivot
  // from its owner; the owner of column j+1 updates that column first (whole CTA), publishes
  // it with its reciprocal pivot, then every CTA updates its remaining owned columns; one
  // cluster barrier per column.
  const int ncol_own = (m + csize - 1) / csize;
  const bool dist = scols >= ncol_own + 3;
  for (size_t e = gtid; e < mm; e += gnt) {
    const int i = (int)(e % m), j = (int)(e / m);
    const double s = sdsc[i] * sdsc[j];
    const double2 a = A[e], at = A[(size_t)i * m + j];
    am[e] = double2{0.5 * s * (a.x + at.x), 0.5 * s * (a.y - at.y)};
    if (!dist) {
      const double2 b = S[e], bt = S[(size_t)i * m + j];
      lm[e] = double2{0.5 * s * (b.x + bt.x), 0.5 * s * (b.y - bt.y)};
    }
  }
  __shared__ double chol_s;   // 1 / pivot of the current column (negative: not positive definite)
  bool failed = false;
  if (dist) {
    double2* cb = stg;                               // owned columns, column j at (j / csize) * m
    double2* colb = stg + (size_t)ncol_own * m;      // the column this CTA publishes; [m].x = 1 / pivot
    double2* colj = colb + (m + 1);                  // local copy of the current column
    for (int e = tid; e < ncol_own * m; e += RRC_THREADS) {
      const int lj = e / m, r = e - lj * m, j = lj * csize + crank;
      if (j < m) {
        const double s = sdsc[r] * sdsc[j];
        const double2 b = S[(size_t)j * m + r], bt = S[(size_t)r * m + j];
        cb[e] = double2{0.5 * s * (b.x + bt.x), 0.5 * s * (b.y - bt.y)};
      }
    }
    __syncthreads();
    auto publish = [&](int j) {   // whole CTA; column j is owned here and final
      const double2* cj = cb + (size_t)(j / csize) * m;
      for (int i = j + 1 + tid; i < m; i += RRC_THREADS) colb[i] = cj[i];
      if (tid == 0) {
        const double piv = cj[j].x;
        colb[m] = double2{piv > chol_tol ? rcp_pos(piv) : -1.0, 0.0};
      }
    };
    auto updc = [&](int lk, int i, double inv2) {   // lm[i, k] -= conj(l_kj) l_ij / pivot, i >= k
      const int k = lk * csize + crank;
      if (k >= m || i < k) return;
      double2* c = cb + (size_t)lk * m + i;
      const double2 u = cmulc(colj[k], colj[i]);
      *c = double2{fma(-u.x, inv2, c->x), fma(-u.y, inv2, c->y)};
    };
    if (crank == 0) publish(0);
    cl.sync();
    RR_LAP(7);
    for (int j = 0; j < m; ++j) {
      const int len = m - j - 1;
      const double2* src = cl.map_shared_rank(colb, (unsigned)(j % csize));
      const int r = j + 1 + tid;   // one row per thread (m <= RRC_THREADS + 1)
      double2 x = double2{0.0, 0.0};
      if (r < m) x = src[r];
      if (tid == 0) chol_s = src[m].x;
      if (r < m) colj[r] = x;
      __syncthreads();
      const double inv2 = chol_s;
      if (!(inv2 > 0.0)) {   // the same published value decides in every CTA
        failed = true;
        break;
      }
      RR_LAP(0);
      const int lj0 = (j + 1 - crank + csize - 1) / csize;   // first owned column > j
      const bool next = j + 1 < m && crank == (j + 1) % csize;
      if (next) {
        if (r < m) updc(lj0, r, inv2);
        __syncthreads();
        publish(j + 1);
      }
      const int l1 = lj0 + (next ? 1 : 0);
      for (int e = tid; e < (ncol_own - l1) * len; e += RRC_THREADS) {
        const int q = e / len;
        updc(l1 + q, j + 1 + (e - q * len), inv2);
      }
      RR_LAP(1);
      cl.sync();
      RR_LAP(2);
    }
    if (failed) {
      cl.sync();   // no CTA leaves while another may still read its published column
    } else {
      // L_ij = lm_ij / sqrt(lm_jj) (i > j), L_jj = sqrt(lm_jj), and 1 / L_ii, from the owned columns
      double* linv = lamw + m;
      for (int e = tid; e < ncol_own * m; e += RRC_THREADS) {
        const int lj = e / m, i = e - lj * m, j = lj * csize + crank;
        if (j >= m || i < j) continue;
        const double piv = cb[(size_t)lj * m + j].x;
        const double inv = nr_rsqrt(piv);
        const double2 c = cb[e];
        const double2 v = i == j ? double2{piv * inv, 0.0} : double2{c.x * inv, c.y * inv};
        lf[(size_t)j * m + i] = v;
        lt[(size_t)i * m + j] = v;
        if (i == j) linv[j] = inv;
      }
    }
  } else {
  cl.sync();
  // 2. Cholesky: column j of L from the (final) column j of lm; trailing update in lm.
  // Every thread reads the same pivot, so the failure decision is uniform over the cluster.
  // Right-looking on the unscaled columns: lm[:, k] -= conj(lm_kj) lm[:, j] / lm_jj, so the
  // critical path of a column is one reciprocal (formed once per CTA by thread 0 and shared)
  // and the trailing update; every thread loads its first trailing element before the
  // reciprocal is known.  L is formed from the final columns in one pass after the loop.
  RR_LAP(7);
  for (int j = 0; j < m; ++j) {
    const int len = m - j - 1;
    const double2* colj = lm + (size_t)j * m;
    int i0 = 0, k0 = 0;
    bool has0 = false;
    double2 lij0{0, 0}, lkj0{0, 0}, c00{0, 0};
    if (gtid < len * len) {
      i0 = j + 1 + gtid % len;
      k0 = j + 1 + gtid / len;
      if (k0 <= i0) {
        has0 = true;
        lij0 = colj[i0];
        lkj0 = colj[k0];
        c00 = lm[(size_t)k0 * m + i0];
      }
    }
    if (tid == 0) {
      const double piv = colj[j].x;
      chol_s = piv > chol_tol ? rcp_pos(piv) : -1.0;
    }
    __syncthreads();
    const double inv2 = chol_s;
    if (!(inv2 > 0.0)) {   // the same global pivot decides in every CTA
      failed = true;
      break;
    }
    RR_LAP(0);
    // trailing update lm[:, k] -= conj(l_kj) l_ij / pivot for j < k <= i
    if (has0) {
      const double2 u = cmulc(lkj0, lij0);
      lm[(size_t)k0 * m + i0] = double2{fma(-u.x, inv2, c00.x), fma(-u.y, inv2, c00.y)};
    }
    for (int e = gtid + gnt; e < len * len; e += gnt) {
      const int i = j + 1 + e % len, k = j + 1 + e / len;
      if (k <= i) {
        const double2 u = cmulc(colj[k], colj[i]);
        double2* c = lm + (size_t)k * m + i;
        *c = double2{fma(-u.x, inv2, c->x), fma(-u.y, inv2, c->y)};
      }
    }
    RR_LAP(1);
    cl.sync();
    RR_LAP(2);
  }
  if (!failed) {
    // L_ij = lm_ij / sqrt(lm_jj) (i > j), L_jj = sqrt(lm_jj), and 1 / L_ii (the spare m-array)
    double* linv = lamw + m;
    for (size_t e = gtid; e < mm; e += gnt) {
      const int i = (int)(e % m), j = (int)(e / m);
      if (i < j) continue;
      const double piv = lm[(size_t)j * m + j].x;
      const double inv = nr_rsqrt(piv);
      const double2 c = lm[e];
      const double2 v = i == j ? double2{piv * inv, 0.0} : double2{c.x * inv, c.y * inv};
      lf[e] = v;
      lt[(size_t)i * m + j] = v;
      if (i == j) linv[i] = inv;
    }
  }
  }
  if (failed) {
    if (gtid == 0) *flag = 1;
    return;   // every CTA leaves here; the single-CTA SVQB kernel that follows takes over
  }
  if (gtid == 0) *flag = 0;
#ifdef DKS_RR_TIMING
  RR_MARK(1);
  if (gtid == 0) printf("rr_cluster m=%d n=%d csize=%d: scaling+cholesky %.1f us (cycles: pivot %llu update %llu sync %llu)\n", m, n, csize, (tmark[1] - tmark[0]) * 1e-3, tlap[0], tlap[1], tlap[2]);
#endif
  return;   // 3. the two triangular solves run in k_rr_trsm, one right-hand side per CTA
  }
  if (*flag) return;   // Cholesky failed: the single-CTA SVQB kernel takes over
  // Hermitian average into cm (full storage)
  for (size_t e = gtid; e < mm; e += gnt) {
    const int i = (int)(e % m), j = (int)(e / m);
    const double2 a = cc[e], b = cc[(size_t)i * m + j];
    cm[e] = i == j ? double2{a.x, 0.0} : double2{0.5 * (a.x + b.x), 0.5 * (a.y - b.y)};
  }
  cl.sync();
  // 4. Householder reduction of cm to a complex tridiagonal.
  // Distributed form (when the staging area holds this CTA's share of the columns): column j
  // lives in the shared memory of CTA j % csize, as double-float (re hi, re lo, im hi, im lo).
  // Step k (reflector v of column k, rows > k):
  //   A  every CTA copies v and tau from the owner of column k (DSMEM)
  //   B  p_i = tau C[:, i]^H v for the owned columns i > k (Hermitian C: p = tau C v) and the
  //      partial sum of conj(v_i) p_i
  //   -- cluster barrier --
  //   C  K = tau/2 sum of the partials, w = p - K v (p gathered from the owners)
  //   D  owned columns j > k: C[:, j] -= v conj(w_j) + w conj(v_j)
  //   E  the owner of column k+1 forms the next reflector (FP64 from the double-float column)
  //   -- cluster barrier --
  // B-D run in double-float arithmetic on the FP32 lanes (about 2^-47 per operation): in FP64
  // they were bound by the FP64 pipe of each SM.  The reflectors stay in their columns (first
  // element replaced by v0), as in the global form.
  const int ncol_own = (m + csize - 1) / csize;
  if (m >= 3 && scols >= ncol_own) {
    float4* cb = reinterpret_cast<float4*>(stg);             // owned columns, column j at (j / csize) * m
    float4* vl = reinterpret_cast<float4*>(rrc_smem);        // v of the current step, by row
    float4* wf = vl + m;                                     // w, by row
    float4* pb = wf + m;                                     // p at the owned indices (read by the cluster)
    float4* bc = pb + m;                                     // 2 x (m + 1): reflector + tau, by parity
    float4* kp = bc + 2 * (m + 1);                           // this CTA's partial of v^H p
    float4* kw = kp + 1;                                     // per-warp partials
    __shared__ float4 hk;                                    // K of the current step
    __shared__ float2 tpart[RRC_WARPS];                      // per-warp partial norms of the next column
    for (int e = tid; e < ncol_own * m; e += RRC_THREADS) {
      const int lj = e / m, r = e - lj * m, j = lj * csize + crank;
      if (j < m) cb[e] = c4(cm[(size_t)j * m + r]);
    }
    __syncthreads();
    // reflector of column k by warp 0 of its owner: broadcast buffer, v0 into the column, tau/ph.
    // All scalars in double-float on the FP32 lanes (a chain of FP64 operations here was the
    // critical path of every step); tau[k] and ph[k] are left as double-float quadruples in
    // their double2 slots and converted after the loop.
    // tsum: the sum of |x_i|^2 over i >= 1 when the caller has it (nullptr: formed here)
    auto make_reflector = [&](int k, const dfl* tsum) {
      float4* x = cb + (size_t)(k / csize) * m + k + 1;
      const int len = m - k - 1;
      dfl t2{0.f, 0.f};
      if (tsum) {
        t2 = *tsum;
      } else {
        for (int i = 1 + lane; i < len; i += 32) {
          const cdf xi = ucdf(x[i]);
          t2 = dd_fma(xi.re, xi.re, t2);
          t2 = dd_fma(xi.im, xi.im, t2);
        }
        t2 = warp_dsum(t2);
      }
      const cdf x0 = ucdf(x[0]);
      const dfl ax02 = dd_fma(x0.im, x0.im, df_mul(x0.re, x0.re));
      const dfl a2 = df_add(t2, ax02);
      cdf beta = x0, v0 = x0;
      dfl t{0.f, 0.f};
      if (a2.h > 0.f && t2.h > 1e-30f * a2.h) {
        const dfl alpha = df_sqrt(a2);
        if (ax02.h > 0.f) {
          // beta = -alpha x0 / |x0|, v0 = x0 - beta = x0 (1 + alpha / |x0|)
          const dfl s_ = df_div(alpha, df_sqrt(ax02));
          beta = cdf{df_neg(df_mul(x0.re, s_)), df_neg(df_mul(x0.im, s_))};
        } else {
          beta = cdf{df_neg(alpha), dfl{0.f, 0.f}};
        }
        v0 = csub(x0, beta);
        const dfl nv = df_add(t2, dd_fma(v0.im, v0.im, df_mul(v0.re, v0.re)));
        t = df_div(dfl{2.f, 0.f}, nv);
        // a tail so small that its squares leave the FP32 exponent range (below ~1e-19 in norm)
        // gives no representable reflector: the column is left as it is (already reduced to
        // double-float precision unless the whole matrix is that small)
        if (!(isfinite(t.h) && isfinite(t.l) && isfinite(v0.re.h) && isfinite(v0.im.h) && isfinite(beta.re.h) &&
              isfinite(beta.im.h))) {
          t = dfl{0.f, 0.f};
          beta = x0;
          v0 = x0;
        }
      }
      float4* out = bc + (size_t)(k & 1) * (m + 1);
      const float4 v04 = c4(v0);
      for (int i = lane; i < len; i += 32) out[k + 1 + i] = i == 0 ? v04 : x[i];
      __syncwarp();
      if (lane == 0) {
        out[m] = float4{t.h, t.l, 0.f, 0.f};
        if (t.h != 0.f) x[0] = v04;
        reinterpret_cast<float4*>(tau)[k] = float4{t.h, t.l, 0.f, 0.f};
        reinterpret_cast<float4*>(ph)[k] = c4(beta);
      }
    };
    if (crank == 0 && wl == 0) make_reflector(0, nullptr);
    cl.sync();
    RR_LAP(7);
    for (int k = 0; k + 2 < m; ++k) {
      const int len = m - k - 1;
      // A
      const float4* src = cl.map_shared_rank(bc + (size_t)(k & 1) * (m + 1), (unsigned)(k % csize));
      for (int r = k + 1 + tid; r <= m; r += RRC_THREADS) vl[r == m ? 0 : r] = src[r];   // vl[0] <- tau
      __syncthreads();
      RR_LAP(0);
      const dfl t = ucdf(vl[0]).re;
      // B
      const int lj0 = (k + 1 - crank + csize - 1) / csize;   // first owned column > k
      cdf kacc = cdf0();
      for (int lj = lj0 + wl; lj < ncol_own; lj += RRC_WARPS) {
        const int i = lj * csize + crank;
        if (i >= m) break;
        const float4* ci = cb + (size_t)lj * m;
        cdf sacc = cdf0();
        for (int r = k + 1 + lane; r < m; r += 32) sacc = cdf_fmac(ucdf(ci[r]), ucdf(vl[r]), sacc);
        sacc = warp_cdsum(sacc);
        const cdf p = cdf{df_mul(t, sacc.re), df_mul(t, sacc.im)};
        if (lane == 0) pb[i] = c4(p);
        kacc = cdf_fmac(ucdf(vl[i]), p, kacc);
      }
      if (lane == 0) kw[wl] = c4(kacc);
      __syncthreads();
      if (wl == 0) {
        cdf ks = lane < RRC_WARPS ? ucdf(kw[lane]) : cdf0();
        ks = warp_cdsum(ks);
        if (lane == 0) kp[0] = c4(ks);
      }
      RR_LAP(1);
      cl.sync();
      RR_LAP(2);
      // C: p_r gathered from the owners (one row per thread, issued first so that its latency
      // overlaps the K reduction), K = tau/2 * sum of the partials, w = p - K v
      const int rr = k + 1 + tid;
      float4 p4 = float4{0.f, 0.f, 0.f, 0.f};
      if (rr < m) p4 = *cl.map_shared_rank(pb + rr, (unsigned)(rr % csize));
      if (wl == 0) {
        cdf ks = lane < csize ? ucdf(*cl.map_shared_rank(kp, (unsigned)lane)) : cdf0();
        ks = warp_cdsum(ks);
        const dfl ht = df_mul(t, dfl{0.5f, 0.f});
        if (lane == 0) hk = c4(cdf{df_mul(ht, ks.re), df_mul(ht, ks.im)});
      }
      __syncthreads();
      const cdf kv = ucdf(hk);
      if (rr < m) wf[rr] = c4(csub(ucdf(p4), cmul(kv, ucdf(vl[rr]))));
      __syncthreads();
      RR_LAP(3);
      // D: owned columns j > k: C[:, j] -= v conj(w_j) + w conj(v_j).  The owner of column k+1
      // updates that column first, one row per thread, with the partial sums of |C_r,k+1|^2 over
      // the rows below its subdiagonal; warp 0 then forms the next reflector (E) while the
      // other warps update the remaining columns.
      const int nown = ncol_own - lj0;
      auto upd = [&](int lj, int r) {
        const int j = lj * csize + crank;
        if (j >= m) return cdf0();
        const cdf vr = ucdf(vl[r]), wr = ucdf(wf[r]), vj = ucdf(vl[j]), wj = ucdf(wf[j]);
        float4* cjr = cb + (size_t)lj * m + r;
        cdf c = ucdf(*cjr);
        c.re = dd_fma(df_neg(vr.re), wj.re, c.re);
        c.re = dd_fma(df_neg(vr.im), wj.im, c.re);
        c.re = dd_fma(df_neg(wr.re), vj.re, c.re);
        c.re = dd_fma(df_neg(wr.im), vj.im, c.re);
        c.im = dd_fma(df_neg(vr.im), wj.re, c.im);
        c.im = dd_fma(vr.re, wj.im, c.im);
        c.im = dd_fma(df_neg(wr.im), vj.re, c.im);
        c.im = dd_fma(wr.re, vj.im, c.im);
        *cjr = c4(c);
        return c;
      };
      if (k + 3 < m && crank == (k + 1) % csize) {
#ifdef DKS_RR_TIMING
        const unsigned long long o0 = clock64();
#endif
        dfl part{0.f, 0.f};
        if (rr < m) {
          const cdf c = upd(lj0, rr);
          if (rr >= k + 3) part = dd_fma(c.im, c.im, df_mul(c.re, c.re));
        }
        if (32 * wl < len) {
          part = warp_dsum(part);
          if (lane == 0) tpart[wl] = float2{part.h, part.l};
        }
        __syncthreads();
        if (wl == 0) {
#ifdef DKS_RR_TIMING
          const unsigned long long o1 = clock64();
#endif
          dfl t2{0.f, 0.f};
          const int nw = (len + 31) / 32;
          if (lane < nw) t2 = dfl{tpart[lane].x, tpart[lane].y};
          t2 = warp_dsum(t2);
          make_reflector(k + 1, &t2);   // E
#ifdef DKS_RR_TIMING
          if (gtid == 0) {
            town[0] += o1 - o0;
            town[1] += clock64() - o1;
            ++town[2];
          }
#endif
        } else {
          for (int e = tid - 32; e < (nown - 1) * len; e += RRC_THREADS - 32) {
            const int q = e / len;
            upd(lj0 + 1 + q, k + 1 + (e - q * len));
          }
        }
      } else {
        for (int e = tid; e < nown * len; e += RRC_THREADS) {
          const int q = e / len;
          upd(lj0 + q, k + 1 + (e - q * len));
        }
      }
      RR_LAP(4);
      cl.sync();
      RR_LAP(6);
    }
    for (int e = tid; e < ncol_own * m; e += RRC_THREADS) {
      const int lj = e / m, r = e - lj * m, j = lj * csize + crank;
      if (j < m) {
        const cdf c = ucdf(cb[e]);
        cm[(size_t)j * m + r] = double2{df_val(c.re), df_val(c.im)};
      }
    }
    // tau and ph of the reflectors from double-float to FP64 (every owner wrote before a barrier)
    for (int k = gtid; k + 2 < m; k += gnt) {
      const cdf tk = ucdf(reinterpret_cast<const float4*>(tau)[k]);
      const cdf pk = ucdf(reinterpret_cast<const float4*>(ph)[k]);
      tau[k] = double2{df_val(tk.re), 0.0};
      ph[k] = double2{df_val(pk.re), df_val(pk.im)};
    }
    cl.sync();
  } else {
  // 4. Householder reduction of cm.  Warp 0 of every CTA forms the reflector (norm, phase, tau)
  // and the scalar K and hands them to its CTA through shared memory.
  __shared__ double2 hh[4];   // {tau, 0}, beta, v0, K
  for (int k = 0; k + 2 < m; ++k) {
    const int len = m - k - 1;
    double2* x = cm + (size_t)k * m + k + 1;
    if (wl == 0) {
      double a2 = 0;
      for (int i = lane; i < len; i += 32) a2 += x[i].x * x[i].x + x[i].y * x[i].y;
      a2 = warp_sum(a2);
      const double2 x0 = x[0];
      const double ax0 = nr_hypot(x0.x, x0.y);
      const double alpha = nr_sqrt(a2);
      double t = 0.0;
      double2 beta = x0, v0 = x0;
      if (alpha > 1e-300 && a2 - ax0 * ax0 > 1e-30 * a2) {
        const double ri = ax0 > 0 ? nr_rcp(ax0) : 0.0;
        const double2 phs = ax0 > 0 ? double2{x0.x * ri, x0.y * ri} : double2{1, 0};
        beta = double2{-phs.x * alpha, -phs.y * alpha};
        v0 = double2{x0.x - beta.x, x0.y - beta.y};
        t = 2.0 * nr_rcp(a2 - ax0 * ax0 + v0.x * v0.x + v0.y * v0.y);
      }
      if (lane == 0) {
        hh[0] = double2{t, 0.0};
        hh[1] = beta;
        hh[2] = v0;
      }
    }
    __syncthreads();
    const double t = hh[0].x;
    const double2 beta = hh[1], v0 = hh[2];
    if (t != 0.0) {
      double2* a22 = cm + (size_t)(k + 1) * m + (k + 1);
      // p_i = t sum_j A22[i, j] v_j = t sum_j conj(A22[j, i]) v_j (read column i)
      for (int i = gw; i < len; i += gnw) {
        double2 sacc{0, 0};
        for (int j = lane; j < len; j += 32) {
          const double2 vj = j == 0 ? v0 : x[j];
          sacc = cadd(sacc, cmulc(a22[(size_t)i * m + j], vj));
        }
        sacc = warp_csum(sacc);
        if (lane == 0) pv[i] = double2{t * sacc.x, t * sacc.y};
      }
    }
    cl.sync();
    if (t != 0.0) {
      double2* a22 = cm + (size_t)(k + 1) * m + (k + 1);
      if (wl == 0) {
        double2 kv{0, 0};
        for (int i = lane; i < len; i += 32) kv = cadd(kv, cmulc(i == 0 ? v0 : x[i], pv[i]));
        kv = warp_csum(kv);
        if (lane == 0) hh[3] = double2{0.5 * t * kv.x, 0.5 * t * kv.y};
      }
      __syncthreads();
      const double2 kv = hh[3];
      for (int e = gtid; e < len * len; e += gnt) {
        const int i = e % len, j = e / len;
        const double2 vi = i == 0 ? v0 : x[i], vj = j == 0 ? v0 : x[j];
        const double2 wi = csub(pv[i], cmul(kv, vi)), wj = csub(pv[j], cmul(kv, vj));
        const double2 u1 = cmul(vi, double2{wj.x, -wj.y});
        const double2 u2 = cmul(wi, double2{vj.x, -vj.y});
        a22[(size_t)j * m + i] = csub(a22[(size_t)j * m + i], cadd(u1, u2));
      }
    }
    if (gtid == 0) {
      tau[k] = double2{t, 0};
      ph[k] = beta;
    }
    cl.sync();
    if (gtid == 0 && t != 0.0) x[0] = v0;    // reflector stored after every warp has read x[0]
    // (no barrier needed: x[0] of column k is not read again until the back-transformation)
  }
  cl.sync();
  }
  RR_MARK(3);
  // 5. real tridiagonal (every CTA keeps its own copy in shared memory for the multisection).
  // CTA 0: d_k = Re C_kk, e_k = |beta_k| and the unit factors u_k = beta_k / e_k in parallel,
  // then the phases ph_k = u_0 ... u_(k-1) (which make the subdiagonal real) as a prefix
  // product by warp 0: a serial chunk per lane and a shuffle scan over the lanes.
  if (crank == 0) {
    double2* su = reinterpret_cast<double2*>(rrc_smem);   // m factors (the per-warp vectors are free here)
    for (int k = tid; k < m; k += RRC_THREADS) {
      dd[k] = cm[(size_t)k * m + k].x;
      if (k + 1 < m) {
        const double2 e = k == m - 2 ? cm[(size_t)(m - 2) * m + (m - 1)] : ph[k];
        const double ae = nr_hypot(e.x, e.y);
        ee[k] = ae;
        e2[k] = ae * ae;
        double2 u{1.0, 0.0};
        if (ae > 0) {
          const double ri = nr_rcp(ae);
          u = double2{e.x * ri, e.y * ri};
        }
        su[k] = u;
      } else {
        ee[k] = 0;
        e2[k] = 0;
      }
    }
    if (tid == 0 && m >= 2) tau[m - 2] = double2{0, 0};
    __syncthreads();
    if (wl == 0) {
      const int nf = m - 1;                        // factors u_0 .. u_(m-2)
      const int c = (nf + 31) / 32;
      const int b0 = min(nf, lane * c), b1 = min(nf, b0 + c);
      double2 pr{1.0, 0.0};
      for (int j = b0; j < b1; ++j) pr = cmul(pr, su[j]);
      double2 inc = pr;                            // inclusive scan of the chunk products
      for (int o = 1; o < 32; o <<= 1) {
        const double2 y{__shfl_up_sync(0xffffffffu, inc.x, o), __shfl_up_sync(0xffffffffu, inc.y, o)};
        if (lane >= o) inc = cmul(y, inc);
      }
      double2 ex{__shfl_up_sync(0xffffffffu, inc.x, 1), __shfl_up_sync(0xffffffffu, inc.y, 1)};
      if (lane == 0) ex = double2{1.0, 0.0};
      for (int j = b0; j < b1; ++j) {
        ph[j] = ex;
        ex = cmul(ex, su[j]);
      }
      if (b0 < b1 && b1 == nf) ph[nf] = ex;        // the product of all factors
      if (nf == 0 && lane == 0) ph[0] = double2{1.0, 0.0};
    }
  }
  cl.sync();
  // copy the tridiagonal into this CTA's shared memory (behind the per-warp vectors)
  double* sd = reinterpret_cast<double*>(rrc_smem + rr_tri_smem_offset(m));
  dfl* ge = reinterpret_cast<dfl*>(sd + m);   // |e| as double-float (inverse iteration)
  double* se2 = sd + 2 * m;
  float* fd = reinterpret_cast<float*>(se2 + m);
  float* fe2 = fd + m;
  dfl* gd = reinterpret_cast<dfl*>(fe2 + m);
  dfl* ge2 = gd + m;
  for (int k = tid; k < m; k += RRC_THREADS) {
    sd[k] = dd[k];
    ge[k] = df_from(ee[k]);
    se2[k] = e2[k];
    fd[k] = (float)dd[k];
    fe2[k] = (float)e2[k];
    gd[k] = df_from(dd[k]);
    ge2[k] = df_from(e2[k]);
  }
  // Gershgorin interval and the largest e^2, by warp 0
  __shared__ double gersh[3];
  if (wl == 0) {
    double lo_ = INFINITY, hi_ = -INFINITY, me = 0.0;
    for (int k = lane; k < m; k += 32) {
      const double r = (k > 0 ? ee[k - 1] : 0.0) + (k + 1 < m ? ee[k] : 0.0);
      lo_ = fmin(lo_, dd[k] - r);
      hi_ = fmax(hi_, dd[k] + r);
      me = fmax(me, e2[k]);
    }
    for (int o = 16; o; o >>= 1) {
      lo_ = fmin(lo_, __shfl_xor_sync(0xffffffffu, lo_, o));
      hi_ = fmax(hi_, __shfl_xor_sync(0xffffffffu, hi_, o));
      me = fmax(me, __shfl_xor_sync(0xffffffffu, me, o));
    }
    if (lane == 0) {
      gersh[0] = lo_;
      gersh[1] = hi_;
      gersh[2] = me;
    }
  }
  __syncthreads();
  const double lo0 = gersh[0], hi0 = gersh[1];
  const double tnorm = fmax(fabs(lo0), fabs(hi0));
  // pivot guard of the FP32 and double-float counts: e^2 / q stays below the FP32 overflow level
  const float fpiv = 1.2e-38f * fmaxf(1.0f, (float)fmin(gersh[2], 1e30));
  // 5. eigenvalue idx by one warp (eigenvalues spread round-robin over the CTAs): 33-way
  // multisection of the Sturm count, lane l counting at lo + (l+1)(hi-lo)/33, the bracket then
  // narrowed to the first section whose count exceeds idx.  FP32 counts take the bracket to
  // ~2e-7 relative (or 1e-7 of the matrix norm); it is widened by the FP32 error level and
  // refined with double-float counts (~2^-47 per operation) to ~3e-14 relative or 1e-14 of the
  // matrix norm, whichever is larger.
  for (int r0 = 0; r0 < n; r0 += gnw) {
    const int idx = r0 + wl * csize + crank;
    if (idx >= n) continue;
    double lo = lo0 - 1e-14 * tnorm - 1e-300, hi = hi0 + 1e-14 * tnorm + 1e-300;
    float flo = (float)lo, fhi = (float)hi;
    const float fabs_tol = (float)(1e-7 * tnorm);
    for (int it = 0; it < 10; ++it) {
      if (!(fhi - flo > fmaxf(2e-7f * fmaxf(fabsf(flo), fabsf(fhi)), fabs_tol))) break;
      const float step = (fhi - flo) * (1.0f / 33.0f);
      const float x = flo + step * (float)(lane + 1);
      const unsigned bal = __ballot_sync(0xffffffffu, sturm_count_f(fd, fe2, m, x, fpiv) > idx);
      const int l = bal ? __ffs(bal) - 1 : 32;
      const float nlo = l == 0 ? flo : flo + step * (float)l;
      const float nhi = l == 32 ? fhi : flo + step * (float)(l + 1);
      flo = nlo;
      fhi = nhi;
    }
    const double pad = 4e-6 * tnorm + 1e-300;
    lo = fmax(lo, (double)flo - pad);
    hi = fmin(hi, (double)fhi + pad);
    for (int it = 0; it < 12; ++it) {
      if (!(hi - lo > fmax(3e-14 * fmax(fabs(lo), fabs(hi)), 1e-14 * tnorm) + 1e-300)) break;
      const double step = (hi - lo) * (1.0 / 33.0);
      const double x = lo + step * (double)(lane + 1);
      const unsigned bal = __ballot_sync(0xffffffffu, sturm_count_df(gd, ge2, m, df_from(x), fpiv) > idx);
      const int l = bal ? __ffs(bal) - 1 : 32;
      const double nlo = l == 0 ? lo : lo + step * (double)l;
      const double nhi = l == 32 ? hi : lo + step * (double)(l + 1);
      lo = nlo;
      hi = nhi;
    }
    if (lane == 0) lamw[idx] = 0.5 * (lo + hi);
  }
  cl.sync();
  RR_MARK(4);
  // 6. inverse iteration; clusters of close eigenvalues go to one lane in order.  Warps that own
  // a shared-memory slot (nslots per CTA) take the cluster starts round-robin over the CTAs first
  // (a lone FP64 lane still occupies its SM's FP64 pipe for a whole warp instruction, so chains
  // sharing an SM slow each other down).
  const double ortol = 1e-7 * fmax(tnorm, 1e-300);
  const int nslots = min(RRC_WARPS, (int)(rr_tri_smem_offset(m) / (sizeof(double) * 6 * (size_t)m)));
  dfl* fws = reinterpret_cast<dfl*>(rrc_smem);   // per-slot 5m factors + m vector
  // the eigenvectors of T are written as double-float pairs into the double slots of zt
  float2* zt2 = reinterpret_cast<float2*>(zt);
  if (wl < nslots && lane == 0) {
    const int gslot = wl * csize + crank, nslot_all = csize * nslots;
    const float tiny = fmaxf((float)(DBL_EPSILON * tnorm), 1e-30f);
    for (int start = gslot; start < n; start += nslot_all) {
      const bool begins = start == 0 || lamw[start] - lamw[start - 1] > ortol;
      if (!begins) continue;
      int end = start + 1;
      while (end < n && lamw[end] - lamw[end - 1] <= ortol) ++end;
      dfl* f = fws + (size_t)wl * 6 * m;
      dfl* xv = f + 5 * m;
      for (int v = start; v < end; ++v) {
        const double shift = lamw[v] + (double)(v - start) * 10.0 * DBL_EPSILON * tnorm;
        tri_factor_df(gd, ge, m, df_from(shift), tiny, f);
        for (int i = 0; i < m; ++i) xv[i] = dfl{start_val(i, v), 0.f};
        for (int itr = 0; itr < 3; ++itr) {
          tri_solve_df(m, f, xv);
          for (int u = start; u < v; ++u) {        // orthogonalise against the cluster's earlier vectors
            const float2* zu = zt2 + (size_t)u * m;
            dfl dot{0.f, 0.f};
            for (int i = 0; i < m; ++i) dot = dd_fma(dfl{zu[i].x, zu[i].y}, xv[i], dot);
            const dfl nd = df_neg(dot);
            for (int i = 0; i < m; ++i) xv[i] = dd_fma(nd, dfl{zu[i].x, zu[i].y}, xv[i]);
          }
          df_normalize(m, xv);
        }
        for (int i = 0; i < m; ++i) zt2[(size_t)v * m + i] = float2{xv[i].h, xv[i].l};
      }
    }
  }
  cl.sync();
  RR_MARK(5);
#ifdef DKS_RR_TIMING
  if (gtid == 0)
    printf("rr_cluster m=%d n=%d: householder %.1f multisect %.1f invit %.1f us (cycles: A %llu B %llu sync1 %llu C %llu D %llu E %llu sync2 %llu)\n", m, n,
           (tmark[3] - tmark[0]) * 1e-3, (tmark[4] - tmark[3]) * 1e-3, (tmark[5] - tmark[4]) * 1e-3,
           tlap[0], tlap[1], tlap[2], tlap[3], tlap[4], tlap[5], tlap[6]);
  if (gtid == 0)
    printf("  owner steps of CTA 0: %llu, column update %llu cycles, reflector %llu cycles\n", town[2], town[0], town[1]);
#endif
}

// Bulk global -> shared copies for the per-column kernels (TMA, completion on an mbarrier).
// Sources and destinations are 16-byte aligned and sizes multiples of 16 bytes (double2 arrays).
__device__ __forceinline__ uint32_t sh_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// thread 0: expect `bytes` on the mbarrier and issue the copy in pieces of at most 48 KB
__device__ __forceinline__ void stage_issue(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sh_u32(mbar)), "r"(bytes) : "memory");
  for (uint32_t off = 0; off < bytes; off += 48u * 1024u) {
    const uint32_t len = min(bytes - off, 48u * 1024u);
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            sh_u32(static_cast<char*>(dst) + off)),
        "l"(static_cast<const char*>(src) + off), "r"(len), "r"(sh_u32(mbar))
        : "memory");
  }
}

// polls allowed to the first wait for each staging copy (the wait whose give-up hands the step
// to the single-CTA kernel).  1 << 24 in normal use; the failure-detection test hook sets it to
// 0, so that every such wait gives up at once while the copy itself still lands (the second,
// draining wait keeps the full limit)
__device__ unsigned int g_rr_first_wait = 1u << 24;

// every thread: bounded wait for the phase of the mbarrier
__device__ __forceinline__ bool stage_wait(uint64_t* mbar, uint32_t parity, uint32_t limit = 1u << 24) {
  uint32_t done = 0;
  for (uint32_t it = 0; it < limit && !done; ++it)
    asm volatile(
        "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\tselp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(done)
        : "r"(sh_u32(mbar)), "r"(parity)
        : "memory");
  return done != 0;
}

// stage `bytes` from src into dst (whole block); false (uniform over the block) on a timeout,
// after a second bounded wait for the copy still in flight
__device__ bool stage_block(void* dst, const void* src, uint32_t bytes, uint64_t* mbar, uint32_t& phase) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // earlier generic reads of dst
  __syncthreads();
  if (threadIdx.x == 0) stage_issue(dst, src, bytes, mbar);
  const bool ok = __syncthreads_and(stage_wait(mbar, phase & 1, g_rr_first_wait) ? 1 : 0) != 0;
  if (!ok) stage_wait(mbar, phase & 1);   // the copy in flight lands before the block goes on
  ++phase;
  return ok;
}

__device__ __forceinline__ void stage_init(uint64_t* mbar) {
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sh_u32(mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
}

// 3. Forward substitution with L, column-oriented, one right-hand side per CTA (so each column
// has an SM's FP64 pipes to itself): the 128 threads own rows k of b (one warp on each of the
// SM's four FP64 units); at step i every thread forms w_i = b_i / L_ii and updates its
// b_k -= L_ki w_i (k > i); columns of L are staged in shared memory in blocks.
//   pass 0: W = L^-1 A'   (column c of A')              -> cm
//   pass 1: C = L^-1 W^H  (column c = conj(row c of W))  -> lm (free after the Cholesky)
__global__ void __launch_bounds__(128, 1) k_rr_trsm(double2* __restrict__ scr, int m, int pass, int scols) {
  extern __shared__ __align__(16) unsigned char trs_smem[];
  const size_t mm = (size_t)m * m;
  double2* am = scr;
  double2* lm = am + mm;
  double2* lf = lm + mm;
  double2* lt = lf + mm;
  double2* cm = lt + mm;
  double* lamw = reinterpret_cast<double*>(cm + mm) + 4 * m;
  const double* linv = lamw + m;
  int* flag = reinterpret_cast<int*>(reinterpret_cast<double2*>(lamw + 2 * m) + 3 * m);
  if (*flag) return;
  (void)lt;
  __shared__ __align__(8) uint64_t mbar;
  uint32_t phase = 0;
  stage_init(&mbar);
  double2* stg = reinterpret_cast<double2*>(trs_smem);           // scols x m
  double2* b = stg + (size_t)scols * m;                          // right-hand side / solution
  double* sl = reinterpret_cast<double*>(b + m);
  const int tid = threadIdx.x;
  const int c = blockIdx.x;
  for (int k = tid; k < m; k += blockDim.x) {
    sl[k] = linv[k];
    if (pass == 0) {
      b[k] = am[(size_t)c * m + k];
    } else {
      const double2 w = cm[(size_t)k * m + c];
      b[k] = double2{w.x, -w.y};
    }
  }
  for (int i0 = 0; i0 < m; i0 += scols) {
    const int nb = min(scols, m - i0);
    if (!stage_block(stg, lf + (size_t)i0 * m, (uint32_t)(nb * m * sizeof(double2)), &mbar, phase)) {
      if (tid == 0) *flag = 2;   // the single-CTA kernel recomputes the whole step
      return;
    }
    for (int i = i0; i < i0 + nb; ++i) {
      const double2 bi = b[i];
      const double li = sl[i];
      const double2 w = double2{bi.x * li, bi.y * li};
      const double2* lc = stg + (size_t)(i - i0) * m;
      for (int k = tid; k < m; k += blockDim.x)
        if (k > i) b[k] = csub(b[k], cmul(lc[k], w));
      __syncthreads();
    }
  }
  double2* out = pass == 0 ? cm : lm;
  for (int k = tid; k < m; k += blockDim.x) out[(size_t)c * m + k] = double2{b[k].x * sl[k], b[k].y * sl[k]};
}

// 7. u = H_0 ... H_{m-3} (Phi z_j); V_j = D L^-H u, one eigenvector per CTA; the 128 threads own
// rows (one warp per FP64 unit of the SM); reflectors and rows of L are staged in shared
// memory.  A reflector step sums four warp partials through shared memory (double-buffered by
// step parity, so one barrier per step).
__global__ void __launch_bounds__(128, 1) k_rr_backtr(double2* __restrict__ scr, int m, int n, double2* __restrict__ V,
                                                   double* __restrict__ lam, int* __restrict__ info, int scols) {
  extern __shared__ __align__(16) unsigned char btr_smem[];
  const size_t mm = (size_t)m * m;
  double2* am = scr;
  double2* lm = am + mm;
  double2* lf = lm + mm;
  double2* lt = lf + mm;
  double2* cm = lt + mm;
  double* dsc = reinterpret_cast<double*>(cm + mm);
  double* lamw = dsc + 4 * m;
  const double* linv = lamw + m;
  const double2* tau = reinterpret_cast<const double2*>(lamw + 2 * m);
  const double2* ph = tau + m;
  int* flag = reinterpret_cast<int*>(const_cast<double2*>(ph) + 2 * m);
  const double* zt = reinterpret_cast<const double*>(lm);
  if (*flag) return;
  (void)lf;
  __shared__ __align__(8) uint64_t mbar;
  uint32_t phase = 0;
  stage_init(&mbar);
  double2* stg = reinterpret_cast<double2*>(btr_smem);           // scols x m
  double2* wv = stg + (size_t)scols * m;
  double2* sph = wv + m;
  double* sl = reinterpret_cast<double*>(sph + m);
  double* stau = sl + m;
  double* sdsc = stau + m;
  __shared__ float4 red[8];    // warp partials of the reflector dot products, by step parity
  const int tid = threadIdx.x, lane = tid & 31, wl = tid >> 5;
  const int j = blockIdx.x;
  for (int k = tid; k < m; k += blockDim.x) {
    sl[k] = linv[k];
    stau[k] = tau[k].x;
    sdsc[k] = dsc[k];
  }
  // the reflectors are applied in double-float arithmetic (an orthogonal transformation, so
  // 2^-47 rounding per operation stays at that level; FP64 chains cost a whole FP64-unit
  // warp instruction per dependent step): reflector elements are split as they are read, the
  // vector is kept as double-float in the rows each thread owns
  constexpr int RPT = 4;                       // rows per thread: m <= 512
  // start vector: ph_r z_r, z the double-float eigenvector of the real tridiagonal
  const float2* zj = reinterpret_cast<const float2*>(zt) + (size_t)j * m;
  cdf wq[RPT];
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int r = tid + 128 * q;
    if (r < m) {
      const dfl z{zj[r].x, zj[r].y};
      const double2 p = ph[r];
      wq[q] = cdf{df_mul(df_from_bits(p.x), z), df_mul(df_from_bits(p.y), z)};
    } else {
      wq[q] = cdf0();
    }
  }
  for (int k1 = m - 3; k1 >= 0; k1 -= scols) {
    const int k0 = max(0, k1 - scols + 1);
    if (!stage_block(stg, cm + (size_t)k0 * m, (uint32_t)((k1 - k0 + 1) * m * sizeof(double2)), &mbar, phase)) {
      if (tid == 0) *flag = 2;
      return;
    }
    for (int k = k1; k >= k0; --k) {
      const double t = stau[k];
      if (t == 0.0) continue;   // uniform: every thread reads the same tau
      const double2* v = stg + (size_t)(k - k0) * m;
      // rows r > k, thread-owned (r = tid + 128 q): partial dot, warp sums, four partials
      cdf sacc = cdf0();
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        const int r = tid + 128 * q;
        if (r > k && r < m) sacc = cdf_fmac(cdf{df_from_bits(v[r].x), df_from_bits(v[r].y)}, wq[q], sacc);
      }
      sacc = warp_cdsum(sacc);
      float4* part = red + 4 * (k & 1);
      if (lane == 0) part[wl] = c4(sacc);
      __syncthreads();
      cdf tot = ucdf(part[0]);
      tot = cadd(tot, ucdf(part[1]));
      tot = cadd(tot, ucdf(part[2]));
      tot = cadd(tot, ucdf(part[3]));
      const dfl td = df_from(t);
      const cdf f = cdf{df_mul(td, tot.re), df_mul(td, tot.im)};
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        const int r = tid + 128 * q;
        if (r > k && r < m) wq[q] = csub(wq[q], cmul(f, cdf{df_from_bits(v[r].x), df_from_bits(v[r].y)}));
      }
    }
  }
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int r = tid + 128 * q;
    if (r < m) wv[r] = double2{df_val(wq[q].re), df_val(wq[q].im)};
  }
  // L^H y = u, column-oriented: y_i = u_i / L_ii, then u_k -= conj(L[i, k]) y_i for k < i
  for (int i1 = m - 1; i1 >= 0; i1 -= scols) {
    const int i0 = max(0, i1 - scols + 1);
    if (!stage_block(stg, lt + (size_t)i0 * m, (uint32_t)((i1 - i0 + 1) * m * sizeof(double2)), &mbar, phase)) {
      if (tid == 0) *flag = 2;
      return;
    }
    __syncthreads();
    for (int i = i1; i >= i0; --i) {
      const double2 u = wv[i];
      const double li = sl[i];
      const double2 y = double2{u.x * li, u.y * li};
      const double2* lr = stg + (size_t)(i - i0) * m;
      for (int k = tid; k < i; k += blockDim.x) wv[k] = csub(wv[k], cmulc(lr[k], y));
      __syncthreads();
    }
  }
  for (int i = tid; i < m; i += blockDim.x) {
    const double f = sdsc[i] * sl[i];
    V[(size_t)j * m + i] = double2{f * wv[i].x, f * wv[i].y};
  }
  if (tid == 0) {
    lam[j] = lamw[j];
    if (j == 0) {
      info[0] = 0;
      info[1] = m;
      info[2] = 0;
    }
  }
}

int rr_set_first_wait(unsigned polls) {
  DKS_CUDA_TRY(cudaMemcpyToSymbol(g_rr_first_wait, &polls, sizeof(polls)));
  return DKS_OK;
}

// byte offset of the hand-off flag inside the scratch layout above
size_t rr_cluster_flag_offset(int m) {
  const size_t mm = (size_t)m * m;
  return 5 * mm * sizeof(double2) + 6 * (size_t)m * sizeof(double) + 3 * (size_t)m * sizeof(double2);
}

static int g_cluster = 0;   // 0 = unknown, else cluster size that launched successfully

static cudaError_t launch_cluster(int csz, size_t smem, cudaStream_t st, const double2* a, const double2* s, int nz,
                                  int n, double2* v, double* lam, int* info, double2* scratch, double chol_tol,
                                  int scols, int phase) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(csz, 1, 1);
  cfg.blockDim = dim3(RRC_THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = csz;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_rr_cluster, a, s, nz, n, v, lam, info, scratch, chol_tol, scols, phase);
}

// Five launches: scaling + Cholesky (cluster), W = L^-1 A' and C = L^-1 W^H (one right-hand side
// per CTA), Householder + multisection + inverse iteration (cluster), back-transformation (one
// eigenvector per CTA).  Each later launch returns at once when the Cholesky factorisation failed.
int rayleigh_ritz_cluster(const double2* a, const double2* s, int nz, int n, double2* v, double* lam, int* info,
                          double2* scratch, cudaStream_t st, double chol_tol, bool* launched) {
  *launched = false;
  // staging columns: as many as fit (at most 64); too few and the single-CTA kernel takes over
  const size_t base = rr_cluster_smem(nz, 0);
  if (base + 8 * (size_t)nz * sizeof(double2) > kRrSmemMax) return DKS_OK;
  const int scols = (int)std::min<size_t>({(size_t)64, (size_t)nz, (kRrSmemMax - base) / ((size_t)nz * sizeof(double2))});
  const size_t smem = rr_cluster_smem(nz, scols);
  // per-column kernels: staging area + one complex vector + four m-length scalar arrays
  const size_t col_extra = (size_t)nz * (2 * sizeof(double2) + 4 * sizeof(double));
  const int scols1 = (int)std::max<size_t>(1, std::min<size_t>((size_t)nz, (kRrSmemMax - col_extra) / ((size_t)nz * sizeof(double2))));
  const size_t smem1 = (size_t)scols1 * nz * sizeof(double2) + col_extra;
  static bool attr_done = false;
  if (!attr_done) {
    cudaFuncSetAttribute((const void*)k_rr_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute((const void*)k_rr_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRrSmemMax);
    cudaFuncSetAttribute((const void*)k_rr_trsm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRrSmemMax);
    cudaFuncSetAttribute((const void*)k_rr_backtr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRrSmemMax);
    attr_done = true;
  }
  Prof pr(P_RR, st, 2.0 * nz * nz * 16.0 + 16.0 * nz * n, rr_flops(nz, n));
  const int tries[2] = {16, 8};
  for (int t = 0; t < 2; ++t) {
    const int csz = g_cluster ? g_cluster : tries[t];
    const cudaError_t e = launch_cluster(csz, smem, st, a, s, nz, n, v, lam, info, scratch, chol_tol, scols, 0);
    if (e == cudaSuccess) {
      g_cluster = csz;
      *launched = true;
      break;
    }
    cudaGetLastError();   // clear the launch error and try the portable size
    if (g_cluster) break;
  }
  if (!*launched) {
    pr.count(-1);   // nothing ran in this scope
    return DKS_OK;
  }
  pr.count(4);      // five kernels in all
  k_rr_trsm<<<nz, 128, smem1, st>>>(scratch, nz, 0, scols1);
  k_rr_trsm<<<nz, 128, smem1, st>>>(scratch, nz, 1, scols1);
  DKS_CUDA_TRY(launch_cluster(g_cluster, smem, st, a, s, nz, n, v, lam, info, scratch, chol_tol, scols, 1));
  k_rr_backtr<<<n, 128, smem1, st>>>(scratch, nz, n, v, lam, info, scols1);
  DKS_CUDA_TRY(cudaGetLastError());
  return DKS_OK;
}

}  // namespace dks

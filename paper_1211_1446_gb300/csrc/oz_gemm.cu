// FP64-accurate complex contractions of the refinement phase of Algorithm 1 on the tcgen05
// tensor cores, through exact integer slices (a splitting of the Ozaki type): the Gram matrices
// A = Z^H HZ, S = Z^H Z and the rotations OUT = Z W of complex128 blocks.
//
// Representation.  A block Z (rows x ncol complex128, column-major) is cut into windows of 128
// rows.  For window w and column c an exponent E = E(w, c) is chosen with |Re z|, |Im z| <
// 2^(E-1) over the window; every real value v is rounded to the integer F = round(v 2^(56-E))
// (|F| <= 2^55, rounding error at most 2^-57 2^E) and F is written as seven balanced base-256
// digits F = sum_s d_s 256^(6-s), -128 <= d_s <= 127 (s >= 1), |d_0| <= 128.  Thus
// v = 2^(E-8) sum_s d_s 2^(-8s) up to that rounding, and slice s of v is the BF16 number
// d_s 2^(-8s) (at most 8 significant bits: exact).  The slices are stored once per block, in
// the tensor cores' 8 x 8 core-matrix layout, [slice][re, im][column group][row group][8 x 8].
//
// Exact accumulation.  A product of slices s and t is an integer of magnitude at most 2^14 in
// units of 2^(-8(s+t)).  The 28 pairs with s + t <= 6 are kept.  Levels 0, 1, 2 and 3 (1, 2, 3
// and 4 pairs) accumulate in separate FP32 accumulators in tensor memory over at most 256 real
// terms (a window of 128 rows of a Gram matrix, or at most 128 columns of a rotation, real and
// imaginary parts): every partial sum is an integer multiple of its level's unit of magnitude at
// most 4 x 2^14 x 256 = 2^24 units, hence exact in FP32 whatever order or alignment the tensor
// core uses.  Levels 4 to 6 share a fifth accumulator; its FP32 rounding, even if every step
// truncated, stays near 2^-45 of the window's leading level, and at random about 2^-49.  The
// levels left out (s + t >= 7) and the rounding of F lie near 2^-53 max|a| max|b| per product.
// The window sums are combined in double-float registers and the chunk partials in FP64 in a
// fixed order: the result is deterministic and about as accurate as a double-float evaluation.
//
// Complex arithmetic is real arithmetic on the planar (re, im) slices: D_re = a_re b_re +
// a_im b_im and D_im = a_re b_im - a_im b_re for A^H B (the minus through the instruction's
// negate-B bit), D_re = a_re w_re - a_im w_im and D_im = a_re w_im + a_im w_re for A W.
//
// Every mbarrier wait is bounded: a wait that gives up records DKS_ERR_TIMEOUT in a device status
// word, the CTA drains its own copies and MMAs in flight (bounded again), frees its TMEM and
// returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <mutex>
#include <vector>

#include "dks_internal.h"
#include "tc_ptx.cuh"

namespace dks {
namespace tc {
int encoder(PFN_cuTensorMapEncodeTiled_v12000* out);
int device_ok();
}  // namespace tc

namespace oz {
using namespace dks::tc;

constexpr int kS = 7;            // slices per real value
constexpr int kWin = 128;        // rows of an exponent window (= rows of a rotation tile)
constexpr int kPairs = 28;       // slice pairs (s, t) with s + t <= 6
constexpr int kRegs = 5;         // accumulators: levels 0, 1, 2, 3 and 4..6
constexpr uint32_t kCore = 128;  // bytes of one 8 x 8 BF16 core matrix

__device__ int g_oz_status = 0;  // DKS_ERR_TIMEOUT after a wait gave up

// slice pairs level by level; the first pair of each of the five accumulators (levels 0, 1, 2,
// 3, and 4..6) initialises it: pairs 0, 1, 3, 6 and 10
__host__ __device__ constexpr int pair_s(int p) {
  constexpr int s[kPairs] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3, 0, 1, 2, 3, 4, 0, 1, 2, 3, 4, 5, 0, 1, 2, 3, 4, 5, 6};
  return s[p];
}
__host__ __device__ constexpr int pair_t(int p) {
  constexpr int t[kPairs] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0, 4, 3, 2, 1, 0, 5, 4, 3, 2, 1, 0, 6, 5, 4, 3, 2, 1, 0};
  return t[p];
}
__host__ __device__ constexpr int pair_reg(int p) { return pair_s(p) + pair_t(p) < 4 ? pair_s(p) + pair_t(p) : 4; }
__host__ __device__ constexpr bool pair_first(int p) { return p == 0 || p == 1 || p == 3 || p == 6 || p == 10; }

// ---------------------------------------------------------------- integer digit extraction
// F = round(|v| 2^(56 - E)) with the sign of v, from the bits of v (E: the window exponent;
// |v| < 2^(E-1) so the right shift of the 53-bit significand is 1019 + E - e >= -2, a left
// shift of at most 2).  Zero and subnormal v give 0.
__device__ __forceinline__ long long fixed56(unsigned long long bits, int E) {
  const int e = (int)((bits >> 52) & 0x7FF);
  if (!e) return 0;
  const int sh = 1019 + E - e;
  if (sh >= 55) return 0;
  const unsigned long long m53 = (bits & ((1ull << 52) - 1)) | (1ull << 52);
  const long long f = sh <= 0 ? (long long)(m53 << (-sh)) : (long long)((m53 + (1ull << (sh - 1))) >> sh);
  return (bits >> 63) ? -f : f;
}
// seven balanced base-256 digits of F (F = sum_s d_s 256^(6-s), -128 <= d_s <= 127 for s >= 1), as
// the BF16 bit patterns of d_s 2^(-8s).  Adding 128 to each of the six low bytes makes them plain
// bytes of G = F + 0x808080808080: d_s = byte - 128 for s >= 1 and d_0 = G >> 48 (the unique
// balanced representation, without a carry chain).
__device__ __forceinline__ void digits7(long long f, uint16_t (&out)[kS]) {
  const long long g = f + 0x0000808080808080LL;
  const uint32_t lo = (uint32_t)g, hi = (uint32_t)((unsigned long long)g >> 32);
  int d[kS];
  d[0] = (int)(g >> 48);
  d[1] = (int)((hi >> 8) & 255u) - 128;
  d[2] = (int)(hi & 255u) - 128;
  d[3] = (int)(lo >> 24) - 128;
  d[4] = (int)((lo >> 16) & 255u) - 128;
  d[5] = (int)((lo >> 8) & 255u) - 128;
  d[6] = (int)(lo & 255u) - 128;
#pragma unroll
  for (int s = 0; s < kS; ++s) {
    const float x = (float)d[s] * __int_as_float((127 - 8 * s) << 23);   // d_s 2^(-8s), exact
    out[s] = (uint16_t)(__float_as_uint(x) >> 16);                       // exact in BF16
  }
}
// A NaN or an infinity of a sliced block becomes seven BF16 NaN digits, so that every
// tensor-core product that uses it is NaN (as in IEEE arithmetic) and a non-finite block still
// fails the solver's finiteness checks.  (W of a rotation is sliced without that check: in the
// solver it comes from the Rayleigh-Ritz step, whose non-finite results show in its eigenvalues.)
__device__ __forceinline__ bool non_finite(unsigned long long bits) { return ((bits >> 52) & 0x7FF) == 0x7FF; }

// biased exponent field of the larger of |re|, |im| (0 for zero and subnormal values)
__device__ __forceinline__ int exp_field(double x) {
  return (int)((__double_as_longlong(x) >> 52) & 0x7FF);
}

// ---------------------------------------------------------------- split
// One CTA per (window of 128 rows, group of 8 columns): column maxima, window exponents, slices.
// Thread t handles column 8 g + (t & 7), rows 8 (t >> 4) + 4 ((t >> 3) & 1) .. + 3 of the window.
__global__ void __launch_bounds__(256) k_oz_split(const double2* __restrict__ z, long long ld, int rows, int ncol,
                                                  int rowsp, int ncolp, uint16_t* __restrict__ sl,
                                                  int* __restrict__ ex) {
  __shared__ int cmax[8];
  const int w = blockIdx.x, g = blockIdx.y, t = threadIdx.x;
  const int c8 = t & 7, half = (t >> 3) & 1, rg = t >> 4;
  const int c = g * 8 + c8;
  const int r0 = w * kWin + rg * 8 + half * 4;
  if (t < 8) cmax[t] = 0;
  __syncthreads();
  unsigned long long bits[8];
  int em = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = r0 + i;
    double2 v = double2{0.0, 0.0};
    if (c < ncol && r < rows) v = z[(size_t)c * ld + r];
    bits[2 * i] = (unsigned long long)__double_as_longlong(v.x);
    bits[2 * i + 1] = (unsigned long long)__double_as_longlong(v.y);
    em = max(em, max(exp_field(v.x), exp_field(v.y)));
  }
  atomicMax(&cmax[c8], em);
  __syncthreads();
  const int eb = cmax[c8];
  const int E = eb ? eb - 1021 : 0;   // max |v| < 2^(eb - 1022) = 2^(E - 1)
  if (t < 8) ex[(size_t)w * ncolp + c] = E;
  const size_t plane = (size_t)rowsp * ncolp;   // elements of one (slice, part) plane
  const size_t blk = ((size_t)g * (rowsp / 8) + (size_t)w * (kWin / 8) + rg) * 64 + c8 * 8 + half * 4;
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    uint16_t dg[4][kS];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const bool nf = non_finite(bits[2 * i + p]);
      digits7(nf ? 0LL : fixed56(bits[2 * i + p], E), dg[i]);
#pragma unroll
      for (int s = 0; s < kS; ++s) dg[i][s] = nf ? (uint16_t)0x7FC0 : dg[i][s];
    }
#pragma unroll
    for (int s = 0; s < kS; ++s) {
      const uint2 v = make_uint2((uint32_t)dg[0][s] | ((uint32_t)dg[1][s] << 16),
                                 (uint32_t)dg[2][s] | ((uint32_t)dg[3][s] << 16));
      *reinterpret_cast<uint2*>(sl + (size_t)(2 * s + p) * plane + blk) = v;
    }
  }
}

// double-float helpers (FP32 pairs; no reassociation)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// (h, l) += v
__device__ __forceinline__ void df_add1(float& h, float& l, float v) {
  float s, e;
  two_sum(h, v, s, e);
  e += l;
  h = s + e;
  l = e - (h - s);
}
// (h, l) += (h2, l2)
__device__ __forceinline__ void df_add2(float& h, float& l, float h2, float l2) {
  float s, e;
  two_sum(h, h2, s, e);
  e += l + l2;
  h = s + e;
  l = e - (h - s);
}
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((127 + k) << 23); }   // -126 <= k <= 127
// (h + l) 2^k as a double, from a normalised double-float pair (|l| <= ulp(h) / 2), with integer
// operations only (FP64 instructions, conversions included, are slow on this part): the
// significands are aligned in a 64-bit integer; exact up to a truncation below 2^-52 of h.
// The caller keeps the result's exponent in range (|k| <= 60 and h a normal FP32 number).
__device__ __forceinline__ double df_to_double(float h, float l, int k) {
  const uint32_t hb = __float_as_uint(h), lb = __float_as_uint(l);
  const int eh = (int)((hb >> 23) & 255u);
  if (eh == 0) return 0.0;
  if (eh == 255) return __longlong_as_double(0x7FF8000000000000LL);   // NaN or infinity
  long long m = (long long)((hb & 0x7FFFFFu) | 0x800000u) << 29;   // implicit bit at position 52
  const int el = (int)((lb >> 23) & 255u);
  if (el) {
    const int d = eh - el;                                          // >= 24 for a normalised pair
    if (d < 53) {
      const long long ml = ((long long)((lb & 0x7FFFFFu) | 0x800000u) << 29) >> d;
      m += ((hb ^ lb) >> 31) ? -ml : ml;
    }
  }
  long long e = (long long)(eh - 127 + 1023 + k);
  if (m < (1LL << 52)) {   // a borrow took the leading bit
    m <<= 1;
    --e;
  }
  return __longlong_as_double(((long long)(hb >> 31) << 63) | (e << 52) | (m & ((1LL << 52) - 1)));
}

// ================================================================ Gram: A = Z^H HZ, S = Z^H Z
// A tile is 128 columns of Z (MMA M) against 48 columns of HZ (A) or of Z (S), over a chunk of
// whole windows.  Warp 0: TMA producer (per 16-row stage one 5-D copy of the A slices and one
// copy per slice of the B slices); warp 1: MMA issuer and TMEM owner; warps 2-17: fold; warp 18:
// writes -B_re next to each slice's B_im.  Per slice t the stage then holds [B_re | B_im | -B_re]
// (48 rows each), and per pair (s, t) two MMAs of N = 96, A_re(s) [B_re | B_im] and A_im(s)
// [B_im | -B_re], add the real and imaginary parts into one accumulator (the N = 96 operands keep
// the tensor core's shared-memory reads per multiply-add low).  TMEM: five accumulators x
// (re 48 | im 48) columns.  At the end of a window the fold warps read the five accumulators
// (the MMAs of the next window wait only for that read), scale by 2^(E_a + E_b - 16) and add
// into double-float registers.
constexpr int G_N = 48;
constexpr uint32_t G_A_BYTES = kS * 2 * 16 * 2 * kCore;     // [s][p][16 column groups][2 row groups]
constexpr uint32_t G_BP_BYTES = (G_N / 8) * 2 * kCore;      // one part of one B slice: 6 groups x 2
constexpr uint32_t G_BS_BYTES = 3 * G_BP_BYTES;             // [B_re | B_im | -B_re] of one slice
constexpr uint32_t G_STG = G_A_BYTES + kS * G_BS_BYTES;
constexpr uint32_t G_TX = G_A_BYTES + kS * 2 * G_BP_BYTES;   // bytes landed by TMA per stage
constexpr int G_NSTG = 2;
constexpr int G_THREADS = 19 * 32;
constexpr size_t G_SMEM = 1024 + G_NSTG * (size_t)G_STG + 256;
constexpr int G_STEPS = kWin / 16;                          // 16-row stages per window
constexpr uint32_t G_REG = 2 * G_N;                         // TMEM columns per accumulator

struct GTile {
  int ia0, jb, src;   // Z columns [ia0, ia0 + 128) against columns [jb, jb + 48) of HZ (src 0) or Z (src 1)
};
struct GramArgs {
  int nwin, wpc, ntiles, ncolp, ncolpb;   // column capacities of A (Z) and of the B operand
  const GTile* tile;
  const int* exz;     // [window][ncolp] exponents of Z
  const int* exh;     // of HZ
  double2* part;      // [split][tile][48 columns][128 rows]
};

__global__ void __launch_bounds__(G_THREADS, 1) k_oz_gram(const __grid_constant__ CUtensorMap tz,
                                                         const __grid_constant__ CUtensorMap tzb,
                                                         const __grid_constant__ CUtensorMap th, GramArgs p) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const GTile tl = p.tile[blockIdx.x];
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + G_NSTG * (size_t)G_STG);
  uint64_t* stg_full = bars;               // [G_NSTG] copies landed
  uint64_t* neg_full = stg_full + G_NSTG;  // [G_NSTG] -B_re written
  uint64_t* stg_empty = neg_full + G_NSTG; // [G_NSTG] MMAs done with the stage
  uint64_t* acc_full = stg_empty + G_NSTG; // window sums in TMEM
  uint64_t* acc_empty = acc_full + 1;      // read by the 16 fold warps
  uint64_t* drainb = acc_empty + 1;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(drainb + 1);
  volatile int* sflag = reinterpret_cast<volatile int*>(tmem_holder + 1);

  const int w0 = blockIdx.y * p.wpc;
  const int nw = max(0, min(p.nwin, w0 + p.wpc) - w0);
  const int total = nw * G_STEPS;

  if (tid == 0) {
    for (int i = 0; i < G_NSTG; ++i) {
      mbar_init(&stg_full[i], 1);
      mbar_init(&neg_full[i], 1);
      mbar_init(&stg_empty[i], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, 16);
    mbar_init(drainb, 1);
    *sflag = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(tmem_holder, 512u);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      int issued = 0;
      const CUtensorMap* mb = tl.src ? &tzb : &th;   // B boxes: 6 column groups, one slice
      for (int q = 0; q < total && !*sflag; ++q) {
        const int st = q % G_NSTG;
        if (q >= G_NSTG && !mbar_wait(&stg_empty[st], (uint32_t)((q / G_NSTG) - 1) & 1u)) {
          *sflag = 1;
          break;
        }
        unsigned char* s = sm + (size_t)st * G_STG;
        const int rgc = (w0 + q / G_STEPS) * (kWin / 8) + (q % G_STEPS) * 2;
        mbar_expect_tx(&stg_full[st], G_TX);
        tma_load_5d(s, &tz, 0, rgc, tl.ia0 / 8, 0, 0, &stg_full[st]);
        for (int t = 0; t < kS; ++t)
          tma_load_5d(s + G_A_BYTES + t * G_BS_BYTES, mb, 0, rgc, tl.jb / 8, 0, t, &stg_full[st]);
        issued = q + 1;
      }
      for (int q = max(0, issued - G_NSTG); q < issued; ++q) mbar_wait(&stg_full[q % G_NSTG], (uint32_t)(q / G_NSTG) & 1u);
    }
  } else if (warp == 18) {
    // ---------------------------------------------------------------- -B_re next to B_im
    for (int q = 0; q < total && !*sflag; ++q) {
      const int st = q % G_NSTG;
      if (!mbar_wait(&stg_full[st], (uint32_t)(q / G_NSTG) & 1u)) {
        *sflag = 1;
        break;
      }
      unsigned char* b = sm + (size_t)st * G_STG + G_A_BYTES;
      for (int i = lane; i < kS * (int)(G_BP_BYTES / 16); i += 32) {
        const int t = i / (G_BP_BYTES / 16), o = (i % (G_BP_BYTES / 16)) * 16;
        const uint4 v = *reinterpret_cast<const uint4*>(b + t * G_BS_BYTES + o);
        *reinterpret_cast<uint4*>(b + t * G_BS_BYTES + 2 * G_BP_BYTES + o) =
            make_uint4(v.x ^ 0x80008000u, v.y ^ 0x80008000u, v.z ^ 0x80008000u, v.w ^ 0x80008000u);
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&neg_full[st]);
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t id96 = idesc_bf16(128, 2 * G_N);
      for (int q = 0; q < total && !*sflag; ++q) {
        const int st = q % G_NSTG, wl = q / G_STEPS, ks = q % G_STEPS;
        bool ok = mbar_wait(&neg_full[st], (uint32_t)(q / G_NSTG) & 1u);
        if (ok && ks == 0 && wl >= 1) ok = mbar_wait(acc_empty, (uint32_t)(wl - 1) & 1u);
        if (!ok) {
          *sflag = 1;
          break;
        }
        tc_fence_after();
        const uint32_t sa = saddr(sm + (size_t)st * G_STG), sb = sa + G_A_BYTES;
#pragma unroll
        for (int pr = 0; pr < kPairs; ++pr) {
          const int s = pair_s(pr), t = pair_t(pr), reg = pair_reg(pr);
          const uint32_t acc = (ks == 0 && pair_first(pr)) ? 0u : 1u;
          const uint64_t are = sdesc(sa + (uint32_t)(2 * s) * 4096u, 128, 256);
          const uint64_t aim = sdesc(sa + (uint32_t)(2 * s + 1) * 4096u, 128, 256);
          const uint64_t p1 = sdesc(sb + (uint32_t)t * G_BS_BYTES, 128, 256);               // [B_re | B_im]
          const uint64_t p2 = sdesc(sb + (uint32_t)t * G_BS_BYTES + G_BP_BYTES, 128, 256);  // [B_im | -B_re]
          const uint32_t d = tmem + G_REG * (uint32_t)reg;
          mma_bf16(d, are, p1, id96, acc);
          mma_bf16(d, aim, p2, id96, 1u);
        }
        mma_commit(&stg_empty[st]);
        if (ks == G_STEPS - 1) mma_commit(acc_full);
      }
      mma_commit(drainb);
      mbar_wait(drainb, 0u);
    }
  } else {
    // ---------------------------------------------------------------- fold, then the partial tile
    const int lq = warp & 3, cq = (warp - 2) >> 2;     // lanes [32 lq, +32), columns [12 cq, 12 cq + 12)
    const int row = 32 * lq + lane;
    const int ia = tl.ia0 + row;
    const int* exb = tl.src ? p.exz : p.exh;
    float ah[24], al[24];                              // re: 0..11, im: 12..23
    int eref[12];
#pragma unroll
    for (int e = 0; e < 24; ++e) ah[e] = al[e] = 0.f;
#pragma unroll
    for (int e = 0; e < 12; ++e) eref[e] = INT_MIN;
    for (int wl = 0; wl < nw && !*sflag; ++wl) {
      // scales of this window (loaded while the window's MMAs run)
      const int w = w0 + wl;
      const int ea = ia < p.ncolp ? p.exz[(size_t)w * p.ncolp + ia] : 0;
      float sc[12];
#pragma unroll
      for (int e = 0; e < 12; ++e) {
        const int j = tl.jb + 12 * cq + e;
        const int k = ea + (j < p.ncolpb ? exb[(size_t)w * p.ncolpb + j] : 0) - 16;
        if (eref[e] == INT_MIN) eref[e] = k;
        int d = k - eref[e];
        if (d > 60) {   // a window far larger than the reference: rescale the running sums
          const float r = d > 126 ? 0.f : pow2f(-d);
          ah[e] *= r;
          al[e] *= r;
          ah[12 + e] *= r;
          al[12 + e] *= r;
          eref[e] = k;
          d = 0;
        }
        sc[e] = d < -100 ? 0.f : pow2f(d);   // below 2^-100 of the running sums: dropped
      }
      if (!mbar_wait(acc_full, (uint32_t)wl & 1u)) {
        *sflag = 1;
        break;
      }
      tc_fence_after();
      const uint32_t base = tmem + ((uint32_t)(32 * lq) << 16) + 12u * (uint32_t)cq;
#pragma unroll
      for (int reg = 0; reg < kRegs; ++reg) {
        float re[12], im[12];
        tmem_ld12x2(base + G_REG * (uint32_t)reg, base + G_REG * (uint32_t)reg + G_N, re, im);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          df_add2(ah[k], al[k], re[k] * sc[k], 0.f);
          df_add2(ah[12 + k], al[12 + k], im[k] * sc[k], 0.f);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty);
    }
    if (!*sflag) {
      double2* dst = p.part + ((size_t)blockIdx.y * p.ntiles + blockIdx.x) * (size_t)G_N * 128;
#pragma unroll
      for (int e = 0; e < 12; ++e) {
        const int col = 12 * cq + e;
        const int k = eref[e] == INT_MIN ? 0 : eref[e];
        dst[(size_t)col * 128 + row] = double2{ldexp((double)ah[e] + (double)al[e], k),
                                               ldexp((double)ah[12 + e] + (double)al[12 + e], k)};
      }
    }
  }
  if (*sflag && tid == 0) atomicExch(&g_oz_status, DKS_ERR_TIMEOUT);
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 512u);
  }
}

// Sum of the partial tiles over the chunks in FP64, fixed order (warp order of strided sums).
// mode 0 (Gram): lower triangles of A (tiles of HZ) and S (tiles of Z), column-major with ldc;
// mode 1: C[j ldc + i] = (A^H B)_ij for i < m, j < n; mode 2: C[i ldc + j] = conj (= B^H A).
struct GRedArgs {
  int splits, ntiles, m, n, ldc, mode;
  const GTile* tile;
  const double2* part;
  double2* a;
  double2* s;
};
__global__ void __launch_bounds__(256) k_oz_gram_reduce(GRedArgs p) {
  __shared__ double2 red[8][32];
  const int tile = blockIdx.y;
  const GTile tl = p.tile[tile];
  const int col = blockIdx.x >> 2, r0 = (blockIdx.x & 3) * 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = r0 + lane;
  double sx = 0.0, sy = 0.0;
  const size_t stride = (size_t)p.ntiles * G_N * 128;
  const double2* src = p.part + (size_t)tile * G_N * 128 + (size_t)col * 128 + row;
  for (int s = warp; s < p.splits; s += 8) {
    const double2 v = src[(size_t)s * stride];
    sx += v.x;
    sy += v.y;
  }
  red[warp][lane] = double2{sx, sy};
  __syncthreads();
  if (warp == 0) {
    double2 t = red[0][lane];
#pragma unroll
    for (int w = 1; w < 8; ++w) {
      t.x += red[w][lane].x;
      t.y += red[w][lane].y;
    }
    const int i = tl.ia0 + row, j = tl.jb + col;
    if (p.mode == 0) {
      if (i < p.m && j <= i) (tl.src ? p.s : p.a)[(size_t)j * p.ldc + i] = t;
    } else if (i < p.m && j < p.n) {
      if (p.mode == 1) p.a[(size_t)j * p.ldc + i] = t;
      else p.a[(size_t)i * p.ldc + j] = double2{t.x, -t.y};
    }
  }
}

// W'[j][c] = alpha ws[c] w[j ldw + c] (projector update: the channel weights D and the filter scale)
__global__ void k_oz_scale_w(const double2* __restrict__ w, int ldw, const double* __restrict__ ws, double alpha,
                             int m, int n, double2* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m * n) return;
  const int c = i % m, j = i / m;
  const double2 v = w[(size_t)j * ldw + c];
  const double f = ws ? alpha * ws[c] : alpha;
  out[i] = double2{v.x * f, v.y * f};
}

// ================================================================ rotation: OUT = alpha Z W (+ beta OUT)
// Persistent over row tiles of 128 rows (= one exponent window); grid row y: output columns
// [nt y, nt y + nt), nt <= 48.  The B operand W' = diag(2^E(t, c)) W depends on the row tile t
// through the window exponents of Z and is sliced per tile: per output column j the exponent
// F_j = max_c (E(t, c) + e(W[c][j])) + 1 makes |W'[c][j]| < 2^(F_j - 1), and the products
// a_s w_t carry the scale 2^(F_j - 16).  Per slice t the converters write two B operands of
// N = 2 nt rows, P1 = [W'_re ; W'_im] and P2 = [-W'_im ; W'_re], so that per pair (s, t) two MMAs
// A_re(s) P1(t) + A_im(s) P2(t) give (re | im) of the product in one accumulator.
//   warp 0       producer: per 16-column chunk one 5-D TMA copy of the Z slices (128 rows)
//   warp 1       MMA issuer, TMEM owner
//   warps 2-5    converters: exponents F_j of the tile, then per chunk the W' slices (K-major B)
//   warps 6-21   fold: the five accumulators of the tile in double-float, scaled, written
// The A operand is stored MN-major (rows contiguous within a core matrix).  TMEM: five
// accumulators x (re nt | im nt) columns.
constexpr int R_NTMAX = 48;
constexpr int R_KC = 16;                                   // columns of Z per chunk (one MMA K-step)
constexpr uint32_t R_A_BYTES = kS * 2 * 2 * 16 * kCore;    // [s][p][2 column groups][16 row groups]
constexpr int R_NSTG = 2;
constexpr int R_CMAX = 128;                                // columns of Z per launch (exact level sums)
constexpr int R_CWIN = 120;                                // columns of W per launch (R_CMAX less a group)
constexpr int R_CONV = 4;                                  // converter warps
constexpr int R_THREADS = 22 * 32;
// one B operand (P1 or P2) of a slice: [2 nt / 8 row groups][2 K groups][core]
__host__ __device__ constexpr uint32_t r_b_op(int nt) { return (uint32_t)(2 * nt / 8) * 2 * kCore; }
__host__ __device__ constexpr uint32_t r_b_bytes(int nt) { return (uint32_t)kS * 2 * r_b_op(nt); }
constexpr size_t R_SMEM = 1024 + R_NSTG * (size_t)R_A_BYTES + 2 * (size_t)r_b_bytes(R_NTMAX) +
                          (size_t)R_CMAX * R_NTMAX * sizeof(int16_t) + (size_t)R_CONV * R_CMAX * sizeof(int) +
                          2 * R_NTMAX * sizeof(int) + 256;

struct RotArgs {
  int rows, tiles, ncolp;
  int cg0, kch;          // first column group of Z, chunks of 16 columns
  int c0, m;             // columns [c0, c0 + m) of Z meet rows [0, m) of W
  int n, nt;             // output columns, per grid row
  int ldw, ldo;
  uint32_t a_lbo, a_sbo; // MN-major descriptor offsets of the A operand (K direction, M direction)
  const double2* w;
  const int* ex;         // [window][ncolp]
  double2* out;
  double beta;
};

__global__ void __launch_bounds__(R_THREADS, 1) k_oz_rot(const __grid_constant__ CUtensorMap tz, RotArgs p) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nt = p.nt, n0 = (int)blockIdx.y * nt;
  const uint32_t bbytes = r_b_bytes(nt);
  const uint32_t bop = r_b_op(nt);                                      // one of P1, P2 of a slice
  const int kcols = p.kch * R_KC;
  unsigned char* sa = sm;                                               // [R_NSTG][R_A_BYTES]
  unsigned char* sbw = sa + R_NSTG * (size_t)R_A_BYTES;                 // [2][slice][P1, P2]
  int16_t* ew = reinterpret_cast<int16_t*>(sbw + 2 * (size_t)r_b_bytes(R_NTMAX));   // [kcols][R_NTMAX]
  int* et = reinterpret_cast<int*>(ew + R_CMAX * R_NTMAX);              // [R_CONV][kcols] window exponents
  int* fj = et + R_CONV * R_CMAX;                                       // [2][R_NTMAX] column exponents
  uint64_t* bars = reinterpret_cast<uint64_t*>(fj + 2 * R_NTMAX);
  uint64_t* stg_full = bars;                 // [R_NSTG]
  uint64_t* stg_empty = stg_full + R_NSTG;   // [R_NSTG]
  uint64_t* bop_full = stg_empty + R_NSTG;   // [2] (converter warps)
  uint64_t* bop_empty = bop_full + 2;        // [2]
  uint64_t* acc_full = bop_empty + 2;
  uint64_t* acc_empty = acc_full + 1;        // (16 fold warps)
  uint64_t* fj_full = acc_empty + 1;         // [2] column exponents of a tile written (converter warps)
  uint64_t* fj_read = fj_full + 2;           // [2] read by the 16 fold warps
  uint64_t* drainb = fj_read + 2;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(drainb + 1);
  volatile int* sflag = reinterpret_cast<volatile int*>(tmem_holder + 1);

  const int my_tiles = (int)blockIdx.x < p.tiles ? (p.tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int total = my_tiles * p.kch;

  if (tid == 0) {
    for (int i = 0; i < R_NSTG; ++i) {
      mbar_init(&stg_full[i], 1);
      mbar_init(&stg_empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bop_full[i], R_CONV);
      mbar_init(&bop_empty[i], 1);
      mbar_init(&fj_full[i], R_CONV);
      mbar_init(&fj_read[i], 16);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, 16);
    mbar_init(drainb, 1);
    *sflag = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(tmem_holder, 512u);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      int issued = 0;
      for (int q = 0; q < total && !*sflag; ++q) {
        const int st = q % R_NSTG;
        if (q >= R_NSTG && !mbar_wait(&stg_empty[st], (uint32_t)((q / R_NSTG) - 1) & 1u)) {
          *sflag = 1;
          break;
        }
        const int t = (int)blockIdx.x + (q / p.kch) * (int)gridDim.x, ch = q % p.kch;
        mbar_expect_tx(&stg_full[st], R_A_BYTES);
        tma_load_5d(sa + (size_t)st * R_A_BYTES, &tz, 0, t * (kWin / 8), p.cg0 + 2 * ch, 0, 0, &stg_full[st]);
        issued = q + 1;
      }
      for (int q = max(0, issued - R_NSTG); q < issued; ++q) mbar_wait(&stg_full[q % R_NSTG], (uint32_t)(q / R_NSTG) & 1u);
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(128, 2 * nt) | kAMajorMN;
      for (int q = 0; q < total && !*sflag; ++q) {
        const int st = q % R_NSTG, ob = q & 1, ti = q / p.kch, ch = q % p.kch;
        bool ok = mbar_wait(&stg_full[st], (uint32_t)(q / R_NSTG) & 1u);
        if (ok) ok = mbar_wait(&bop_full[ob], (uint32_t)(q >> 1) & 1u);
        if (ok && ch == 0 && ti >= 1) ok = mbar_wait(acc_empty, (uint32_t)(ti - 1) & 1u);
        if (!ok) {
          *sflag = 1;
          break;
        }
        tc_fence_after();
        const uint32_t a0 = saddr(sa + (size_t)st * R_A_BYTES), b0 = saddr(sbw + (size_t)ob * bbytes);
#pragma unroll
        for (int pr = 0; pr < kPairs; ++pr) {
          const int s = pair_s(pr), t = pair_t(pr), reg = pair_reg(pr);
          const uint32_t acc = (ch == 0 && pair_first(pr)) ? 0u : 1u;
          const uint64_t are = sdesc(a0 + (uint32_t)(2 * s) * 4096u, p.a_lbo, p.a_sbo);
          const uint64_t aim = sdesc(a0 + (uint32_t)(2 * s + 1) * 4096u, p.a_lbo, p.a_sbo);
          const uint64_t p1 = sdesc(b0 + (uint32_t)(2 * t) * bop, 128, 256);
          const uint64_t p2 = sdesc(b0 + (uint32_t)(2 * t + 1) * bop, 128, 256);
          const uint32_t d = tmem + (uint32_t)(2 * nt * reg);
          mma_bf16(d, are, p1, idesc, acc);
          mma_bf16(d, aim, p2, idesc, 1u);
        }
        mma_commit(&stg_empty[st]);
        mma_commit(&bop_empty[ob]);
        if (ch == p.kch - 1) mma_commit(acc_full);
      }
      mma_commit(drainb);
      mbar_wait(drainb, 0u);
    }
  } else if (warp < 2 + R_CONV) {
    // ---------------------------------------------------------------- converters
    // Warp v owns output columns [16 v, 16 v + 16) of the tile (lane pair per column, one lane per
    // 8-column half of a chunk); every warp works on its own data and hands over by mbarriers.
    const int v = warp - 2;
    const int jl = 16 * v + (lane >> 1), kg = lane & 1;
    const bool mine = jl < nt;
    int* etw = et + v * R_CMAX;
    // exponents of W (once): e(W[c][j]) for the chunk columns c, INT_MIN/2 for zero entries
    for (int it = lane; it < kcols * 16; it += 32) {
      const int cl = it >> 4, jj = 16 * v + (it & 15);
      if (jj >= nt) continue;
      const int wc = p.cg0 * 8 + cl - p.c0, j = n0 + jj;
      int e = -30000;   // zero entry
      if (wc >= 0 && wc < p.m && j < p.n) {
        const double2 x = p.w[(size_t)j * p.ldw + wc];
        const int eb = max(exp_field(x.x), exp_field(x.y));
        if (eb) e = eb - 1022;
      }
      ew[cl * R_NTMAX + jj] = (int16_t)e;
    }
    int q = 0;
    for (int ti = 0; ti < my_tiles && !*sflag; ++ti) {
      const int t = (int)blockIdx.x + ti * (int)gridDim.x;
      __syncwarp();
      for (int cl = lane; cl < kcols; cl += 32) {
        const int c = p.cg0 * 8 + cl;
        etw[cl] = c < p.ncolp ? p.ex[(size_t)t * p.ncolp + c] : 0;
      }
      __syncwarp();
      // F_j of the tile into buffer ti & 1, once the fold warps have read it for tile ti - 2
      if (ti >= 2 && !mbar_wait(&fj_read[ti & 1], (uint32_t)((ti >> 1) - 1) & 1u)) {
        *sflag = 1;
        break;
      }
      int fjv = 0;
      if (mine) {
        int f = INT_MIN / 2;
        for (int cl = 0; cl < kcols; ++cl)
          if (ew[cl * R_NTMAX + jl] > -30000) f = max(f, etw[cl] + (int)ew[cl * R_NTMAX + jl]);
        fjv = f > INT_MIN / 4 ? f + 1 : 0;
        if (kg == 0) fj[(ti & 1) * R_NTMAX + jl] = fjv;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&fj_full[ti & 1]);
      bool broke = false;
      for (int ch = 0; ch < p.kch; ++ch, ++q) {
        const int ob = q & 1;
        if (q >= 2 && !mbar_wait(&bop_empty[ob], (uint32_t)((q >> 1) - 1) & 1u)) {
          *sflag = 1;
          broke = true;
          break;
        }
        if (mine) {
          unsigned char* dstb = sbw + (size_t)ob * bbytes;
          // core-matrix row of B row r (of 2 nt) for the 8 columns of half kg
          auto off = [&](int r) { return (uint32_t)(((r >> 3) * 2 + kg) * kCore + (r & 7) * 16); };
          // the eight W values of this lane first (independent read-only loads, one latency),
          // then their digits
          double2 wv[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int wc = p.cg0 * 8 + ch * R_KC + kg * 8 + e - p.c0, j = n0 + jl;
            wv[e] = (wc >= 0 && wc < p.m && j < p.n) ? __ldg(p.w + (size_t)j * p.ldw + wc) : double2{0.0, 0.0};
          }
#pragma unroll
          for (int pp = 0; pp < 2; ++pp) {
            uint32_t wd[kS][4];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const int cl = ch * R_KC + kg * 8 + e;
              // W' = 2^E(t, c) W relative to 2^F_j: the window exponent enters the shift
              const double x = pp ? wv[e].y : wv[e].x;
              const long long f = fixed56((unsigned long long)__double_as_longlong(x), fjv - etw[cl]);
              uint16_t dg[kS];
              digits7(f, dg);
#pragma unroll
              for (int s = 0; s < kS; ++s) {
                if (e & 1) wd[s][e >> 1] |= (uint32_t)dg[s] << 16;
                else wd[s][e >> 1] = (uint32_t)dg[s];
              }
            }
#pragma unroll
            for (int s = 0; s < kS; ++s) {
              const uint4 v = make_uint4(wd[s][0], wd[s][1], wd[s][2], wd[s][3]);
              unsigned char* p1 = dstb + (size_t)(2 * s) * bop;
              unsigned char* p2 = p1 + bop;
              if (pp == 0) {   // re: P1 row jl, P2 row nt + jl
                *reinterpret_cast<uint4*>(p1 + off(jl)) = v;
                *reinterpret_cast<uint4*>(p2 + off(nt + jl)) = v;
              } else {         // im: P1 row nt + jl, P2 row jl negated
                *reinterpret_cast<uint4*>(p1 + off(nt + jl)) = v;
                *reinterpret_cast<uint4*>(p2 + off(jl)) =
                    make_uint4(v.x ^ 0x80008000u, v.y ^ 0x80008000u, v.z ^ 0x80008000u, v.w ^ 0x80008000u);
              }
            }
          }
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bop_full[ob]);
      }
      if (broke) break;
    }
  } else {
    // ---------------------------------------------------------------- fold and write
    const int lq = warp & 3, cq = (warp - 2 - R_CONV) >> 2;   // lanes [32 lq, +32), columns [cq ncw, +ncw)
    const int ncw = nt / 4;                                    // 4, 8 or 12 columns per warp
    for (int ti = 0; ti < my_tiles && !*sflag; ++ti) {
      const int t = (int)blockIdx.x + ti * (int)gridDim.x;
      bool ok = mbar_wait(&fj_full[ti & 1], (uint32_t)(ti >> 1) & 1u);
      if (ok) ok = mbar_wait(acc_full, (uint32_t)ti & 1u);
      if (!ok) {
        *sflag = 1;
        break;
      }
      tc_fence_after();
      int fcol[12];
#pragma unroll
      for (int e = 0; e < 12; ++e) fcol[e] = e < ncw ? fj[(ti & 1) * R_NTMAX + cq * ncw + e] : 0;
      __syncwarp();
      if (lane == 0) mbar_arrive(&fj_read[ti & 1]);
      float h[24], l[24];                                      // re: e, im: 12 + e
      const uint32_t base = tmem + ((uint32_t)(32 * lq) << 16) + (uint32_t)(cq * ncw);
#pragma unroll
      for (int reg = 0; reg < kRegs; ++reg) {
        // 12 columns from the warp's first: those past its ncw belong to the next warp's columns
        // of the same accumulators (read, not used)
        float re[12], im[12];
        tmem_ld12x2(base + (uint32_t)(2 * nt * reg), base + (uint32_t)(2 * nt * reg + nt), re, im);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          if (reg == 0) {
            h[k] = re[k];
            h[12 + k] = im[k];
            l[k] = l[12 + k] = 0.f;
          } else {
            df_add1(h[k], l[k], re[k]);
            df_add1(h[12 + k], l[12 + k], im[k]);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty);
      // FP64 is slow on this part: scale the double-float pair in FP32 (exact power of two while
      // in range), then one FP64 add per value (and one FMA for beta)
      const int r = t * kWin + 32 * lq + lane;
      if (r < p.rows) {
#pragma unroll
        for (int e = 0; e < 12; ++e) {
          const int j = n0 + cq * ncw + e;
          if (e < ncw && j < p.n) {
            const int k = fcol[e] - 16;
            double2 v;
            if (k >= -60 && k <= 60) {
              v.x = df_to_double(h[e], l[e], k);
              v.y = df_to_double(h[12 + e], l[12 + e], k);
            } else {
              v.x = ldexp((double)h[e] + (double)l[e], k);
              v.y = ldexp((double)h[12 + e] + (double)l[12 + e], k);
            }
            double2* o = p.out + (size_t)j * p.ldo + r;
            if (p.beta != 0.0) {
              const double2 old = *o;
              v.x = fma(p.beta, old.x, v.x);
              v.y = fma(p.beta, old.y, v.y);
            }
            *o = v;
          }
        }
      }
    }
  }
  if (*sflag && tid == 0) atomicExch(&g_oz_status, DKS_ERR_TIMEOUT);
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 512u);
  }
}

// ---------------------------------------------------------------- host side
std::mutex g_mu;
bool g_attr = false;
// MN-major A operand without swizzle: LBO = stride of the core matrices along K (2 column groups
// apart: 16 row groups x 128 bytes), SBO = stride along M (adjacent row groups)
#ifndef OZ_A_LBO
#define OZ_A_LBO 2048
#endif
#ifndef OZ_A_SBO
#define OZ_A_SBO 128
#endif
constexpr uint32_t g_a_lbo = OZ_A_LBO, g_a_sbo = OZ_A_SBO;

// 5-D map over a slice buffer: (64 core elements, row groups, column groups, part, slice)
int make_map5(CUtensorMap* map, const OzBlock& z, int box_rg, int box_cg, int box_s = kS) {
  PFN_cuTensorMapEncodeTiled_v12000 enc;
  DKS_TRY(tc::encoder(&enc));
  const cuuint64_t R = (cuuint64_t)(z.rowsp / 8), G = (cuuint64_t)(z.ncolp / 8);
  const cuuint64_t dims[5] = {64, R, G, 2, (cuuint64_t)kS};
  const cuuint64_t strides[4] = {kCore, R * kCore, G * R * kCore, 2 * G * R * kCore};
  const cuuint32_t box[5] = {64, (cuuint32_t)box_rg, (cuuint32_t)box_cg, 2, (cuuint32_t)box_s};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, z.sl, dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(DKS_ERR_CUDA, "exact-slice contractions: cuTensorMapEncodeTiled failed (" +
                                                       std::to_string((int)r) + ")");
  return DKS_OK;
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

int set_attrs() {
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_attr) {
    DKS_CUDA_TRY(cudaFuncSetAttribute((const void*)k_oz_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G_SMEM));
    DKS_CUDA_TRY(cudaFuncSetAttribute((const void*)k_oz_rot, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)R_SMEM));
    g_attr = true;
  }
  return DKS_OK;
}

}  // namespace oz

// ================================================================ entry points (dks_internal.h)
size_t oz_bytes(int rows, int ncol) {
  const size_t rowsp = (size_t)(rows + oz::kWin - 1) / oz::kWin * oz::kWin;
  const size_t ncolp = (size_t)(ncol + 7) / 8 * 8;
  return 2 * oz::kS * rowsp * ncolp * sizeof(uint16_t) + (rowsp / oz::kWin) * ncolp * sizeof(int) + 256;
}

int oz_layout(void* buf, int rows, int ncol, OzBlock* out) {
  OzBlock z;
  z.rows = rows;
  z.ncol = ncol;
  z.rowsp = (rows + oz::kWin - 1) / oz::kWin * oz::kWin;
  z.ncolp = (ncol + 7) / 8 * 8;
  z.sl = reinterpret_cast<uint16_t*>(buf);
  const size_t sl_bytes = 2 * oz::kS * (size_t)z.rowsp * z.ncolp * sizeof(uint16_t);
  z.ex = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(buf) + (sl_bytes + 255) / 256 * 256);
  *out = z;
  return DKS_OK;
}

int oz_split(const double2* a, long long lda, int ncol, const OzBlock& z, cudaStream_t st) {
  if (ncol <= 0 || z.rows <= 0) return DKS_OK;
  if (ncol > z.ncol) return fail(DKS_ERR_INVALID_ARG, "exact slices: more columns than the block holds");
  Prof pr(P_MISC, st, 16.0 * ncol * z.rows + 28.0 * (double)z.rowsp * std::min(z.ncolp, (ncol + 23) / 8 * 8), 0.0);
  // 16 columns past ncol are written as zeros: a rotation's last 16-column chunk may reach them
  const dim3 grid(z.rowsp / oz::kWin, std::min(z.ncolp / 8, (ncol + 16 + 7) / 8));
  oz::k_oz_split<<<grid, 256, 0, st>>>(a, lda, z.rows, ncol, z.rowsp, z.ncolp, z.sl, z.ex);
  DKS_CUDA_TRY(cudaGetLastError());
  return DKS_OK;
}

namespace oz {
// A^H B over tiles: A (tz, 128-column boxes), B from hz (src 0) or z (src 1), partial tiles per
// chunk of windows, then the fixed-order reduction in the given mode.
int hn_tiles(const OzBlock& z, const OzBlock& hz, const std::vector<GTile>& tiles, int m, int n, double2* a,
             double2* s, int ldc, int mode, cudaStream_t st) {
  DKS_TRY(set_attrs());
  const int nt = (int)tiles.size();
  const int nwin = z.rowsp / kWin;
  const int nsm = sm_count();
  // chunks of whole windows: about two CTAs per SM in total
  int splits = std::max(1, std::min(nwin, (2 * nsm + nt - 1) / nt));
  const int wpc = (nwin + splits - 1) / splits;
  splits = (nwin + wpc - 1) / wpc;
  CUtensorMap tz, th;
  DKS_TRY(make_map5(&tz, z, 2, 16));
  DKS_TRY(make_map5(&th, hz, 2, G_N / 8, 1));
  CUtensorMap tzb;   // Z as the B operand: boxes of 6 column groups, one slice
  DKS_TRY(make_map5(&tzb, z, 2, G_N / 8, 1));
  if (nt > 65535) return fail(DKS_ERR_UNSUPPORTED, "exact-slice A^H B: too many tiles");
  const size_t tl_bytes = (tiles.size() * sizeof(GTile) + 255) / 256 * 256;
  const size_t part_bytes = (size_t)splits * nt * G_N * 128 * sizeof(double2);
  unsigned char* buf = nullptr;
  DKS_CUDA_TRY(cudaMallocAsync((void**)&buf, tl_bytes + part_bytes, st));
  GTile* dtiles = reinterpret_cast<GTile*>(buf);
  double2* part = reinterpret_cast<double2*>(buf + tl_bytes);
  cudaError_t e = cudaMemcpyAsync(dtiles, tiles.data(), tiles.size() * sizeof(GTile), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    GramArgs p{};
    p.nwin = nwin;
    p.wpc = wpc;
    p.ntiles = nt;
    p.ncolp = z.ncolp;
    p.ncolpb = hz.ncolp;   // tiles of src 1 (B from Z) occur only in the Gram form, where both agree
    p.tile = dtiles;
    p.exz = z.ex;
    p.exh = hz.ex;
    p.part = part;
    k_oz_gram<<<dim3(nt, splits), G_THREADS, G_SMEM, st>>>(tz, tzb, th, p);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    GRedArgs r{};
    r.splits = splits;
    r.ntiles = nt;
    r.m = m;
    r.n = n;
    r.ldc = ldc;
    r.mode = mode;
    r.tile = dtiles;
    r.part = part;
    r.a = a;
    r.s = s;
    k_oz_gram_reduce<<<dim3(G_N * 4, nt), 256, 0, st>>>(r);
    e = cudaGetLastError();
  }
  cudaFreeAsync(buf, st);
  if (e != cudaSuccess) return fail(DKS_ERR_CUDA, std::string("exact-slice A^H B launch: ") + cudaGetErrorString(e));
  return DKS_OK;
}
}  // namespace oz

// lower triangles of A = Z^H HZ and S = Z^H Z over the first m columns (ldc = m)
int oz_gram(const OzBlock& z, const OzBlock& hz, int m, double2* a, double2* s, cudaStream_t st) {
  using namespace oz;
  if (m <= 0) return DKS_OK;
  if (z.rowsp != hz.rowsp || z.ncolp != hz.ncolp || m > z.ncol)
    return fail(DKS_ERR_INVALID_ARG, "exact-slice Gram: mismatched blocks");
  std::vector<GTile> tiles;
  const int mt = (m + 127) / 128;
  for (int ib = 0; ib < mt; ++ib) {
    const int jmax = std::min(m, ib * 128 + 128);   // lower triangle: columns j <= i
    for (int src = 0; src < 2; ++src)
      for (int jb = 0; jb < jmax; jb += G_N) tiles.push_back(GTile{ib * 128, jb, src});
  }
  Prof pr(P_GRAM, st, 2.0 * 28.0 * z.rowsp * ((m + 7) / 8 * 8) + 32.0 * m * m, 8.0 * m * (m + 1.0) * (double)z.rows);
  return hn_tiles(z, hz, tiles, m, m, a, s, m, 0, st);
}

// C = A^H B (m x n, ldc), or with conj_transpose_out C = B^H A (n x m, ldc)
int oz_gemm_hn(const OzBlock& a, int m, const OzBlock& b, int n, double2* c, int ldc, bool conj_transpose_out,
               cudaStream_t st, int cat) {
  using namespace oz;
  if (m <= 0 || n <= 0) return DKS_OK;
  if (a.rowsp != b.rowsp || m > a.ncol || n > b.ncol)
    return fail(DKS_ERR_INVALID_ARG, "exact-slice A^H B: mismatched blocks");
  std::vector<GTile> tiles;
  for (int ib = 0; ib < (m + 127) / 128; ++ib)
    for (int jb = 0; jb < n; jb += G_N) tiles.push_back(GTile{ib * 128, jb, 0});
  Prof pr(cat, st, 28.0 * a.rowsp * ((m + 7) / 8 * 8 + (n + 7) / 8 * 8) + 16.0 * m * n, 8.0 * m * n * (double)a.rows);
  return hn_tiles(a, b, tiles, m, n, c, nullptr, ldc, conj_transpose_out ? 2 : 1, st);
}

// OUT (rows x n, ldo) = alpha Z[:, c0 : c0 + m] W (+ beta OUT), W: m x n complex128 (ldw)
int oz_rotate(const OzBlock& z, int c0, int m, const double2* w, int ldw, int n, double2* out, int ldo, double beta,
              cudaStream_t st, double alpha, const double* wscale, int cat) {
  using namespace oz;
  if (m <= 0 || n <= 0 || z.rows <= 0) return DKS_OK;
  if (c0 < 0 || c0 + m > z.ncol) return fail(DKS_ERR_INVALID_ARG, "exact-slice rotation: columns outside the block");
  if (wscale || alpha != 1.0) {
    // W' = alpha diag(ws) W (a small FP64 pass), then the plain rotation
    double2* ws2 = nullptr;
    DKS_CUDA_TRY(cudaMallocAsync((void**)&ws2, (size_t)m * n * sizeof(double2), st));
    k_oz_scale_w<<<(m * n + 255) / 256, 256, 0, st>>>(w, ldw, wscale, alpha, m, n, ws2);
    int rc = cudaGetLastError() == cudaSuccess ? DKS_OK : fail(DKS_ERR_CUDA, "exact-slice rotation: scaling launch");
    if (!rc) rc = oz_rotate(z, c0, m, ws2, m, n, out, ldo, beta, st, 1.0, nullptr, cat);
    cudaFreeAsync(ws2, st);
    return rc;
  }
  DKS_TRY(set_attrs());
  Prof pr(cat, st, 28.0 * z.rowsp * ((m + 7) / 8 * 8) + (beta != 0.0 ? 2.0 : 1.0) * 16.0 * n * z.rows,
          8.0 * (double)z.rows * m * n);
  const int ytiles = (n + R_NTMAX - 1) / R_NTMAX;
  const int nt = (((n + ytiles - 1) / ytiles) + 15) / 16 * 16;
  const int tiles = z.rowsp / kWin;
  const int grid_x = std::min(tiles, sm_count());
  CUtensorMap tz;
  DKS_TRY(make_map5(&tz, z, kWin / 8, 2));
  const uint32_t lbo = g_a_lbo, sbo = g_a_sbo;
  // windows of at most 120 columns (with the offset into the first column group at most 128:
  // exact level sums); later windows add into OUT in FP64
  for (int cs = 0; cs < m; cs += R_CWIN) {
    const int mc = std::min(R_CWIN, m - cs);
    const int cstart = c0 + cs;
    RotArgs p{};
    p.rows = z.rows;
    p.tiles = tiles;
    p.ncolp = z.ncolp;
    p.cg0 = cstart / 8;
    p.kch = ((cstart + mc) - p.cg0 * 8 + R_KC - 1) / R_KC;
    p.c0 = cstart;
    p.m = mc;
    p.n = n;
    p.nt = nt;
    p.ldw = ldw;
    p.ldo = ldo;
    p.a_lbo = lbo;
    p.a_sbo = sbo;
    p.w = w + cs;
    p.ex = z.ex;
    p.out = out;
    p.beta = cs == 0 ? beta : 1.0;
    if (p.kch * R_KC > R_CMAX) return fail(DKS_ERR_UNSUPPORTED, "exact-slice rotation: chunk bound");
    k_oz_rot<<<dim3(grid_x, ytiles), R_THREADS, R_SMEM, st>>>(tz, p);
    DKS_CUDA_TRY(cudaGetLastError());
  }
  return DKS_OK;
}

bool projector_slices(dks_ctx* ctx, int ik, cudaStream_t st) {
  static std::mutex mu;
  std::lock_guard<std::mutex> g(mu);
  KPoint& kp = ctx->k[ik];
  if (kp.btoz_state) return kp.btoz_state > 0;
  kp.btoz_state = -1;
  if (!ctx->nproj || !kp.bt64) return false;
  // the slices are a speed-up (the double-float contractions remain): held only with room to spare
  const size_t bytes = oz_bytes(2 * kp.npw, ctx->nproj);
  size_t freeb = 0, totalb = 0;
  if (cudaMemGetInfo(&freeb, &totalb) != cudaSuccess || bytes > freeb / 4) {
    cudaGetLastError();
    return false;
  }
  if (cudaMalloc(&kp.btoz, bytes) != cudaSuccess) {
    cudaGetLastError();
    kp.btoz = nullptr;
    return false;
  }
  OzBlock b;
  oz_layout(kp.btoz, 2 * kp.npw, ctx->nproj, &b);
  // made once on this stream, then read from any stream of the context
  if (oz_split(kp.bt64, 2 * kp.npw, ctx->nproj, b, st) != DKS_OK || cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(kp.btoz);
    kp.btoz = nullptr;
    return false;
  }
  kp.btoz_state = 1;
  return true;
}

int oz_status_take() {
  int v = 0;
  DKS_CUDA_TRY(cudaMemcpyFromSymbol(&v, oz::g_oz_status, sizeof(int)));
  if (v) {
    const int zero = 0;
    DKS_CUDA_TRY(cudaMemcpyToSymbol(oz::g_oz_status, &zero, sizeof(int)));
  }
  return v;
}

}  // namespace dks

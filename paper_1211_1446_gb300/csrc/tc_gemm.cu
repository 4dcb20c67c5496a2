// Tall-skinny complex contractions of Algorithm 1 on the fifth-generation tensor cores (tcgen05).
//
// Complex64 blocks are multiplied with FP32 accuracy through BF16 slices: every FP32 value x is
// the exact sum x = h + m + l of three bfloat16 values (h = bf16(x), m = bf16(x - h),
// l = x - h - m, each remainder exact in FP32), and a product a b is formed from the six slice
// products h h' + h m' + m h' + h l' + l h' + m m'; the three that are left out are below
// 2^-24 |a b| together.  Each slice product is an exact FP32 number, accumulated in FP32 in
// tensor memory (TMEM).  Complex arithmetic is real arithmetic on interleaved (re, im) pairs:
//
//   nn  OUT (rows x n) = A (rows x m) W' (m x n) + beta OUT, W' = alpha diag(ws) W
//       (rotations X <- Z V, P <- [0, Y, P] V, projector update x~ += B (D Z)):
//       D[row][c] = sum_k A[row][k] B[c][k] over the interleaved inner index k = 2j + (re, im),
//       with B[c] = (w_r, -w_i) pairs for the real part of column c and B[n + c] = (w_i, w_r)
//       for its imaginary part; one MMA of N = 2 n columns gives both.
//   hn  C (m x n) = A^H B over the tall index (Gram matrices S = Z^H Z, A = Z^H HZ, projector
//       coefficients B^H x~): D_re = A B^T and D_im = A' B^T over interleaved pairs, with
//       A' = i A = (-a_i, a_r) formed while the operand is converted.  The tall index is split
//       across CTAs (chunks of at most kchunk rows, so each FP32 accumulation in TMEM is short);
//       every CTA writes its FP32 partial tile and a second kernel adds the partials of each
//       entry in FP64 in a fixed order (deterministic).
//
// Data movement: A (and, for hn, B) tiles are copied global -> shared memory by TMA
// (cp.async.bulk.tensor.2d onto an mbarrier with expect-tx) through a staging ring as deep as
// shared memory allows (up to 8 stages); eight converter warps turn a staged tile into the three
// BF16 slices in the canonical no-swizzle K-major layout (8-row x 16-byte core matrices); one
// thread issues the tcgen05.mma
// instructions (kind::f16, BF16 inputs, FP32 accumulator in TMEM, M = 128) and tcgen05.commit
// releases the operand buffers; the epilogue reads TMEM with tcgen05.ld.  Every mbarrier wait
// is bounded: a wait that gives up records DKS_ERR_TIMEOUT in a device status word, the CTA
// drains its own copies and MMAs in flight (bounded again), frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>
#include <vector>

#include "dks_internal.h"
#include "tc_ptx.cuh"

namespace dks {
namespace tc {

__device__ int g_tc_status = 0;             // DKS_ERR_TIMEOUT after a wait gave up

// x = h + m + l exactly (three BF16 slices), for a pair of values (low half = first)
__device__ __forceinline__ void split3(float a, float b, uint32_t& h, uint32_t& m, uint32_t& l) {
  const __nv_bfloat162 hh = __floats2bfloat162_rn(a, b);
  const float ra = a - __low2float(hh), rb = b - __high2float(hh);
  const __nv_bfloat162 mm = __floats2bfloat162_rn(ra, rb);
  const __nv_bfloat162 ll = __floats2bfloat162_rn(ra - __low2float(mm), rb - __high2float(mm));
  h = *reinterpret_cast<const uint32_t*>(&hh);
  m = *reinterpret_cast<const uint32_t*>(&mm);
  l = *reinterpret_cast<const uint32_t*>(&ll);
}
// eight consecutive K values of one operand row -> one 16-byte core-matrix row in each slice
__device__ __forceinline__ void store_slices(unsigned char* base, uint32_t slice_bytes, uint32_t off,
                                             const float (&v)[8]) {
  uint32_t h[4], m[4], l[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) split3(v[2 * q], v[2 * q + 1], h[q], m[q], l[q]);
  *reinterpret_cast<uint4*>(base + off) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(base + slice_bytes + off) = make_uint4(m[0], m[1], m[2], m[3]);
  *reinterpret_cast<uint4*>(base + 2 * slice_bytes + off) = make_uint4(l[0], l[1], l[2], l[3]);
}
// byte offset of (row r, core-matrix column kg) in a K-major no-swizzle tile with kgs core
// matrices along K
__device__ __forceinline__ uint32_t core_off(int r, int kg, int kgs) {
  return (uint32_t)(((r >> 3) * kgs + kg) * 128 + (r & 7) * 16);
}
// slice pairs of the six products, largest first: (h, h'), (h, m'), (m, h'), (h, l'), (l, h'),
// (m, m'); compile-time functions, so the MMA issuer's descriptor offsets fold into constants
__host__ __device__ constexpr int pair_a(int p) { return p == 2 || p == 5 ? 1 : p == 4 ? 2 : 0; }
__host__ __device__ constexpr int pair_b(int p) { return p == 1 || p == 5 ? 1 : p == 3 ? 2 : 0; }

// ================================================================ nn: OUT = A W' (+ beta OUT)
// W' is split once per call into BF16 slices laid out as the MMA's B operand (k_tc_split_w), per
// column tile and 16-band chunk.  The main kernel is warp-specialised and persistent over 128-row
// tiles of one column tile (grid row y: output columns [nt y, nt (y + 1)), nt <= 64):
//   warp 0       producer: per stage one TMA copy of A (16 bands x 128 rows, FP32) and one bulk
//                copy of the W' chunk into a staging slot
//   warp 1       MMA issuer (one lane) and owner of the TMEM allocation
//   warps 2-9    converters: staged A -> BF16 slices (two operand buffers)
//   warps 10-17  fold and epilogue: per stage, the leading products h h' are read from TMEM
//                and added into FP32 registers; at the end of a tile the set of the smaller
//                products is added and the tile is written (+ beta OUT)
// With beta != 0 the producer also copies the tile's old OUT values into shared memory by TMA
// at the tile's first chunk (one or two tile buffers), so the epilogue reads them from shared
// memory instead of waiting on its own global loads while the tensor core idles.
// TMEM (512 columns): two or three buffers of the leading products (one per stage in flight,
// fresh each stage; three when five buffers fit), two buffers of the smaller products (one per
// tile in flight), so the tensor core can run ahead while the fold warps write a tile.  The
// leading products thus take at most two accumulation steps in TMEM: the tensor core's FP32
// accumulation is not correctly rounded, and its error grows coherently when one accumulator
// takes many steps, while the sums in registers are rounded to nearest.  Every hand-off is an
// mbarrier; every wait is bounded.
constexpr int NN_KT = 16;                           // complex inner indices per stage
constexpr int NN_KR = 2 * NN_KT;                    // interleaved real K per stage (2 MMA K-steps)
constexpr uint32_t NN_STG_A = kM * NN_KT * 8;       // FP32 staging of A: [16 j][128 rows] float2
constexpr uint32_t NN_A_SLICE = kM * NN_KR * 2;     // one BF16 slice of A: 128 rows x 32 K
constexpr int NN_STG_MAX = 8;                       // staging ring depth (chosen per launch)
constexpr int NN_OPS = 2;                           // A operand buffers
constexpr int NN_NTMAX = 64;                        // output columns of a CTA's column tile
constexpr int NN_THREADS = 18 * 32;
constexpr size_t NN_SMEM_LIMIT = 227 * 1024;

struct NNArgs {
  int k, m, n, nt, ldo, sw, nstg;
  int nob;                             // OUT tile buffers staged by TMA (0: the epilogue loads them)
  int nhi;                             // TMEM buffers of the leading products (2 or 3)
  const unsigned char* wsl;            // [ytile][chunk][3 slices][2 nt rows][32 K] BF16
  float2* out;
  float beta;
};

__host__ __device__ inline uint32_t nn_b_slice(int nt) { return (uint32_t)(2 * nt) * NN_KR * 2; }
__host__ inline size_t nn_slot(int nt) { return NN_STG_A + 3 * (size_t)nn_b_slice(nt); }
__host__ __device__ inline uint32_t nn_old_bytes(int nt) { return (uint32_t)kM * nt * 8; }
__host__ inline size_t nn_fixed() { return 1024 + NN_OPS * 3 * (size_t)NN_A_SLICE + 512; }

// W'[j][c] = alpha ws[j] w[c ldw + j] (rounded to FP32) -> BF16 slices of the B operand: row c of
// a column tile holds (w_r, -w_i) pairs, row nt + c holds (w_i, w_r); bands j >= m and columns
// c >= n are zero
__global__ void k_tc_split_w(const double2* __restrict__ w, int ldw, const double* __restrict__ ws, double alpha,
                             int m, int n, int nt, int nch, int ytiles, unsigned char* __restrict__ wsl) {
  const uint32_t bslice = nn_b_slice(nt);
  const int items = ytiles * nch * nt * 4;
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < items; it += gridDim.x * blockDim.x) {
    const int g = it & 3, c = (it >> 2) % nt, tc_ = (it >> 2) / nt;
    const int ch = tc_ % nch, yt = tc_ / nch;
    const int col = yt * nt + c;
    float re8[8], im8[8];
#pragma unroll
    for (int q4 = 0; q4 < 4; ++q4) {
      const int j = ch * NN_KT + 4 * g + q4;
      float wr = 0.f, wi = 0.f;
      if (j < m && col < n) {
        const double2 v = w[(size_t)col * ldw + j];
        const double sc = (ws ? ws[j] : 1.0) * alpha;
        wr = (float)(v.x * sc);
        wi = (float)(v.y * sc);
      }
      re8[2 * q4] = wr;
      re8[2 * q4 + 1] = -wi;
      im8[2 * q4] = wi;
      im8[2 * q4 + 1] = wr;
    }
    unsigned char* base = wsl + ((size_t)yt * nch + ch) * 3 * bslice;
    store_slices(base, bslice, core_off(c, g, 4), re8);
    store_slices(base, bslice, core_off(nt + c, g, 4), im8);
  }
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   saddr(dst)),
               "l"(src), "r"(bytes), "r"(saddr(bar))
               : "memory");
}

template <bool kOld>
__global__ void __launch_bounds__(NN_THREADS, 1) k_tc_gemm_nn(const __grid_constant__ CUtensorMap tmap,
                                                             const __grid_constant__ CUtensorMap tout, NNArgs p) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nt = p.nt, nb2 = 2 * nt, n0 = (int)blockIdx.y * nt, nstg = p.nstg;
  const uint32_t bslice = nn_b_slice(nt);
  const uint32_t slot = NN_STG_A + 3 * bslice;
  unsigned char* stg = sm;                                       // [nstg][A FP32 | W' slices]
  unsigned char* opa = sm + (size_t)nstg * slot;
  unsigned char* oldb = opa + NN_OPS * 3 * NN_A_SLICE;           // [nob][nt cols][128 rows] float2
  const int nob = kOld ? p.nob : 1;   // ring length of the OUT tile buffers (read only with kOld)
  const uint32_t obytes = nn_old_bytes(nt);
  uint64_t* bars = reinterpret_cast<uint64_t*>(oldb + (kOld ? (size_t)nob * obytes : 0));
  uint64_t* stg_full = bars;                        // [nstg] A and W' landed
  uint64_t* stg_empty = stg_full + NN_STG_MAX;      // [nstg] the MMAs reading the slot completed
  uint64_t* op_full = stg_empty + NN_STG_MAX;       // [NN_OPS] A slices written (8 converter warps)
  uint64_t* op_empty = op_full + NN_OPS;            // [NN_OPS] MMAs that read them completed
  uint64_t* acc_full = op_empty + NN_OPS;           // [3] leading products of a stage in TMEM
  uint64_t* acc_empty = acc_full + 3;               // [3] read by the 8 fold warps
  uint64_t* corr_full = acc_empty + 3;              // [2] smaller products of a tile in TMEM
  uint64_t* corr_empty = corr_full + 2;             // [2] read by the 8 fold warps
  uint64_t* old_full = corr_empty + 2;              // [2] old OUT tile landed
  uint64_t* old_empty = old_full + 2;               // [2] read by the 8 fold warps
  uint64_t* drainb = old_empty + 2;                 // every MMA issued has completed
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(drainb + 1);
  volatile int* sflag = reinterpret_cast<volatile int*>(tmem_holder + 1);

  const int rowtiles = (p.k + kM - 1) / kM;
  const int nch = (p.m + NN_KT - 1) / NN_KT;
  const int my_tiles = blockIdx.x < rowtiles ? (rowtiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int total = my_tiles * nch;
  const unsigned char* wsl = p.wsl + (size_t)blockIdx.y * nch * 3 * bslice;

  if (tid == 0) {
    for (int i = 0; i < nstg; ++i) {
      mbar_init(&stg_full[i], 1);
      mbar_init(&stg_empty[i], 1);
    }
    for (int i = 0; i < NN_OPS; ++i) {
      mbar_init(&op_full[i], 8);
      mbar_init(&op_empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&corr_full[i], 1);
      mbar_init(&corr_empty[i], 8);
      mbar_init(&old_full[i], 1);
      mbar_init(&old_empty[i], 8);
    }
    for (int i = 0; i < 3; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], 8);
    }
    mbar_init(drainb, 1);
    *sflag = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(tmem_holder, 512u);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;
  // nhi buffers of the leading products (3 when five accumulator sets fit in TMEM), then two of
  // the smaller products
  const int nhi = p.nhi;
  const uint32_t hi_col[3] = {0u, (uint32_t)p.sw, (uint32_t)(2 * p.sw)};
  const uint32_t corr_col[2] = {(uint32_t)(nhi * p.sw), (uint32_t)((nhi + 1) * p.sw)};

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    int issued = 0, oissued = 0;
    if (lane == 0) {
      for (int q = 0; q < total && !*sflag; ++q) {
        const int st = q % nstg;
        if (q >= nstg && !mbar_wait(&stg_empty[st], (uint32_t)((q / nstg) - 1) & 1u)) {
          *sflag = 1;
          break;
        }
        const int tt = q / nch, t = blockIdx.x + tt * gridDim.x, ch = q % nch;
        unsigned char* s = stg + (size_t)st * slot;
        mbar_expect_tx(&stg_full[st], slot);
        tma_load_2d(s, &tmap, 2 * kM * t, NN_KT * ch, &stg_full[st]);
        bulk_load(s + NN_STG_A, wsl + (size_t)ch * 3 * bslice, 3 * bslice, &stg_full[st]);
        issued = q + 1;
        if (kOld && ch == 0) {
          // the tile's old OUT values (rows and columns outside OUT read as zero)
          const int ob = tt % nob;
          if (tt >= nob && !mbar_wait(&old_empty[ob], (uint32_t)((tt / nob) - 1) & 1u)) {
            *sflag = 1;
            break;
          }
          mbar_expect_tx(&old_full[ob], obytes);
          tma_load_2d(oldb + (size_t)ob * obytes, &tout, 2 * kM * t, n0, &old_full[ob]);
          oissued = tt + 1;
        }
      }
      // copies still in flight land before the CTA exits (bounded)
      for (int q = std::max(0, issued - nstg); q < issued; ++q)
        mbar_wait(&stg_full[q % nstg], (uint32_t)(q / nstg) & 1u);
      if (kOld)
        for (int tt = std::max(0, oissued - nob); tt < oissued; ++tt)
          mbar_wait(&old_full[tt % nob], (uint32_t)(tt / nob) & 1u);
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(kM, nb2);
      const uint64_t da0 = sdesc(saddr(opa), 128, 512), db0 = sdesc(saddr(stg + NN_STG_A), 128, 512);
      for (int q = 0; q < total && !*sflag; ++q) {
        const int st = q % nstg, op = q % NN_OPS, b = q % nhi, tt = q / nch, ch = q % nch, cb = tt & 1;
        bool w = mbar_wait(&stg_full[st], (uint32_t)(q / nstg) & 1u);
        if (w) w = mbar_wait(&op_full[op], (uint32_t)(q / NN_OPS) & 1u);
        if (w && q >= nhi) w = mbar_wait(&acc_empty[b], (uint32_t)((q / nhi) - 1) & 1u);
        if (w && ch == 0 && tt >= 2) w = mbar_wait(&corr_empty[cb], (uint32_t)((tt >> 1) - 1) & 1u);
        if (!w) {
          *sflag = 1;
          break;
        }
        tc_fence_after();
        const uint64_t da = da0 + ((uint64_t)(op * 3 * NN_A_SLICE) >> 4);
        const uint64_t db = db0 + ((uint64_t)(st * slot) >> 4);
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
          mma_bf16(tmem + hi_col[b], da + (uint64_t)(ks * 16), db + (uint64_t)(ks * 16), idesc, (uint32_t)ks);
#pragma unroll
          for (int pr = 1; pr < 6; ++pr) {
            const uint64_t ad = da + ((uint64_t)(pair_a(pr) * NN_A_SLICE + ks * 256) >> 4);
            const uint64_t bd = db + ((uint64_t)(pair_b(pr) * bslice + ks * 256) >> 4);
            mma_bf16(tmem + corr_col[cb], ad, bd, idesc, (ch | ks | (pr - 1)) != 0);
          }
        }
        mma_commit(&op_empty[op]);
        mma_commit(&stg_empty[st]);
        mma_commit(&acc_full[b]);
        if (ch == nch - 1) mma_commit(&corr_full[cb]);
      }
      mma_commit(drainb);
      mbar_wait(drainb, 0u);
    }
  } else if (warp < 10) {
    // ---------------------------------------------------------------- converters
    const int ct = tid - 64;                       // 0 .. 255
    for (int q = 0; q < total && !*sflag; ++q) {
      const int st = q % nstg, op = q % NN_OPS;
      bool w = mbar_wait(&stg_full[st], (uint32_t)(q / nstg) & 1u);
      if (w && q >= NN_OPS) w = mbar_wait(&op_empty[op], (uint32_t)((q / NN_OPS) - 1) & 1u);
      if (!w) {
        *sflag = 1;
        break;
      }
      // A chunk: staging [16 j][128 rows] -> A slices, row r = (re, im) pairs of 16 bands
      const float2* sg = reinterpret_cast<const float2*>(stg + (size_t)st * slot);
      unsigned char* oa = opa + (size_t)op * 3 * NN_A_SLICE;
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int it = ct + u * 256;
        const int r = it & (kM - 1), g = it >> 7;
        float v8[8];
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4) {
          const float2 a = sg[(4 * g + q4) * kM + r];
          v8[2 * q4] = a.x;
          v8[2 * q4 + 1] = a.y;
        }
        store_slices(oa, NN_A_SLICE, core_off(r, g, 4), v8);
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&op_full[op]);
    }
  } else {
    // ---------------------------------------------------------------- fold and epilogue
    const int lq = warp & 3, half = (warp - 10) >> 2;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * lq) << 16);
    float accr[2][16], acci[2][16];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int e = 0; e < 16; ++e) accr[u][e] = acci[u][e] = 0.f;
    auto add_set = [&](uint32_t col0) {
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int c0 = 16 * (2 * u + half);
        if (c0 < nt) {
          float re[16], im[16];
          tmem_ld16x2(lane_base + col0 + (uint32_t)c0, lane_base + col0 + (uint32_t)(nt + c0), re, im);
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            accr[u][e] += re[e];
            acci[u][e] += im[e];
          }
        }
      }
    };
    for (int q = 0; q < total && !*sflag; ++q) {
      const int b = q % nhi, tt = q / nch, ch = q % nch, cb = tt & 1;
      if (!mbar_wait(&acc_full[b], (uint32_t)(q / nhi) & 1u)) {
        *sflag = 1;
        break;
      }
      tc_fence_after();
      add_set(hi_col[b]);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[b]);
      if (ch == nch - 1) {
        if (!mbar_wait(&corr_full[cb], (uint32_t)(tt >> 1) & 1u)) {
          *sflag = 1;
          break;
        }
        tc_fence_after();
        add_set(corr_col[cb]);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&corr_empty[cb]);
        const int t = blockIdx.x + tt * gridDim.x;
        const int row = t * kM + 32 * lq + lane;
        float2* __restrict__ out = p.out;
        const float2* olds = nullptr;
        if (kOld) {
          if (!mbar_wait(&old_full[tt % nob], (uint32_t)(tt / nob) & 1u)) {
            *sflag = 1;
            break;
          }
          olds = reinterpret_cast<const float2*>(oldb + (size_t)(tt % nob) * obytes) + 32 * lq + lane;
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int c0 = 16 * (2 * u + half);
          if (c0 >= nt) continue;
          if (kOld) {
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              if (c0 + e < nt) {
                const float2 o = olds[(size_t)(c0 + e) * kM];
                accr[u][e] += p.beta * o.x;
                acci[u][e] += p.beta * o.y;
              }
            }
          } else if (p.beta != 0.f) {
            // beta OUT: every old value of the chunk is loaded before the first store, so the
            // loads overlap instead of waiting one by one behind possibly aliasing stores
#pragma unroll
            for (int h8 = 0; h8 < 16; h8 += 8) {
              float2 old[8];
#pragma unroll
              for (int e = 0; e < 8; ++e) {
                const int col = n0 + c0 + h8 + e;
                old[e] = (row < p.k && c0 + h8 + e < nt && col < p.n) ? __ldg(out + (size_t)col * p.ldo + row)
                                                                     : float2{0.f, 0.f};
              }
#pragma unroll
              for (int e = 0; e < 8; ++e) {
                accr[u][h8 + e] += p.beta * old[e].x;
                acci[u][h8 + e] += p.beta * old[e].y;
              }
            }
          }
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int col = n0 + c0 + e;
            if (row < p.k && c0 + e < nt && col < p.n)
              out[(size_t)col * p.ldo + row] = float2{accr[u][e], acci[u][e]};
            accr[u][e] = acci[u][e] = 0.f;
          }
        }
        if (kOld) {
          __syncwarp();
          if (lane == 0) mbar_arrive(&old_empty[tt % nob]);
        }
      }
    }
  }
  if (*sflag && tid == 0) atomicExch(&g_tc_status, DKS_ERR_TIMEOUT);
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 512u);
  }
}

// ================================================================ hn: C = A^H B (split over K)
// A tile is 128 columns of A (MMA M) against at most 64 columns of B (from B1 or B2; the Gram
// form takes HZ through B1 and Z through B2).  Warp-specialised like the nn kernel: warp 0 TMA
// producer, warp 1 MMA issuer and TMEM owner, warps 2-9 converters (A, A' = i A and B into BF16
// slices, two groups of four warps on alternate stages), warps 10-17 fold.  Each 16-deep stage
// writes fresh TMEM accumulators (real and
// imaginary part, in a ring of buffers across stages): the five smaller slice products first, the
// leading one last, so that at most one accumulation step at full magnitude enters each stage
// sum; the fold warps add the stage sums into FP32 registers over the CTA's K chunk and write
// the chunk's partial tile, which k_tc_reduce adds over the chunks in FP64 in a fixed order.
// Four operand buffers and four stage-sum buffers in TMEM let the converters run up to four
// stages ahead of the tensor core, and the tensor core four stages ahead of the fold.  A
// tiles narrower than 128 columns (the projector coefficients B^H x~ take the 36-channel table
// as A) convert only their own rows: the rest of every operand buffer is zeroed once, and B is
// then converted by the other half of the converter threads.
constexpr int HN_KT = 8;                            // complex rows per stage (16 real = one MMA K-step)
constexpr int HN_KR = 2 * HN_KT;
constexpr int HN_NB = 64;                           // largest N (B columns) of a tile
constexpr uint32_t HN_STG_A = kM * HN_KR * 4;       // FP32 staging of A: [128 cols][16 floats]
constexpr uint32_t HN_STG_B = HN_NB * HN_KR * 4;    // B box: [64 cols][16 floats]
constexpr uint32_t HN_STG_BYTES = HN_STG_A + HN_STG_B;
constexpr uint32_t HN_A_SLICE = kM * HN_KR * 2;     // 128 rows x 16 K BF16
constexpr uint32_t HN_B_SLICE = HN_NB * HN_KR * 2;  // 64 rows x 16 K BF16
constexpr uint32_t HN_OP_BYTES = 6 * HN_A_SLICE + 3 * HN_B_SLICE;   // A, A' and B slices
constexpr int HN_OPS = 4;                           // operand (BF16 slice) buffers
constexpr int HN_ACC = 4;                           // stage-sum buffers in TMEM (128 columns each)
constexpr size_t HN_SMEM_FIXED = 1024 + HN_OPS * (size_t)HN_OP_BYTES + 512;
constexpr int HN_THREADS = 18 * 32;
constexpr int HN_STG_MAX = 8;

// One output tile: rows = A columns [ia0, ia0 + 128), columns = B1 columns [jb1, jb1 + nb1)
// followed by B2 columns [jb2, jb2 + nb2), nb1 + nb2 <= 64 (<= 128 in the packed form).
struct HNTile {
  int ia0, jb1, nb1, jb2, nb2;
};
constexpr int kMaxTiles = 256;
constexpr int kArgTiles = 8;             // tile lists up to this length travel in the arguments
struct HNArgs {
  int m, k, kchunk, ntiles, nstg;        // m: columns of A
  int boxa, boxb;                        // columns of A and of B per TMA box (multiples of 8)
  int tcols;                             // columns of a partial tile (HN_NB, or HN_NBP packed)
  const HNTile* tile;                    // device copy of the tile list (more than kArgTiles)
  HNTile tv[kArgTiles];                  // the tile list itself (at most kArgTiles)
  float2* part;                          // [split][tile][tcols][128 rows]
};
constexpr int HN_NBP = 128;                         // largest N of a packed tile
// packed form (A of at most 64 columns, one A tile): the MMA's 128 rows hold A in rows 0-63 and
// A' = i A in rows 64-127, so one MMA per slice pair gives the real part in TMEM lanes 0-63 and
// the imaginary part in lanes 64-127, with N up to 128 B columns: 6 MMAs per stage instead of
// 12 per 64-column tile, and no MMA reads rows that are only padding.  Staging holds A in its
// first 4 KB and B (up to 128 columns) after it; the operand buffer holds the A/A' slices and
// then three B slices of 128 rows.
constexpr uint32_t HN_PK_BOFF = 64 * HN_KR * 4;     // staging offset of B in the packed form

template <bool kPacked>
__global__ void __launch_bounds__(HN_THREADS, 1) k_tc_gemm_hn(const __grid_constant__ CUtensorMap ta,
                                                             const __grid_constant__ CUtensorMap tb1,
                                                             const __grid_constant__ CUtensorMap tb2, HNArgs p) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const HNTile tl = p.ntiles <= kArgTiles ? p.tv[blockIdx.x] : p.tile[blockIdx.x];
  const int nbt = tl.nb1 + tl.nb2;
  const int nmma = (nbt + 15) & ~15;                   // MMA N (multiple of 16, <= 64; <= 128 packed)
  const int na = min(kM, p.m - tl.ia0);                // rows of the A tile inside A
  const int nstg = p.nstg;
  unsigned char* stg = sm;
  unsigned char* ops = sm + (size_t)nstg * HN_STG_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(ops + HN_OPS * HN_OP_BYTES);
  uint64_t* stg_full = bars;                           // [nstg] copies landed
  uint64_t* stg_empty = stg_full + HN_STG_MAX;         // [nstg] converted (4 converter warps)
  uint64_t* op_full = stg_empty + HN_STG_MAX;          // [HN_OPS] slices written (4 converter warps)
  uint64_t* op_empty = op_full + HN_OPS;                 // [HN_OPS] MMAs that read them completed
  uint64_t* acc_full = op_empty + HN_OPS;              // [HN_ACC] stage sums in TMEM
  uint64_t* acc_empty = acc_full + HN_ACC;             // [HN_ACC] read by the 8 fold warps
  uint64_t* drainb = acc_empty + HN_ACC;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(drainb + 1);
  volatile int* sflag = reinterpret_cast<volatile int*>(tmem_holder + 1);

  const int kb = blockIdx.y * p.kchunk;
  const int ke = min(p.k, kb + p.kchunk);
  const int total = ke > kb ? (ke - kb + HN_KT - 1) / HN_KT : 0;

  if (tid == 0) {
    for (int i = 0; i < nstg; ++i) {
      mbar_init(&stg_full[i], 1);
      mbar_init(&stg_empty[i], 4);                     // the 4 warps of one converter group
    }
    for (int i = 0; i < HN_OPS; ++i) {
      mbar_init(&op_full[i], 4);
      mbar_init(&op_empty[i], 1);
    }
    for (int i = 0; i < HN_ACC; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], 8);
    }
    mbar_init(drainb, 1);
    *sflag = 0;
    fence_barrier_init();
  }
  // A rows at and beyond na stay zero in every operand buffer; the converters skip them
  for (int e = tid; e < HN_OPS * (int)(HN_OP_BYTES / 16); e += HN_THREADS)
    reinterpret_cast<uint4*>(ops)[e] = make_uint4(0u, 0u, 0u, 0u);
  fence_async_smem();
  if (warp == 1) tmem_alloc(tmem_holder, 128u * HN_ACC);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;   // buffer b: real part at columns [128 b, 128 b + 64), imaginary at +64
  const uint32_t stg_bytes = (uint32_t)(p.boxa + p.boxb) * HN_KR * 4;   // only the columns a tile can use

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      int issued = 0;
      for (int q = 0; q < total && !*sflag; ++q) {
        const int st = q % nstg;
        if (q >= nstg && !mbar_wait(&stg_empty[st], (uint32_t)((q / nstg) - 1) & 1u)) {
          *sflag = 1;
          break;
        }
        unsigned char* s = stg + (size_t)st * HN_STG_BYTES;
        const int x = 2 * (kb + q * HN_KT);
        mbar_expect_tx(&stg_full[st], stg_bytes);
        tma_load_2d(s, &ta, x, tl.ia0, &stg_full[st]);
        const uint32_t boff = kPacked ? HN_PK_BOFF : HN_STG_A;
        if (tl.nb1 > 0) tma_load_2d(s + boff, &tb1, x, tl.jb1, &stg_full[st]);
        else tma_load_2d(s + boff, &tb2, x, tl.jb2, &stg_full[st]);
        issued = q + 1;
      }
      for (int q = std::max(0, issued - nstg); q < issued; ++q)
        mbar_wait(&stg_full[q % nstg], (uint32_t)(q / nstg) & 1u);
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(kM, nmma);
      const uint64_t d0 = sdesc(saddr(ops), 128, 256);
      for (int q = 0; q < total && !*sflag; ++q) {
        const int op = q % HN_OPS, b = q % HN_ACC;
        bool w = mbar_wait(&op_full[op], (uint32_t)(q / HN_OPS) & 1u);
        if (w && q >= HN_ACC) w = mbar_wait(&acc_empty[b], (uint32_t)((q / HN_ACC) - 1) & 1u);
        if (!w) {
          *sflag = 1;
          break;
        }
        tc_fence_after();
        const uint64_t da = d0 + ((uint64_t)(op * HN_OP_BYTES) >> 4);
        const uint32_t dre = tmem + 128u * (uint32_t)b;
        // the smaller products first, the leading one (pair 0) last
        if constexpr (kPacked) {
          const uint64_t db = da + ((uint64_t)(3 * HN_A_SLICE) >> 4);
#pragma unroll
          for (int k6 = 0; k6 < 6; ++k6) {
            const int pr = (k6 + 1) % 6;
            mma_bf16(dre, da + ((uint64_t)(pair_a(pr) * HN_A_SLICE) >> 4),
                     db + ((uint64_t)(pair_b(pr) * HN_A_SLICE) >> 4), idesc, k6 != 0);
          }
        } else {
          const uint64_t da2 = da + ((uint64_t)(3 * HN_A_SLICE) >> 4);
          const uint64_t db = da + ((uint64_t)(6 * HN_A_SLICE) >> 4);
          const uint32_t dim = dre + 64u;
#pragma unroll
          for (int k6 = 0; k6 < 6; ++k6) {
            const int pr = (k6 + 1) % 6;
            const uint64_t bd = db + ((uint64_t)(pair_b(pr) * HN_B_SLICE) >> 4);
            const uint64_t oa = (uint64_t)(pair_a(pr) * HN_A_SLICE) >> 4;
            mma_bf16(dre, da + oa, bd, idesc, k6 != 0);
            mma_bf16(dim, da2 + oa, bd, idesc, k6 != 0);
          }
        }
        mma_commit(&op_empty[op]);
        mma_commit(&acc_full[b]);
      }
      mma_commit(drainb);
      mbar_wait(drainb, 0u);
    }
  } else if (warp < 10) {
    // ---------------------------------------------------------------- converters
    // two groups of four warps take alternate stages, so one group's conversion and hand-off
    // overlap the other's
    const int grp = (warp - 2) >> 2;                  // 0 or 1
    const int ct = tid - 64 - 128 * grp;              // 0 .. 127
    const int na2 = 2 * na, items = na2 + 2 * nmma;
    for (int q = grp; q < total && !*sflag; q += 2) {
      const int st = q % nstg, op = q % HN_OPS;
      bool w = mbar_wait(&stg_full[st], (uint32_t)(q / nstg) & 1u);
      if (w && q >= HN_OPS) w = mbar_wait(&op_empty[op], (uint32_t)((q / HN_OPS) - 1) & 1u);
      if (!w) {
        *sflag = 1;
        break;
      }
      const float* sa = reinterpret_cast<const float*>(stg + (size_t)st * HN_STG_BYTES);
      // A slices, then A' slices (packed: A' in rows 64-127 of the A slices), then B slices
      unsigned char* oa = ops + (size_t)op * HN_OP_BYTES;
      unsigned char* oa2 = kPacked ? oa : oa + 3 * HN_A_SLICE;
      unsigned char* ob = oa + (kPacked ? 3 : 6) * HN_A_SLICE;
      const uint32_t bsl = kPacked ? HN_A_SLICE : HN_B_SLICE;
      const float* sb = sa + (kPacked ? HN_PK_BOFF : HN_STG_A) / 4;
      for (int it = ct; it < items; it += 128) {
        if (it < na2) {
          // A and A' = i A: row r = column ia0 + r of A, 16 interleaved values = 8 complex rows
          const int r = it >> 1, g = it & 1;
          const float* src = sa + r * HN_KR + 8 * g;
          float v8[8], w8[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) v8[e] = src[e];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            w8[2 * e] = -v8[2 * e + 1];
            w8[2 * e + 1] = v8[2 * e];
          }
          store_slices(oa, HN_A_SLICE, core_off(r, g, 2), v8);
          store_slices(oa2, HN_A_SLICE, core_off(kPacked ? 64 + r : r, g, 2), w8);
        } else {
          // B: rows [0, nbt) from the staged box, zero up to nmma
          const int r = (it - na2) >> 1, g = (it - na2) & 1;
          float v8[8];
          const float* src = sb + r * HN_KR + 8 * g;
#pragma unroll
          for (int e = 0; e < 8; ++e) v8[e] = r < nbt ? src[e] : 0.f;
          store_slices(ob, bsl, core_off(r, g, 2), v8);
        }
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&op_full[op]);
        mbar_arrive(&stg_empty[st]);
      }
    }
  } else {
    // ---------------------------------------------------------------- fold, then the partial tile
    // unpacked: warp (lq, half) holds rows 32 lq + lane, columns [32 half, 32 half + 32) of the
    // real (accr) and imaginary (acci) parts; packed: lanes 32 lq + lane hold the real part
    // (lq < 2) or the imaginary part (lq >= 2) of A row 32 (lq & 1) + lane, columns
    // [64 half, 64 half + 64) in accr (first 32) and acci (last 32)
    const int lq = warp & 3, half = (warp - 10) >> 2;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * lq) << 16);
    float accr[2][16], acci[2][16];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int e = 0; e < 16; ++e) accr[u][e] = acci[u][e] = 0.f;
    for (int q = 0; q < total && !*sflag; ++q) {
      const int b = q % HN_ACC;
      if (!mbar_wait(&acc_full[b], (uint32_t)(q / HN_ACC) & 1u)) {
        *sflag = 1;
        break;
      }
      tc_fence_after();
      const uint32_t bb = lane_base + 128u * (uint32_t)b;
      if constexpr (kPacked) {
        const int c0 = 64 * half;
        if (c0 < nbt) {
          float x0[16], x1[16];
          tmem_ld16x2(bb + (uint32_t)c0, bb + (uint32_t)(c0 + 16), x0, x1);
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            accr[0][e] += x0[e];
            accr[1][e] += x1[e];
          }
        }
        if (c0 + 32 < nbt) {
          float x0[16], x1[16];
          tmem_ld16x2(bb + (uint32_t)(c0 + 32), bb + (uint32_t)(c0 + 48), x0, x1);
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            acci[0][e] += x0[e];
            acci[1][e] += x1[e];
          }
        }
      } else {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int c0 = 32 * half + 16 * u;
          if (c0 < nbt) {
            float re[16], im[16];
            tmem_ld16x2(bb + (uint32_t)c0, bb + 64u + (uint32_t)c0, re, im);
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              accr[u][e] += re[e];
              acci[u][e] += im[e];
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[b]);
    }
    if (!*sflag) {
      float2* dst = p.part + ((size_t)blockIdx.y * p.ntiles + blockIdx.x) * (size_t)p.tcols * kM;
      if constexpr (kPacked) {
        float* df = reinterpret_cast<float*>(dst) + (lq >> 1);   // real or imaginary component
        const int ar = 32 * (lq & 1) + lane;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int c0 = 64 * half + 16 * u;
#pragma unroll
          for (int e = 0; e < 16; ++e)
            if (c0 + e < nbt) df[((size_t)(c0 + e) * kM + ar) * 2] = u < 2 ? accr[u][e] : acci[u - 2][e];
        }
      } else {
        const int row = 32 * lq + lane;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int c0 = 32 * half + 16 * u;
#pragma unroll
          for (int e = 0; e < 16; ++e)
            if (c0 + e < nbt) dst[(size_t)(c0 + e) * kM + row] = float2{accr[u][e], acci[u][e]};
        }
      }
    }
  }
  if (*sflag && tid == 0) atomicExch(&g_tc_status, DKS_ERR_TIMEOUT);
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 128u * HN_ACC);
  }
}

// Sum of the partial tiles over the splits in FP64, fixed order; 32 entries (consecutive rows
// of one column of a tile) per warp-slot, the splits spread over the 8 warps and added in warp
// order.  mode 0: C[(jb + j) * ldc + ia0 + i] (= A^H B), mode 1: C[(ia0 + i) * ldc + jb + j] =
// conj (= B^H A); gram: B1 columns go to C1, B2 columns to C2, lower triangle only.
struct RedArgs {
  int splits, ntiles, m, ldc, mode, gram, tcols;
  const HNTile* tile;                    // device copy of the tile list (more than kArgTiles)
  HNTile tv[kArgTiles];                  // the tile list itself (at most kArgTiles)
  const float2* part;
  double2* c1;
  double2* c2;
};

__global__ void __launch_bounds__(256) k_tc_reduce(RedArgs p) {
  __shared__ double2 red[8][32];
  const int tile = blockIdx.y;
  const HNTile tl = p.ntiles <= kArgTiles ? p.tv[tile] : p.tile[tile];
  const int nbt = tl.nb1 + tl.nb2;
  const int col = blockIdx.x >> 2, r0 = (blockIdx.x & 3) * 32;   // 4 slots of 32 rows per column
  if (col >= nbt || tl.ia0 + r0 >= p.m) return;                  // no row of the slot inside C
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = r0 + lane;
  double sx = 0.0, sy = 0.0;
  const size_t stride = (size_t)p.ntiles * p.tcols * kM;
  const float2* src = p.part + (size_t)tile * p.tcols * kM + (size_t)col * kM + row;
  int s = warp;
  // four loads in flight, added in split order
  for (; s + 24 < p.splits; s += 32) {
    float2 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = src[(size_t)(s + 8 * u) * stride];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      sx += (double)v[u].x;
      sy += (double)v[u].y;
    }
  }
  for (; s < p.splits; s += 8) {
    const float2 v = src[(size_t)s * stride];
    sx += (double)v.x;
    sy += (double)v.y;
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
    const int i = tl.ia0 + row;
    const bool second = col >= tl.nb1;
    const int j = second ? tl.jb2 + (col - tl.nb1) : tl.jb1 + col;
    if (i < p.m) {
      if (p.gram) {
        if (i >= j) (second ? p.c2 : p.c1)[(size_t)j * p.ldc + i] = t;
      } else if (p.mode == 0) {
        p.c1[(size_t)j * p.ldc + i] = t;
      } else {
        p.c1[(size_t)i * p.ldc + j] = double2{t.x, -t.y};
      }
    }
  }
}

// ---------------------------------------------------------------- host side
std::mutex g_mu;
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
int g_mask = -1;            // contractions on the tensor cores (TC_* bits); -1: not yet read
int g_kchunk = 512;         // longest K range of one FP32 accumulation in the hn kernel
bool g_attr_nn = false, g_attr_hn = false;

int encoder(PFN_cuTensorMapEncodeTiled_v12000* out) {
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
      return fail(DKS_ERR_CUDA, "tensor cores: cuTensorMapEncodeTiled is not available");
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  *out = g_encode;
  return DKS_OK;
}

// 2D FP32 tensor map over complex columns: inner = 2 * rows floats, outer = ncols columns of
// stride ld complex elements; box = (box_inner floats, box_rows columns)
int make_map(CUtensorMap* map, const void* base, long long rows, int ncols, long long ld, int box_inner, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc;
  DKS_TRY(encoder(&enc));
  const cuuint64_t dims[2] = {(cuuint64_t)(2 * rows), (cuuint64_t)ncols};
  const cuuint64_t strides[1] = {(cuuint64_t)(ld * 8)};
  const cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(DKS_ERR_CUDA, "tensor cores: cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return DKS_OK;
}

bool aligned_for_tma(const void* p, long long ld) {
  return (reinterpret_cast<uintptr_t>(p) & 15u) == 0 && (ld & 1) == 0 && ld > 0;
}

int device_ok() {
  static int ok = -1;
  std::lock_guard<std::mutex> g(g_mu);
  if (ok < 0) {
    int dev = 0, major = 0, minor = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    ok = (major == 10 && minor == 3) ? 1 : 0;
    if (ok) {
      // the partial tiles are stream-ordered allocations: keep freed blocks in the device's
      // default pool instead of returning them to the system at every synchronisation
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
      }
    }
  }
  return ok;
}

}  // namespace tc

int tc_mask() {
  std::lock_guard<std::mutex> g(tc::g_mu);
  if (tc::g_mask < 0) tc::g_mask = TC_DEFAULT;
  return tc::g_mask;
}

bool tc_enabled(int bit) { return (tc_mask() & bit) != 0 && tc::device_ok() == 1; }

bool tc_device() { return tc::device_ok() == 1; }

int tc_set(int mask, int kchunk) {
  std::lock_guard<std::mutex> g(tc::g_mu);
  tc::g_mask = mask & TC_ALL;
  if (kchunk > 0) tc::g_kchunk = std::max(tc::HN_KT, (kchunk / tc::HN_KT) * tc::HN_KT);
  return DKS_OK;
}

int tc_get(int* mask, int* kchunk) {
  if (mask) *mask = tc_mask();
  std::lock_guard<std::mutex> g(tc::g_mu);
  if (kchunk) *kchunk = tc::g_kchunk;
  return DKS_OK;
}

int tc_status_take() {
  int v = 0;
  DKS_CUDA_TRY(cudaMemcpyFromSymbol(&v, tc::g_tc_status, sizeof(int)));
  if (v) {
    const int z = 0;
    DKS_CUDA_TRY(cudaMemcpyToSymbol(tc::g_tc_status, &z, sizeof(int)));
  }
  const int w = oz_status_take();   // the exact-slice kernels keep their own word
  return v ? v : w;
}

bool tc_nn_supported(const float2* a, int lda, int k, int m, int n) {
  return k > 0 && m > 0 && n > 0 && tc::aligned_for_tma(a, lda);
}

int tc_gemm_nn(const float2* a, int lda, int k, int m, const double2* w, int ldw, const double* wscale, int n,
               float2* out, int ldo, double beta, cudaStream_t st, double alpha, int nsm) {
  using namespace tc;
  if (k <= 0 || n <= 0) return DKS_OK;
  CUtensorMap map;
  DKS_TRY(make_map(&map, a, k, m, lda, 2 * kM, NN_KT));
  const int ytiles = (n + NN_NTMAX - 1) / NN_NTMAX;
  const int nt = ((n + ytiles - 1) / ytiles + 7) & ~7;
  const int sw = (nt + ((nt + 15) & ~15) + 31) & ~31;   // one accumulator buffer (<= 128 columns)
  const int nch = (m + NN_KT - 1) / NN_KT;
  // beta OUT staged by TMA: two tile buffers when three staging slots still fit, else one when
  // two fit, else the epilogue loads the old values itself
  auto stages = [&](int nob) {
    const size_t fixed = nn_fixed() + (size_t)nob * nn_old_bytes(nt);
    return fixed >= NN_SMEM_LIMIT ? 0 : (int)std::min<size_t>(NN_STG_MAX, (NN_SMEM_LIMIT - fixed) / nn_slot(nt));
  };
  int nob = 0;
  CUtensorMap mout = map;
  if (beta != 0.0 && aligned_for_tma(out, ldo)) {
    nob = stages(2) >= 3 ? 2 : stages(1) >= 2 ? 1 : 0;
    if (nob) DKS_TRY(make_map(&mout, out, k, n, ldo, 2 * kM, nt));
  }
  const int nstg = stages(nob);
  const size_t smem = nn_fixed() + (size_t)nob * nn_old_bytes(nt) + (size_t)nstg * nn_slot(nt);
  {
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_attr_nn) {
      DKS_CUDA_TRY(cudaFuncSetAttribute((const void*)k_tc_gemm_nn<false>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)NN_SMEM_LIMIT));
      DKS_CUDA_TRY(cudaFuncSetAttribute((const void*)k_tc_gemm_nn<true>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)NN_SMEM_LIMIT));
      g_attr_nn = true;
    }
  }
  // W' in BF16 slices, per column tile and chunk (stream-ordered scratch)
  const size_t wbytes = (size_t)ytiles * nch * 3 * nn_b_slice(nt);
  unsigned char* wsl = nullptr;
  DKS_CUDA_TRY(cudaMallocAsync((void**)&wsl, wbytes, st));
  const int items = ytiles * nch * nt * 4;
  k_tc_split_w<<<std::max(1, std::min(4 * nsm, (items + 255) / 256)), 256, 0, st>>>(w, ldw, wscale, alpha, m, n, nt,
                                                                                 nch, ytiles, wsl);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    const int rowtiles = (k + kM - 1) / kM;
    const int gx = std::max(1, std::min(rowtiles, nsm / ytiles));
    NNArgs p;
    p.k = k;
    p.m = m;
    p.n = n;
    p.nt = nt;
    p.ldo = ldo;
    p.sw = sw;
    p.nstg = nstg;
    p.nob = nob;
    p.nhi = 5 * sw <= 512 ? 3 : 2;
    p.wsl = wsl;
    p.out = out;
    p.beta = (float)beta;
    if (nob)
      k_tc_gemm_nn<true><<<dim3(gx, ytiles), NN_THREADS, smem, st>>>(map, mout, p);
    else
      k_tc_gemm_nn<false><<<dim3(gx, ytiles), NN_THREADS, smem, st>>>(map, mout, p);
    e = cudaGetLastError();
  }
  cudaFreeAsync(wsl, st);
  if (e != cudaSuccess) return fail(DKS_ERR_CUDA, std::string("tensor-core OUT = A W launch: ") + cudaGetErrorString(e));
  return DKS_OK;
}

bool tc_hn_supported(const float2* a, int lda, const float2* b, int ldb, int k) {
  return k > 0 && tc::aligned_for_tma(a, lda) && tc::aligned_for_tma(b, ldb);
}

// C = A^H [B1 | B2] over k rows on the tensor cores.  gram: A = Z (m columns), B1 = HZ, B2 = Z,
// lower triangles of c1 = Z^H HZ and c2 = Z^H Z (m x m, ldc = m).  Otherwise B2 is absent and
// c1 (ldc) receives A^H B1 (mode 0) or its conjugate transpose B1^H A (mode 1).
int tc_gemm_hn_impl(const float2* a, int lda, int m, const float2* b1, const float2* b2, int ldb, int n, int k,
                    double2* c1, double2* c2, int ldc, int mode, bool gram, cudaStream_t st, int nsm) {
  using namespace tc;
  if (k <= 0 || m <= 0 || n <= 0) return DKS_OK;
  std::vector<HNTile> tiles;
  const int mt = (m + kM - 1) / kM;
  // A of at most 64 columns (the projector table): A and i A share the MMA's 128 rows
  const bool packed = !gram && m <= 64;
  const int tcols = packed ? HN_NBP : HN_NB;
  if (gram) {
    // block (ib, jb), jb <= ib, of 128 rows: HZ columns of block jb through B1, then Z columns
    // through B2, each in pieces of at most 64
    for (int ib = 0; ib < mt; ++ib)
      for (int jb = 0; jb <= ib; ++jb) {
        const int nbj = std::min(kM, m - jb * kM);
        const int pieces = (nbj + HN_NB - 1) / HN_NB, per = (nbj + pieces - 1) / pieces;
        for (int j0 = 0; j0 < nbj; j0 += per) tiles.push_back(HNTile{ib * kM, jb * kM + j0, std::min(per, nbj - j0), 0, 0});
        for (int j0 = 0; j0 < nbj; j0 += per) tiles.push_back(HNTile{ib * kM, 0, 0, jb * kM + j0, std::min(per, nbj - j0)});
      }
  } else {
    const int cap = packed ? HN_NBP : HN_NB;
    const int pieces = (n + cap - 1) / cap, per = (n + pieces - 1) / pieces;
    for (int ib = 0; ib < mt; ++ib)
      for (int j0 = 0; j0 < n; j0 += per) tiles.push_back(HNTile{ib * kM, j0, std::min(per, n - j0), 0, 0});
  }
  const int nt = (int)tiles.size();
  if (nt > kMaxTiles) return fail(DKS_ERR_UNSUPPORTED, "tensor-core A^H B: too many tiles");
  int kchunk;
  {
    std::lock_guard<std::mutex> g(g_mu);
    kchunk = g_kchunk;
    if (!g_attr_hn) {
      DKS_CUDA_TRY(cudaFuncSetAttribute((const void*)k_tc_gemm_hn<false>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)NN_SMEM_LIMIT));
      DKS_CUDA_TRY(cudaFuncSetAttribute((const void*)k_tc_gemm_hn<true>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)NN_SMEM_LIMIT));
      g_attr_hn = true;
    }
  }
  // splits: each K range at most kchunk rows, rounded up to whole waves of one CTA per SM, and
  // the partial tiles (64 KB per CTA) held to kPartBudget (longer ranges beyond that)
  constexpr size_t kPartBudget = 256u << 20;
  const size_t tile_bytes = (size_t)tcols * kM * sizeof(float2);
  long long splits = (k + kchunk - 1) / kchunk;
  const long long waves = (splits * nt + nsm - 1) / nsm;
  splits = std::max(splits, waves * nsm / nt);
  splits = std::max(1LL, std::min(splits, (long long)(kPartBudget / (tile_bytes * nt))));
  const int kc = (int)(((k + splits - 1) / splits + HN_KT - 1) / HN_KT * HN_KT);
  splits = (k + kc - 1) / kc;
  // TMA boxes cover only the columns a tile can use: a narrow A (the 36 projector channels) or
  // narrow B pieces fetch fewer 64-byte rows per stage
  const int boxa = std::min(kM, (m + 7) & ~7);
  int boxb = 8;
  for (const HNTile& t : tiles) boxb = std::max(boxb, (std::max(t.nb1, t.nb2) + 7) & ~7);
  boxb = std::min(boxb, tcols);
  CUtensorMap ta, tb1, tb2;
  DKS_TRY(make_map(&ta, a, k, m, lda, HN_KR, boxa));
  DKS_TRY(make_map(&tb1, b1, k, gram ? m : n, ldb, HN_KR, boxb));
  DKS_TRY(make_map(&tb2, b2 ? b2 : b1, k, gram ? m : n, ldb, HN_KR, boxb));
  const size_t part_bytes = (size_t)splits * nt * tile_bytes;
  // short tile lists travel in the kernel arguments; longer ones are copied to the device
  const bool copy_tiles = nt > kArgTiles;
  const size_t tl_bytes = copy_tiles ? (tiles.size() * sizeof(HNTile) + 255) / 256 * 256 : 0;
  unsigned char* buf = nullptr;
  DKS_CUDA_TRY(cudaMallocAsync((void**)&buf, tl_bytes + part_bytes, st));
  HNTile* dtiles = copy_tiles ? reinterpret_cast<HNTile*>(buf) : nullptr;
  float2* part = reinterpret_cast<float2*>(buf + tl_bytes);
  cudaError_t e = cudaSuccess;
  if (copy_tiles)
    e = cudaMemcpyAsync(dtiles, tiles.data(), tiles.size() * sizeof(HNTile), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    const int nstg = (int)std::min<size_t>(HN_STG_MAX, (NN_SMEM_LIMIT - HN_SMEM_FIXED) / HN_STG_BYTES);
    HNArgs p{};
    p.m = m;
    p.boxa = boxa;
    p.boxb = boxb;
    p.tcols = tcols;
    p.k = k;
    p.kchunk = kc;
    p.ntiles = nt;
    p.nstg = nstg;
    p.tile = dtiles;
    for (int i = 0; i < nt && i < kArgTiles; ++i) p.tv[i] = tiles[i];
    p.part = part;
    const size_t smem = HN_SMEM_FIXED + (size_t)nstg * HN_STG_BYTES;
    if (packed)
      k_tc_gemm_hn<true><<<dim3(nt, (unsigned)splits), HN_THREADS, smem, st>>>(ta, tb1, tb2, p);
    else
      k_tc_gemm_hn<false><<<dim3(nt, (unsigned)splits), HN_THREADS, smem, st>>>(ta, tb1, tb2, p);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    RedArgs r{};
    r.splits = (int)splits;
    r.ntiles = nt;
    r.m = m;
    r.ldc = ldc;
    r.mode = mode;
    r.gram = gram ? 1 : 0;
    r.tcols = tcols;
    r.tile = dtiles;
    for (int i = 0; i < nt && i < kArgTiles; ++i) r.tv[i] = tiles[i];
    r.part = part;
    r.c1 = c1;
    r.c2 = c2;
    k_tc_reduce<<<dim3(tcols * 4, nt), 256, 0, st>>>(r);
    e = cudaGetLastError();
  }
  cudaFreeAsync(buf, st);
  if (e != cudaSuccess) return fail(DKS_ERR_CUDA, std::string("tensor-core A^H B launch: ") + cudaGetErrorString(e));
  return DKS_OK;
}

int tc_gram(const float2* z, const float2* hz, int ld, int k, int m, double2* a, double2* s, cudaStream_t st, int nsm) {
  Prof pr(P_GRAM + kProf32, st, 2.0 * m * 8.0 * k + 32.0 * m * m, 8.0 * m * (m + 1.0) * (double)k);
  pr.count(1);
  return tc_gemm_hn_impl(z, ld, m, hz, z, ld, m, k, a, s, m, 0, true, st, nsm);
}

int tc_gemm_hn(const float2* a, int lda, const float2* b, int ldb, int k, int m, int n, double2* c, int ldc,
               bool conj_transpose_out, cudaStream_t st, int nsm) {
  return tc_gemm_hn_impl(a, lda, m, b, nullptr, ldb, n, k, c, nullptr, ldc, conj_transpose_out ? 1 : 0, false, st,
                         nsm);
}

}  // namespace dks

// Algorithm 1 (LOBPCG-F) driver on the device.
//
// Per k-point the blocks Z = [X | Y | P] and HZ = [HX | HY | HP] live in two
// ping-pong column buffers of capacity 3n columns (n = nev + nbuf), each column
// ncomp npw complex values.  One iteration:
//   Y  = K(x_G) (HX - X Lambda) on the active columns           (preconditioned residual)
//   Y  = f(H) Y      two H' passes with shift C and scale 1/Omega (filter)
//   HY = H' Y                                                     (one H' pass)
//   A = Z^H HZ, S = Z^H Z, FP64 Rayleigh-Ritz, first n pairs      (Rayleigh-Ritz)
//   X, HX <- Z V, HZ V into the other buffer                       (rotation)
//   (emulated FP64: Z and HZ are split into double-float copies once, before the Gram matrices,
//    and the Gram and rotation kernels read the copies)
//   column norms of HX - X Lambda (FP64), host reads them          (convergence test)
//   P, HP <- [0, Y, P] V_active, HZ likewise                        (soft locking, new P)
// so H' is applied 3 times per active column per iteration (Sec. 3.2).
//
// DKS_MODE_MIXED runs the same loop with complex64 blocks (FP32 H', Gram and
// rotations; FP64 small problem and norms) until the largest residual drops
// below refine_tol or stops improving, then restarts Algorithm 1 in FP64 from
// that X with N_init = 1 -- the paper's warm start (Sec. 3.1: N_init = 1 when X0
// is a previous solution), which also removes the negative-band noise that FP32
// rounding leaves in X.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "dks_internal.h"

namespace dks {

template <typename V>
struct Blocks {
  V* z[2];
  V* hz[2];
  V* tmp;
  // double-float copies of Z and HZ (emulated-FP64 phase): split once per iteration, read by
  // the Gram matrices and all four rotations
  float4* zdf = nullptr;
  float4* hzdf = nullptr;
  // or exact integer slices of Z and HZ for the tensor cores (DKS_TC_FP64): split once per
  // iteration, read by the Gram matrices and all four rotations
  void* ozz = nullptr;
  void* ozh = nullptr;
  int ozcols = 0;      // column capacity of the slice buffers
  // FP32 phase: copy of the X with the lowest residual so far (the FP64 phase starts from it)
  V* best = nullptr;
};

struct Small {
  double2* a;
  double2* s;
  double2* vm;
  double2* vp;
  double* lam;
  double* stats;
  int* act;
  int* info;
  double2* rrs;
};

struct PhaseOut {
  int iterations = 0;
  bool converged = false;
  double max_res = 0;
  long long happ = 0;
  bool neg = false;
  int cur = 0;
};

struct Pinned {
  double* lam = nullptr;
  double* stats = nullptr;
  int* act = nullptr;
  int* info = nullptr;
  int n = 0;
  ~Pinned() {
    if (lam) cudaFreeHost(lam);
    if (stats) cudaFreeHost(stats);
    if (act) cudaFreeHost(act);
    if (info) cudaFreeHost(info);
  }
  int alloc(int nn) {
    n = nn;
    DKS_CUDA_TRY(cudaMallocHost((void**)&lam, nn * sizeof(double)));
    DKS_CUDA_TRY(cudaMallocHost((void**)&stats, 3 * nn * sizeof(double)));
    DKS_CUDA_TRY(cudaMallocHost((void**)&act, nn * sizeof(int)));
    DKS_CUDA_TRY(cudaMallocHost((void**)&info, 4 * sizeof(int)));
    return DKS_OK;
  }
};

template <typename V>
static int filter_inplace(dks_ctx* ctx, Exec& ex, int ik, V* y, V* tmp, int nb, double C, double om,
                          cudaStream_t st) {
  DKS_TRY(apply_h<V>(ctx, ex, ik, y, tmp, nb, C, 1.0 / om, st));
  return apply_h<V>(ctx, ex, ik, tmp, y, nb, C, 1.0 / om, st);
}

// contractions of one phase: native arithmetic of V, or double-float for complex128 blocks
template <typename V>
static int hn(bool df, const V* a, int lda, const V* b, int ldb, int k, int m, int n, double2* c, cudaStream_t st,
              bool lower) {
  if (df) return gemm_hn_df((const double2*)a, lda, (const double2*)b, ldb, k, m, n, c, st, P_GRAM, 0, lower);
  return gemm_hn<V>(a, lda, b, ldb, k, m, n, c, st, P_GRAM, 0, lower);
}
template <typename V>
static int nn(bool df, const V* a, int lda, int k, int m, const double2* w, int ldw, int n, V* out, int ldo,
              cudaStream_t st) {
  if (df) return gemm_nn_df((const double2*)a, lda, k, m, w, ldw, nullptr, n, (double2*)out, ldo, 0.0, st);
  return gemm_nn<V>(a, lda, k, m, w, ldw, nullptr, n, out, ldo, 0.0, st);
}

// Y <- Y - Q (Q^H Y), twice (classical Gram-Schmidt with one reorthogonalisation): the locked
// vectors Q (nq columns) of earlier band blocks leave the span of the ncol columns of Y.  coef
// holds nq x ncol complex128 coefficients.
template <typename V>
static int project_out(const V* q, int nq, V* y, int ncol, int rows, double2* coef, bool df, cudaStream_t st) {
  if (!q || nq <= 0 || ncol <= 0) return DKS_OK;
  for (int pass = 0; pass < 2; ++pass) {
    DKS_CUDA_TRY(cudaMemsetAsync(coef, 0, (size_t)nq * ncol * sizeof(double2), st));
    DKS_TRY(hn<V>(df, q, rows, y, rows, rows, nq, ncol, coef, st, false));
    if (df)
      DKS_TRY(gemm_nn_df((const double2*)q, rows, rows, nq, coef, nq, nullptr, ncol, (double2*)y, rows, 1.0, st, -1.0));
    else
      DKS_TRY(gemm_nn<V>(q, rows, rows, nq, coef, nq, nullptr, ncol, y, rows, 1.0, st, -1.0));
  }
  return DKS_OK;
}

template <typename V>
static int gram(const V* z, const V* hz, int rows, int nz, Small& sm, cudaStream_t st, bool df = false) {
  DKS_CUDA_TRY(cudaMemsetAsync(sm.a, 0, (size_t)nz * nz * sizeof(double2), st));
  DKS_CUDA_TRY(cudaMemsetAsync(sm.s, 0, (size_t)nz * nz * sizeof(double2), st));
  if constexpr (std::is_same<V, float2>::value) {
    DKS_TRY(gram_f32(z, hz, rows, rows, nz, sm.a, sm.s, st));
  } else {
    DKS_TRY(hn<V>(df, z, rows, hz, rows, rows, nz, nz, sm.a, st, true));
    DKS_TRY(hn<V>(df, z, rows, z, rows, rows, nz, nz, sm.s, st, true));
  }
  DKS_TRY(mirror_lower(sm.a, nz, st));
  return mirror_lower(sm.s, nz, st);
}
// the same from double-float copies of Z and HZ
static int gram_split(const float4* z, const float4* hz, int rows, int nz, Small& sm, cudaStream_t st) {
  DKS_CUDA_TRY(cudaMemsetAsync(sm.a, 0, (size_t)nz * nz * sizeof(double2), st));
  DKS_CUDA_TRY(cudaMemsetAsync(sm.s, 0, (size_t)nz * nz * sizeof(double2), st));
  DKS_TRY(gram_df(z, hz, rows, rows, nz, sm.a, sm.s, st));
  DKS_TRY(mirror_lower(sm.a, nz, st));
  return mirror_lower(sm.s, nz, st);
}

// reads lam and residual statistics of the n columns; returns the host residual norms
static int fetch(Small& sm, Pinned& pin, int n, std::vector<double>& res, cudaStream_t st) {
  DKS_CUDA_TRY(cudaMemcpyAsync(pin.lam, sm.lam, n * sizeof(double), cudaMemcpyDeviceToHost, st));
  DKS_CUDA_TRY(cudaMemcpyAsync(pin.stats, sm.stats, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, st));
  DKS_CUDA_TRY(cudaMemcpyAsync(pin.info, sm.info, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
  DKS_CUDA_TRY(cudaStreamSynchronize(st));
  res.resize(n);
  for (int j = 0; j < n; ++j) res[j] = std::sqrt(pin.stats[3 * j] / std::max(pin.stats[3 * j + 1], 1e-300));
  return DKS_OK;
}

template <typename V>
static int phase(dks_ctx* ctx, Exec& ex, int ik, Blocks<V>& b, Small& sm, Pinned& pin, int n, int nconv, double tol,
                 int n_init, int n_iter, double C, double om, int precond, int use_filter, bool stop_on_stall,
                 double chol_tol, double drop_tol, std::vector<double>* hist, PhaseOut& out, cudaStream_t st,
                 bool df = false, const V* q = nullptr, int nq = 0, double2* coef = nullptr) {
  // q: nq locked vectors of earlier band blocks (deflation), projected out of the filtered start
  // block and of every filtered correction Y
  df = df && sizeof(V) == sizeof(double2);
  NvtxRange nvtx(sizeof(V) == sizeof(float2) ? "LOBPCG-F FP32 phase" : df ? "LOBPCG-F FP64 phase (double-float)"
                                                                         : "LOBPCG-F FP64 phase");
  ex.df_gemm = df;   // projector contractions inside apply_h follow the phase's arithmetic
  const KPoint& kp = ctx->k[ik];
  const int nc = ctx->ncomp;
  const int rows = nc * kp.npw;
  const size_t colsz = (size_t)rows;
  int cur = out.cur;
  long long happ = 0;
  // initial filtering
  if (use_filter)
    for (int i = 0; i < n_init; ++i) {
      DKS_TRY(filter_inplace<V>(ctx, ex, ik, b.z[cur], b.tmp, n, C, om, st));
      happ += 2LL * n;
    }
  DKS_TRY(project_out<V>(q, nq, b.z[cur], n, rows, coef, df, st));
  // first Rayleigh-Ritz on X0
  DKS_TRY(apply_h<V>(ctx, ex, ik, b.z[cur], b.hz[cur], n, 0.0, 1.0, st));
  happ += n;
  // Gram matrices and rotations of nz columns of Z, HZ (from double-float copies when present)
  const bool slices = df && b.ozz && b.ozh;
  const bool split = df && !slices && b.zdf && b.hzdf;
  OzBlock ozz, ozh;
  if (slices) {
    DKS_TRY(oz_layout(b.ozz, rows, b.ozcols, &ozz));
    DKS_TRY(oz_layout(b.ozh, rows, b.ozcols, &ozh));
  }
  auto gram_z = [&](int nzc) -> int {
    if (slices) {
      DKS_TRY(oz_split((const double2*)b.z[cur], rows, nzc, ozz, st));
      DKS_TRY(oz_split((const double2*)b.hz[cur], rows, nzc, ozh, st));
      DKS_TRY(oz_gram(ozz, ozh, nzc, sm.a, sm.s, st));
      DKS_TRY(mirror_lower(sm.a, nzc, st));
      return mirror_lower(sm.s, nzc, st);
    }
    if (!split) return gram<V>(b.z[cur], b.hz[cur], rows, nzc, sm, st, df);
    DKS_TRY(split_df((const double2*)b.z[cur], b.zdf, (size_t)nzc * colsz, st));
    DKS_TRY(split_df((const double2*)b.hz[cur], b.hzdf, (size_t)nzc * colsz, st));
    return gram_split(b.zdf, b.hzdf, rows, nzc, sm, st);
  };
  // out <- Z[c0:c0+m] W (h: from HZ instead of Z)
  auto rotate = [&](bool h, size_t c0, int m, const double2* w, int ldw, int ncol, V* outp) -> int {
    if (slices) return oz_rotate(h ? ozh : ozz, (int)c0, m, w, ldw, ncol, (double2*)outp, rows, 0.0, st);
    if (split)
      return gemm_nn_df((h ? b.hzdf : b.zdf) + c0 * colsz, rows, rows, m, w, ldw, nullptr, ncol, (double2*)outp,
                        rows, 0.0, st);
    return nn<V>(df, (h ? b.hz[cur] : b.z[cur]) + c0 * colsz, rows, rows, m, w, ldw, ncol, outp, rows, st);
  };
  DKS_TRY(gram_z(n));
  DKS_TRY(rayleigh_ritz(sm.a, sm.s, n, n, sm.vm, sm.lam, sm.info, sm.rrs, st, chol_tol, drop_tol));
  int nx = cur ^ 1;
  DKS_TRY(rotate(false, 0, n, sm.vm, n, n, b.z[nx]));
  DKS_TRY(rotate(true, 0, n, sm.vm, n, n, b.hz[nx]));
  cur = nx;
  DKS_TRY(col_stats<V>(b.z[cur], b.hz[cur], sm.lam, kp.ek, kp.npw, n, sm.stats, st, nc));
  std::vector<double> res;
  DKS_TRY(fetch(sm, pin, n, res, st));
  if (pin.info[1] < n) return fail(DKS_ERR_RANK, "initial block is rank deficient");
  std::vector<int> act;
  for (int j = 0; j < n; ++j) act.push_back(j);   // the first preconditioning uses every column of R
  int p = 0;
  double best = INFINITY, lowest = INFINITY;
  int since_best = 0;
  bool converged = false;
  int it = 0;
  double maxres = 0;
  // device copy of the active list; refreshed after every soft-locking step below
  std::memcpy(pin.act, act.data(), act.size() * sizeof(int));
  DKS_CUDA_TRY(cudaMemcpyAsync(sm.act, pin.act, act.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  for (it = 1; it <= n_iter; ++it) {
    const int a = (int)act.size();
    V* y = b.z[cur] + (size_t)n * colsz;
    V* hy = b.hz[cur] + (size_t)n * colsz;
    DKS_TRY(precond_apply<V>(b.z[cur], b.hz[cur], sm.lam, sm.stats, sm.act, a, kp.ek, kp.npw, precond, y, st, nc));
    if (use_filter) {
      DKS_TRY(filter_inplace<V>(ctx, ex, ik, y, b.tmp, a, C, om, st));
      happ += 2LL * a;
    }
    DKS_TRY(project_out<V>(q, nq, y, a, rows, coef, df, st));
    DKS_TRY(apply_h<V>(ctx, ex, ik, y, hy, a, 0.0, 1.0, st));
    happ += a;
    const int nz = n + a + p;
    DKS_TRY(gram_z(nz));
    DKS_TRY(rayleigh_ritz(sm.a, sm.s, nz, n, sm.vm, sm.lam, sm.info, sm.rrs, st, chol_tol, drop_tol));
    nx = cur ^ 1;
    DKS_TRY(rotate(false, 0, nz, sm.vm, nz, n, b.z[nx]));
    DKS_TRY(rotate(true, 0, nz, sm.vm, nz, n, b.hz[nx]));
    DKS_TRY(col_stats<V>(b.z[nx], b.hz[nx], sm.lam, kp.ek, kp.npw, n, sm.stats, st, nc));
    DKS_TRY(fetch(sm, pin, n, res, st));
    if (pin.info[1] < n) return fail(DKS_ERR_RANK, "Rayleigh-Ritz subspace rank below the block size");
    maxres = 0;
    for (int j = 0; j < nconv; ++j) maxres = std::max(maxres, res[j]);
    if (hist) hist->push_back(maxres);
    if (!std::isfinite(maxres)) return fail(DKS_ERR_NOT_CONVERGED, "non-finite residual norm");
    if (maxres < tol) {
      cur = nx;
      converged = true;
      break;
    }
    if (stop_on_stall) {
      // FP32 phase: stop at its rounding floor -- the best residual not lowered by 20% within 3
      // iterations (5 while it is still above 30 tol: FP32 rounding can stall it there for a
      // few iterations before it improves again) -- or on a rise above 10x the best (FP32 noise
      // reaching the negative band).
      // Smaller rises are transient and recover; the phase hands on the X with the lowest
      // residual seen, not the last one.
      if (b.best && maxres < lowest) {
        lowest = maxres;
        DKS_CUDA_TRY(cudaMemcpyAsync(b.best, b.z[nx], (size_t)n * colsz * sizeof(V), cudaMemcpyDeviceToDevice, st));
      }
      if (maxres < 0.8 * best) {
        best = maxres;
        since_best = 0;
      } else if (++since_best >= (best > 30.0 * tol ? 5 : 3) || maxres > 10.0 * best) {
        cur = nx;
        if (b.best)
          DKS_CUDA_TRY(cudaMemcpyAsync(b.z[cur], b.best, (size_t)n * colsz * sizeof(V), cudaMemcpyDeviceToDevice,
                                       st));
        break;
      }
    }
    // soft locking, P <- [0, Y, P] V_active
    std::vector<int> act2;
    for (int j = 0; j < n; ++j)
      if (res[j] > tol) act2.push_back(j);
    const int a2 = (int)act2.size();
    std::memcpy(pin.act, act2.data(), a2 * sizeof(int));
    DKS_CUDA_TRY(cudaMemcpyAsync(sm.act, pin.act, a2 * sizeof(int), cudaMemcpyHostToDevice, st));
    DKS_TRY(gather_cols(sm.vm, nz, n, nz - n, sm.act, a2, sm.vp, st));
    V* pz = b.z[nx] + (size_t)(n + a2) * colsz;
    V* phz = b.hz[nx] + (size_t)(n + a2) * colsz;
    DKS_TRY(rotate(false, (size_t)n, nz - n, sm.vp, nz - n, a2, pz));
    DKS_TRY(rotate(true, (size_t)n, nz - n, sm.vp, nz - n, a2, phz));
    // the Teter factor of the next iteration needs statistics of the new X (already in sm.stats)
    cur = nx;
    act.swap(act2);
    p = a2;
  }
  out.iterations = std::min(it, n_iter);
  out.converged = converged;
  out.max_res = maxres;
  out.happ = happ;
  out.cur = cur;
  out.neg = pin.lam[0] < -ctx->c * ctx->c;
  ex.df_gemm = false;
  return DKS_OK;
}


// ---------------------------------------------------------------- Davidson-F
// Block Davidson with the filter of Algorithm 1 (the paper notes that its filter step carries
// over to Davidson-type solvers, Sec. 3): a growing orthonormal basis V replaces [X, Y, P].
// Per iteration: Rayleigh-Ritz on V, X = V C, R = HX - X Theta, T = f(H) K(R) on the active
// columns, restart V = X when V would exceed mmax columns, T projected out of V twice
// (classical Gram-Schmidt with one reorthogonalisation), T orthonormalised through the
// Rayleigh-Ritz kernel on the pencil (T^H T, T^H T) (Cholesky, or SVQB when T is rank
// deficient), then V = [V, T], HV = [HV, H T].
template <typename V>
struct DBlocks {
  V* v = nullptr;      // mmax columns
  V* hv = nullptr;     // mmax columns
  V* x = nullptr;      // n columns: X0 on entry, X on exit
  V* hx = nullptr;
  V* t = nullptr;      // n columns: the new directions
  V* tmp = nullptr;    // n columns: filter intermediate
  V* best = nullptr;   // FP32 phase: X with the lowest residual
};

template <typename V>
static int davidson_phase(dks_ctx* ctx, Exec& ex, int ik, DBlocks<V>& b, Small& sm, Pinned& pin, int n,
                          int nconv, double tol, int n_init, int n_iter, double C, double om, int precond,
                          int use_filter, bool stop_on_stall, double chol_tol, double drop_tol,
                          std::vector<double>* hist, PhaseOut& out, cudaStream_t st, bool df, int mmax) {
  df = df && sizeof(V) == sizeof(double2);
  ex.df_gemm = df;
  const KPoint& kp = ctx->k[ik];
  const int nc = ctx->ncomp;
  const int rows = nc * kp.npw;
  const size_t colsz = (size_t)rows;
  long long happ = 0;
  auto hn_full = [&](const V* a, int m, const V* bb, int nn, double2* c, bool lower) -> int {
    DKS_CUDA_TRY(cudaMemsetAsync(c, 0, (size_t)m * nn * sizeof(double2), st));
    return hn<V>(df, a, rows, bb, rows, rows, m, nn, c, st, lower);
  };
  auto nn_into = [&](const V* a, int m, const double2* w, int ldw, int ncol, V* o, double beta,
                     double alpha) -> int {
    if (df)
      return gemm_nn_df((const double2*)a, rows, rows, m, w, ldw, nullptr, ncol, (double2*)o, rows, beta, st,
                        alpha);
    return gemm_nn<V>(a, rows, rows, m, w, ldw, nullptr, ncol, o, rows, beta, st, alpha);
  };
  // an orthonormal basis of the nt columns of t, written to dst; returns its width (rank).  With
  // FP32 blocks the Gram matrix carries ~1e-7 relative rounding, so directions whose scaled
  // Cholesky pivot or Gram eigenvalue is below 1e-6 are treated as dependent (SVQB drops them).
  const double otol_c = sizeof(V) == sizeof(double2) ? chol_tol : std::max(chol_tol, 1e-6);
  const double otol_d = sizeof(V) == sizeof(double2) ? drop_tol : std::max(drop_tol, 1e-6);
  // The basis comes from the generalized eigenvectors of (diag(1, ..., nt), G), G = T^H T: they
  // are G-orthonormal, so T times them is orthonormal; the distinct diagonal keeps the small
  // eigenproblem free of one large degenerate cluster (the pencil (G, G) would have nt equal
  // eigenvalues).
  auto orthonormalise = [&](const V* t, int nt, V* dst, int& rank) -> int {
    DKS_TRY(hn_full(t, nt, t, nt, sm.s, true));
    DKS_TRY(mirror_lower(sm.s, nt, st));
    DKS_TRY(set_diag_ramp(sm.a, nt, st));
    DKS_TRY(rayleigh_ritz(sm.a, sm.s, nt, nt, sm.vm, sm.lam, sm.info, sm.rrs, st, otol_c, otol_d));
    DKS_CUDA_TRY(cudaMemcpyAsync(pin.info, sm.info, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    DKS_CUDA_TRY(cudaStreamSynchronize(st));
    rank = std::min(nt, pin.info[1]);
    if (rank < nt && rank > 0)   // the first rank pairs of the reduced problem
      DKS_TRY(rayleigh_ritz(sm.a, sm.s, nt, rank, sm.vm, sm.lam, sm.info, sm.rrs, st, otol_c, otol_d));
    if (rank > 0) DKS_TRY(nn_into(t, nt, sm.vm, nt, rank, dst, 0.0, 1.0));
    return DKS_OK;
  };
  // initial filtering of Algorithm 1
  if (use_filter)
    for (int i = 0; i < n_init; ++i) {
      DKS_TRY(filter_inplace<V>(ctx, ex, ik, b.x, b.tmp, n, C, om, st));
      happ += 2LL * n;
    }
  int k = 0;
  DKS_TRY(orthonormalise(b.x, n, b.v, k));
  if (k < n)
    return fail(DKS_ERR_RANK, std::string("Davidson: initial block is rank deficient (") +
                                  (sizeof(V) == sizeof(double2) ? "FP64" : "FP32") + " phase, rank " +
                                  std::to_string(k) + " of " + std::to_string(n) + ")");
  DKS_TRY(apply_h<V>(ctx, ex, ik, b.v, b.hv, n, 0.0, 1.0, st));
  happ += n;
  std::vector<double> res;
  std::vector<int> act;
  double best = INFINITY, lowest = INFINITY, maxres = 0;
  int since_best = 0, it = 0;
  bool converged = false;
  for (it = 1; it <= n_iter; ++it) {
    DKS_TRY(gram<V>(b.v, b.hv, rows, k, sm, st, df));
    DKS_TRY(rayleigh_ritz(sm.a, sm.s, k, n, sm.vm, sm.lam, sm.info, sm.rrs, st, chol_tol, drop_tol));
    // A basis whose Gram matrix needed SVQB (Cholesky pivot below chol_tol) or lost rank has
    // drifted from orthonormal (rounding in the projections, most of all with FP32 blocks):
    // restart it from the current Ritz vectors (X, HX of the previous iteration) instead.
    DKS_CUDA_TRY(cudaMemcpyAsync(pin.info, sm.info, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    DKS_CUDA_TRY(cudaStreamSynchronize(st));
    const bool conditioned = pin.info[0] == 0 && pin.info[1] >= n;
    if (!conditioned && k > n && it > 1) {
      DKS_CUDA_TRY(cudaMemcpyAsync(b.v, b.x, (size_t)n * colsz * sizeof(V), cudaMemcpyDeviceToDevice, st));
      DKS_CUDA_TRY(cudaMemcpyAsync(b.hv, b.hx, (size_t)n * colsz * sizeof(V), cudaMemcpyDeviceToDevice, st));
      k = n;
      continue;
    }
    DKS_TRY(nn_into(b.v, k, sm.vm, k, n, b.x, 0.0, 1.0));
    DKS_TRY(nn_into(b.hv, k, sm.vm, k, n, b.hx, 0.0, 1.0));
    DKS_TRY(col_stats<V>(b.x, b.hx, sm.lam, kp.ek, kp.npw, n, sm.stats, st, nc));
    DKS_TRY(fetch(sm, pin, n, res, st));
    if (pin.info[1] < n) {
      // FP32 phase: a basis that rounding has made numerically dependent ends the phase like a
      // stall, from the best X so far; in FP64 it is an error
      if (stop_on_stall && b.best && std::isfinite(lowest)) {
        DKS_CUDA_TRY(cudaMemcpyAsync(b.x, b.best, (size_t)n * colsz * sizeof(V), cudaMemcpyDeviceToDevice, st));
        break;
      }
      return fail(DKS_ERR_RANK, std::string("Davidson basis rank below the block size (") +
                                    (sizeof(V) == sizeof(double2) ? "FP64" : "FP32") + " phase, iteration " +
                                    std::to_string(it) + ", basis " + std::to_string(k) + ", rank " +
                                    std::to_string(pin.info[1]) + ", svqb " + std::to_string(pin.info[0]) + ")");
    }
    maxres = 0;
    for (int j = 0; j < nconv; ++j) maxres = std::max(maxres, res[j]);
    if (hist) hist->push_back(maxres);
    if (!std::isfinite(maxres)) return fail(DKS_ERR_NOT_CONVERGED, "non-finite residual norm");
    if (maxres < tol) {
      converged = true;
      break;
    }
    if (stop_on_stall) {   // the FP32 phase's floor, as in Algorithm 1's mixed mode
      if (b.best && maxres < lowest && conditioned) {   // hand on only X from a well-conditioned basis
        lowest = maxres;
        DKS_CUDA_TRY(cudaMemcpyAsync(b.best, b.x, (size_t)n * colsz * sizeof(V), cudaMemcpyDeviceToDevice, st));
      }
      if (maxres < 0.8 * best) {
        best = maxres;
        since_best = 0;
      } else if (++since_best >= (best > 30.0 * tol ? 5 : 3) || maxres > 10.0 * best) {
        if (b.best)
          DKS_CUDA_TRY(cudaMemcpyAsync(b.x, b.best, (size_t)n * colsz * sizeof(V), cudaMemcpyDeviceToDevice, st));
        break;
      }
    }
    act.clear();
    for (int j = 0; j < n; ++j)
      if (res[j] > tol) act.push_back(j);
    const int a = (int)act.size();
    std::memcpy(pin.act, act.data(), a * sizeof(int));
    DKS_CUDA_TRY(cudaMemcpyAsync(sm.act, pin.act, a * sizeof(int), cudaMemcpyHostToDevice, st));
    DKS_TRY(precond_apply<V>(b.x, b.hx, sm.lam, sm.stats, sm.act, a, kp.ek, kp.npw, precond, b.t, st, nc));
    if (use_filter) {
      DKS_TRY(filter_inplace<V>(ctx, ex, ik, b.t, b.tmp, a, C, om, st));
      happ += 2LL * a;
    }
    if (k + a > mmax) {   // restart from the Ritz vectors (orthonormal: V C with C^H V^H V C = I)
      DKS_CUDA_TRY(cudaMemcpyAsync(b.v, b.x, (size_t)n * colsz * sizeof(V), cudaMemcpyDeviceToDevice, st));
      DKS_CUDA_TRY(cudaMemcpyAsync(b.hv, b.hx, (size_t)n * colsz * sizeof(V), cudaMemcpyDeviceToDevice, st));
      k = n;
    }
    for (int pass = 0; pass < 2; ++pass) {   // T <- T - V (V^H T)
      DKS_TRY(hn_full(b.v, k, b.t, a, sm.vp, false));
      DKS_TRY(nn_into(b.v, k, sm.vp, k, a, b.t, 1.0, -1.0));
    }
    int r = 0;
    DKS_TRY(orthonormalise(b.t, a, b.v + (size_t)k * colsz, r));
    if (r == 0) return fail(DKS_ERR_NOT_CONVERGED, "Davidson: no new direction outside the basis");
    DKS_TRY(apply_h<V>(ctx, ex, ik, b.v + (size_t)k * colsz, b.hv + (size_t)k * colsz, r, 0.0, 1.0, st));
    happ += r;
    k += r;
  }
  out.iterations = std::min(it, n_iter);
  out.converged = converged;
  out.max_res = maxres;
  out.happ = happ;
  out.cur = 0;
  out.neg = pin.lam[0] < -ctx->c * ctx->c;
  ex.df_gemm = false;
  return DKS_OK;
}

}  // namespace dks

using namespace dks;

extern "C" {

void dks_solve_opts_default(dks_solve_opts* o) {
  if (!o) return;
  o->n_init = 3;
  o->n_iter = 200;
  o->nbuf = 0;
  o->C = NAN;
  o->Omega = NAN;
  o->mode = DKS_MODE_FP64;
  o->refine_tol = 1e-5;
  o->precond = DKS_PRECOND_TETER;
  o->use_filter = 1;
  o->nev_k = nullptr;
  o->stream = nullptr;
  o->chol_tol = 1e-12;
  o->drop_tol = 1e-12;
  o->emulate_fp64 = 1;
  o->concurrency = 0;
  o->solver = DKS_SOLVER_LOBPCG;
  o->m_max = 0;
  o->block = 0;
}

int dks_lobpcgf_solve(dks_ctx* ctx, int nev, double tol, const dks_solve_opts* opts_in, double* eig, void* const* X,
                      dks_solve_report* report) {
  auto t0 = std::chrono::steady_clock::now();
  dks_solve_opts opts;
  if (opts_in) opts = *opts_in;
  else dks_solve_opts_default(&opts);
  if (!ctx || !eig || !X || !(tol > 0) || opts.n_init < 0 || opts.n_iter < 0 || opts.nbuf < 0 ||
      opts.concurrency < 0 || (opts.mode != DKS_MODE_FP64 && opts.mode != DKS_MODE_MIXED) ||
      (opts.solver != DKS_SOLVER_LOBPCG && opts.solver != DKS_SOLVER_DAVIDSON) || opts.m_max < 0 ||
      opts.block < 0 || (opts.block > 0 && opts.solver != DKS_SOLVER_LOBPCG))
    return fail(DKS_ERR_INVALID_ARG, "dks_lobpcgf_solve: bad argument");
  const bool davidson = opts.solver == DKS_SOLVER_DAVIDSON;
  cudaStream_t st = (cudaStream_t)opts.stream;
  // a KSSO operator has no negative continuum: Algorithm 1 without the filter (standard LOBPCG,
  // the solver of the paper's KSSO module)
  if (ctx->ncomp == 2) opts.use_filter = 0;
  if (report) {
    std::memset(report, 0, sizeof(*report));
    report->shift = ctx->ncomp == 4 ? ctx->c * ctx->c : 0.0;
  }
  int nmax = 0, rowsmax = 0, nlockmax = 0;
  std::vector<size_t> eoff(ctx->nk + 1, 0);
  for (int ik = 0; ik < ctx->nk; ++ik) {
    const int nv = opts.nev_k ? opts.nev_k[ik] : nev;
    if (nv <= 0 || !X[ik]) return fail(DKS_ERR_INVALID_ARG, "dks_lobpcgf_solve: nev_k and X[ik] required");
    // band blocks: the iterated width is block + nbuf; the locked vectors are the earlier blocks'
    const bool blocked = opts.block > 0 && nv > opts.block;
    const int n = (blocked ? opts.block : nv) + opts.nbuf;
    if (blocked) {
      nlockmax = std::max(nlockmax, nv);
      if (nv + opts.nbuf > ctx->k[ik].npw * ctx->ncomp) return fail(DKS_ERR_INVALID_ARG, "more pairs than the basis");
    }
    if (3 * n > kMaxRR) return fail(DKS_ERR_UNSUPPORTED, "block wider than the Rayleigh-Ritz limit (3n <= 512)");
    if (davidson) {
      const int mm = opts.m_max ? opts.m_max : std::min(4 * n, kMaxRR);
      if (mm < 2 * n || mm > kMaxRR)
        return fail(DKS_ERR_INVALID_ARG, "dks_lobpcgf_solve: need 2 (nev + nbuf) <= m_max <= 512");
    }
    if (n > ctx->k[ik].npw * ctx->ncomp) return fail(DKS_ERR_INVALID_ARG, "block wider than the basis");
    nmax = std::max(nmax, n);
    rowsmax = std::max(rowsmax, ctx->ncomp * ctx->k[ik].npw);
    eoff[ik + 1] = eoff[ik] + nv;
  }
  const bool mixed = opts.mode == DKS_MODE_MIXED;
  // Davidson: basis of mmax columns (V and HV) and four n-column blocks; LOBPCG: [X|Y|P] ping-pong
  const int mmax = davidson ? (opts.m_max ? opts.m_max : std::min(4 * nmax, kMaxRR)) : 0;
  const size_t cols = (size_t)3 * nmax;
  const size_t big64 = cols * rowsmax * sizeof(double2);
  const size_t big32 = mixed ? cols * rowsmax * sizeof(float2) : 0;
  const size_t tmp64 = (size_t)nmax * rowsmax * sizeof(double2);
  const size_t tmp32 = mixed ? (size_t)nmax * rowsmax * sizeof(float2) : 0;
  const size_t nz = davidson ? (size_t)std::max(mmax, 3 * nmax) : (size_t)3 * nmax;
  const size_t small = (2 * nz * nz + 2 * nz * nmax + rr_scratch_elems((int)nz)) * sizeof(double2) +
                       (nmax + 3 * nmax) * sizeof(double) + (nmax + 4) * sizeof(int) + 16 * 256;
  const bool split_copies = mixed && opts.emulate_fp64 != 0 && !davidson;
  // FP64-phase contractions on the tensor cores: exact integer slices instead of double-float copies
  const bool oz_slices = split_copies && tc_enabled(TC_FP64);
  const size_t ozb = oz_slices ? (oz_bytes(rowsmax, (int)cols) + 255) / 256 * 256 : 0;
  // band blocks: FP32 copy of the locked vectors (mixed mode) and the projection coefficients
  const size_t lock32 = mixed ? (size_t)nlockmax * rowsmax * sizeof(float2) : 0;
  const size_t lockcoef = (size_t)nlockmax * nmax * sizeof(double2);
  const size_t dcols64 = (size_t)2 * mmax + 4 * (size_t)nmax, dcols32 = mixed ? (size_t)2 * mmax + 5 * (size_t)nmax : 0;
  const size_t total =
      davidson ? (dcols64 * sizeof(double2) + dcols32 * sizeof(float2)) * rowsmax + small + 32 * 256
               : 4 * big64 + tmp64 + 4 * big32 + 2 * tmp32 + small + (split_copies ? (oz_slices ? 2 * ozb : 2 * big64) : 0) + lock32 +
                     lockcoef + 18 * 256;
  // concurrent k-point workers, each with its own stream and workspace (bounded by free memory)
  int nworkers = opts.concurrency > 0 ? opts.concurrency : std::min(ctx->nk, 4);
  nworkers = std::max(1, std::min(nworkers, ctx->nk));
  {
    size_t freeb = 0, totalb = 0;
    if (cudaMemGetInfo(&freeb, &totalb) == cudaSuccess) {
      const size_t per = total + (size_t)6 * 64 * 1024 * 1024;   // + H' intermediates
      while (nworkers > 1 && (size_t)nworkers * per > freeb * 8 / 10) --nworkers;
    }
  }
  if (nworkers > 1) DKS_CUDA_TRY(cudaStreamSynchronize(st));   // caller's pending work before ours
  while ((int)ctx->exec.size() < nworkers) ctx->exec.push_back(new Exec());
  for (int w = 0; w < nworkers; ++w) {
    DKS_TRY(grow(ctx->exec[w]->ws_solve, total));
    if (nworkers > 1 && !ctx->exec[w]->own)
      DKS_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->exec[w]->own, cudaStreamNonBlocking));
  }
  // k-points largest first (cost ~ block width x basis size)
  std::vector<int> order(ctx->nk);
  for (int ik = 0; ik < ctx->nk; ++ik) order[ik] = ik;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const double ca = (double)(opts.nev_k ? opts.nev_k[a] : nev) * ctx->k[a].npw;
    const double cb = (double)(opts.nev_k ? opts.nev_k[b] : nev) * ctx->k[b].npw;
    return ca > cb;
  });
  std::atomic<int> next{0};
  std::atomic<long long> happ{0};
  std::vector<int> krc(ctx->nk, DKS_OK);
  std::vector<std::string> kmsg(ctx->nk);
  std::vector<double> hist;
  std::vector<PhaseOut> o32s(ctx->nk), o64s(ctx->nk);
  auto worker = [&](int w) {
    cudaSetDevice(ctx->device);
    Exec& ex = *ctx->exec[w];
    cudaStream_t ws = nworkers > 1 ? ex.own : st;
    char* base = reinterpret_cast<char*>(ex.ws_solve.ptr);
    size_t off = 0;
    auto take = [&](size_t bytes) {
      void* p = base + off;
      off += (bytes + 255) / 256 * 256;
      return p;
    };
    Blocks<double2> b64{};
    Blocks<float2> b32{};
    DBlocks<double2> d64{};
    DBlocks<float2> d32{};
    if (davidson) {
      const size_t r = (size_t)rowsmax;
      d64.v = (double2*)take(mmax * r * sizeof(double2));
      d64.hv = (double2*)take(mmax * r * sizeof(double2));
      d64.x = (double2*)take(nmax * r * sizeof(double2));
      d64.hx = (double2*)take(nmax * r * sizeof(double2));
      d64.t = (double2*)take(nmax * r * sizeof(double2));
      d64.tmp = (double2*)take(nmax * r * sizeof(double2));
      if (mixed) {
        d32.v = (float2*)take(mmax * r * sizeof(float2));
        d32.hv = (float2*)take(mmax * r * sizeof(float2));
        d32.x = (float2*)take(nmax * r * sizeof(float2));
        d32.hx = (float2*)take(nmax * r * sizeof(float2));
        d32.t = (float2*)take(nmax * r * sizeof(float2));
        d32.tmp = (float2*)take(nmax * r * sizeof(float2));
        d32.best = (float2*)take(nmax * r * sizeof(float2));
      }
    } else {
      b64.z[0] = (double2*)take(big64);
      b64.z[1] = (double2*)take(big64);
      b64.hz[0] = (double2*)take(big64);
      b64.hz[1] = (double2*)take(big64);
      b64.tmp = (double2*)take(tmp64);
      if (oz_slices) {
        b64.ozz = take(ozb);
        b64.ozh = take(ozb);
        b64.ozcols = (int)cols;
      } else if (split_copies) {
        b64.zdf = (float4*)take(big64);
        b64.hzdf = (float4*)take(big64);
      }
      if (mixed) {
        b32.z[0] = (float2*)take(big32);
        b32.z[1] = (float2*)take(big32);
        b32.hz[0] = (float2*)take(big32);
        b32.hz[1] = (float2*)take(big32);
        b32.tmp = (float2*)take(tmp32);
        b32.best = (float2*)take(tmp32);
      }
    }
    float2* q32 = lock32 ? (float2*)take(lock32) : nullptr;
    double2* qcoef = lockcoef ? (double2*)take(lockcoef) : nullptr;
    Small sm;
    sm.a = (double2*)take(nz * nz * sizeof(double2));
    sm.s = (double2*)take(nz * nz * sizeof(double2));
    sm.vm = (double2*)take(nz * nmax * sizeof(double2));
    sm.vp = (double2*)take(nz * nmax * sizeof(double2));
    sm.rrs = (double2*)take(rr_scratch_elems((int)nz) * sizeof(double2));
    sm.lam = (double*)take(nmax * sizeof(double));
    sm.stats = (double*)take(3 * nmax * sizeof(double));
    sm.act = (int*)take(nmax * sizeof(int));
    sm.info = (int*)take(4 * sizeof(int));
    Pinned pin;
    if (pin.alloc(nmax) != DKS_OK) {
      const int t = next.fetch_add(ctx->nk);   // stop handing out work
      if (t < ctx->nk) {
        krc[order[t]] = DKS_ERR_OOM;
        kmsg[order[t]] = "pinned host buffer";
      }
      return;
    }
    for (int t = next.fetch_add(1); t < ctx->nk; t = next.fetch_add(1)) {
      const int ik = order[t];
      NvtxRange nvtx_k("k-point solve");
      auto run = [&]() -> int {
        const KPoint& kp = ctx->k[ik];
        const int nv = opts.nev_k ? opts.nev_k[ik] : nev;
        const int n = nv + opts.nbuf;
        const size_t elems = (size_t)n * ctx->ncomp * kp.npw;
        // a start block with a NaN or infinite entry cannot be iterated (every Gram matrix would
        // carry it): refuse it before any other work, naming the first such column
        for (int j0 = 0; j0 < n; j0 += nmax) {
          const int nc = std::min(nmax, n - j0);
          const double2* xs = (const double2*)X[ik] + (size_t)j0 * ctx->ncomp * kp.npw;
          DKS_TRY(col_stats<double2>(xs, xs, sm.lam, kp.ek, kp.npw, nc, sm.stats, ws, ctx->ncomp));
          DKS_CUDA_TRY(cudaMemcpyAsync(pin.stats, sm.stats, 3 * (size_t)nc * sizeof(double), cudaMemcpyDeviceToHost, ws));
          DKS_CUDA_TRY(cudaStreamSynchronize(ws));
          for (int j = 0; j < nc; ++j)
            if (!std::isfinite(pin.stats[3 * j + 1]))
              return fail(DKS_ERR_INVALID_ARG, "start block column " + std::to_string(j0 + j) + " of k-point " +
                                                   std::to_string(ik) + " is not finite");
        }
        const double C = std::isnan(opts.C) ? kp.cshift : opts.C;
        const double om = std::isnan(opts.Omega) ? kp.omega : opts.Omega;
        std::vector<double>* h = ik == 0 ? &hist : nullptr;
        PhaseOut& o32 = o32s[ik];
        PhaseOut& o64 = o64s[ik];
        if (davidson) {
          const bool emu = opts.emulate_fp64 != 0;
          if (mixed) {
            DKS_TRY(convert<double2, float2>((const double2*)X[ik], d32.x, elems, ws));
            DKS_TRY(davidson_phase<float2>(ctx, ex, ik, d32, sm, pin, n, nv, std::max(opts.refine_tol, tol),
                                           opts.n_init, opts.n_iter, C, om, opts.precond, opts.use_filter, true,
                                           opts.chol_tol, opts.drop_tol, h, o32, ws, false, mmax));
            DKS_TRY(convert<float2, double2>(d32.x, d64.x, elems, ws));
            const int left = std::max(0, opts.n_iter - o32.iterations);
            DKS_TRY(davidson_phase<double2>(ctx, ex, ik, d64, sm, pin, n, nv, tol, opts.use_filter ? 1 : 0, left, C,
                                            om, opts.precond, opts.use_filter, false, opts.chol_tol, opts.drop_tol,
                                            h, o64, ws, emu, mmax));
          } else {
            DKS_CUDA_TRY(cudaMemcpyAsync(d64.x, X[ik], elems * sizeof(double2), cudaMemcpyDeviceToDevice, ws));
            DKS_TRY(davidson_phase<double2>(ctx, ex, ik, d64, sm, pin, n, nv, tol, opts.n_init, opts.n_iter, C, om,
                                            opts.precond, opts.use_filter, false, opts.chol_tol, opts.drop_tol, h,
                                            o64, ws, false, mmax));
          }
          DKS_CUDA_TRY(cudaMemcpyAsync(X[ik], d64.x, elems * sizeof(double2), cudaMemcpyDeviceToDevice, ws));
          DKS_CUDA_TRY(cudaStreamSynchronize(ws));
          for (int j = 0; j < nv; ++j) eig[eoff[ik] + j] = pin.lam[j];
          happ += o32.happ + o64.happ;
          return DKS_OK;
        }
        if (opts.block > 0 && nv > opts.block) {
          // band blocks with deflation.  Block bi wants the pairs bi*blk .. bi*blk + nw - 1 and
          // iterates m = nw + nbuf columns.  Its start block: block 0 takes columns 0 .. m-1 of
          // X; block bi > 0 takes the previous block's nbuf buffer columns and then columns
          // nbuf + bi*blk .. nbuf + bi*blk + nw - 1 of X (not yet read by an earlier block).  The
          // converged wanted columns are written to X[bi*blk ..] (columns every earlier block has
          // already consumed) and serve as the locked vectors Q of the later blocks.
          const int blk = opts.block, nb = opts.nbuf;
          const size_t rows = (size_t)ctx->ncomp * kp.npw;
          double2* xk = (double2*)X[ik];
          const int nblk = (nv + blk - 1) / blk;
          int prev_nw = 0, prev_cur = 0;
          PhaseOut acc32, acc64;
          acc64.converged = true;
          for (int bi = 0; bi < nblk; ++bi) {
            const int nw = std::min(blk, nv - bi * blk);
            const int m = nw + nb;
            const int nq = bi * blk;
            const size_t me = (size_t)m * rows;
            const int sidx = bi == 0 ? 0 : (prev_cur ^ 1);
            double2* zs = b64.z[sidx];
            if (bi == 0) {
              DKS_CUDA_TRY(cudaMemcpyAsync(zs, xk, me * sizeof(double2), cudaMemcpyDeviceToDevice, ws));
            } else {
              if (nb)
                DKS_CUDA_TRY(cudaMemcpyAsync(zs, b64.z[prev_cur] + (size_t)prev_nw * rows, (size_t)nb * rows * sizeof(double2),
                                             cudaMemcpyDeviceToDevice, ws));
              DKS_CUDA_TRY(cudaMemcpyAsync(zs + (size_t)nb * rows, xk + (size_t)(nb + bi * blk) * rows,
                                           (size_t)nw * rows * sizeof(double2), cudaMemcpyDeviceToDevice, ws));
            }
            PhaseOut p32, p64;
            if (mixed) {
              DKS_TRY(convert<double2, float2>(zs, b32.z[0], me, ws));
              p32.cur = 0;
              DKS_TRY(phase<float2>(ctx, ex, ik, b32, sm, pin, m, nw, std::max(opts.refine_tol, tol), opts.n_init,
                                    opts.n_iter, C, om, opts.precond, opts.use_filter, true, opts.chol_tol,
                                    opts.drop_tol, h, p32, ws, false, q32, nq, qcoef));
              DKS_TRY(convert<float2, double2>(b32.z[p32.cur], b64.z[0], me, ws));
              p64.cur = 0;
              const int left = std::max(0, opts.n_iter - p32.iterations);
              DKS_TRY(phase<double2>(ctx, ex, ik, b64, sm, pin, m, nw, tol, opts.use_filter ? 1 : 0, left, C, om,
                                     opts.precond, opts.use_filter, false, opts.chol_tol, opts.drop_tol, h, p64, ws,
                                     opts.emulate_fp64 != 0, xk, nq, qcoef));
            } else {
              p64.cur = sidx;
              DKS_TRY(phase<double2>(ctx, ex, ik, b64, sm, pin, m, nw, tol, opts.n_init, opts.n_iter, C, om,
                                     opts.precond, opts.use_filter, false, opts.chol_tol, opts.drop_tol, h, p64, ws,
                                     false, xk, nq, qcoef));
            }
            // lock the wanted columns: X[nq .. nq + nw - 1], and their FP32 copy for later blocks
            DKS_CUDA_TRY(cudaMemcpyAsync(xk + (size_t)nq * rows, b64.z[p64.cur], (size_t)nw * rows * sizeof(double2),
                                         cudaMemcpyDeviceToDevice, ws));
            if (mixed)
              DKS_TRY(convert<double2, float2>(xk + (size_t)nq * rows, q32 + (size_t)nq * rows, (size_t)nw * rows, ws));
            DKS_CUDA_TRY(cudaStreamSynchronize(ws));
            for (int j = 0; j < nw; ++j) eig[eoff[ik] + nq + j] = pin.lam[j];
            acc32.iterations += p32.iterations;
            acc32.happ += p32.happ;
            acc64.iterations += p64.iterations;
            acc64.happ += p64.happ;
            acc64.converged = acc64.converged && p64.converged;
            acc64.max_res = std::max(acc64.max_res, p64.max_res);
            acc64.neg = acc64.neg || p64.neg;
            prev_nw = nw;
            prev_cur = p64.cur;
          }
          // the last block's buffer columns follow the nev_k locked ones
          if (nb)
            DKS_CUDA_TRY(cudaMemcpyAsync(xk + (size_t)nv * rows, b64.z[prev_cur] + (size_t)prev_nw * rows,
                                         (size_t)nb * rows * sizeof(double2), cudaMemcpyDeviceToDevice, ws));
          DKS_CUDA_TRY(cudaStreamSynchronize(ws));
          o32 = acc32;
          o64 = acc64;
          happ += acc32.happ + acc64.happ;
          return DKS_OK;
        }
        if (mixed) {
          DKS_TRY(convert<double2, float2>((const double2*)X[ik], b32.z[0], elems, ws));
          o32.cur = 0;
          DKS_TRY(phase<float2>(ctx, ex, ik, b32, sm, pin, n, nv, std::max(opts.refine_tol, tol), opts.n_init,
                                opts.n_iter, C, om, opts.precond, opts.use_filter, true, opts.chol_tol,
                                opts.drop_tol, h, o32, ws));
          DKS_TRY(convert<float2, double2>(b32.z[o32.cur], b64.z[0], elems, ws));
          o64.cur = 0;
          const int left = std::max(0, opts.n_iter - o32.iterations);
          DKS_TRY(phase<double2>(ctx, ex, ik, b64, sm, pin, n, nv, tol, opts.use_filter ? 1 : 0, left, C, om,
                                 opts.precond, opts.use_filter, false, opts.chol_tol, opts.drop_tol, h, o64, ws,
                                 opts.emulate_fp64 != 0));
        } else {
          DKS_CUDA_TRY(cudaMemcpyAsync(b64.z[0], X[ik], elems * sizeof(double2), cudaMemcpyDeviceToDevice, ws));
          o64.cur = 0;
          DKS_TRY(phase<double2>(ctx, ex, ik, b64, sm, pin, n, nv, tol, opts.n_init, opts.n_iter, C, om,
                                 opts.precond, opts.use_filter, false, opts.chol_tol, opts.drop_tol, h, o64, ws));
        }
        DKS_CUDA_TRY(cudaMemcpyAsync(X[ik], b64.z[o64.cur], elems * sizeof(double2), cudaMemcpyDeviceToDevice,
                                     ws));
        DKS_CUDA_TRY(cudaStreamSynchronize(ws));
        for (int j = 0; j < nv; ++j) eig[eoff[ik] + j] = pin.lam[j];
        happ += o32.happ + o64.happ;
        return DKS_OK;
      };
      const int rc = run();
      if (rc != DKS_OK) {
        krc[ik] = rc;
        kmsg[ik] = dks_last_error();
      }
    }
  };
  if (nworkers == 1) {
    worker(0);
  } else {
    std::vector<std::thread> threads;
    for (int w = 0; w < nworkers; ++w) threads.emplace_back(worker, w);
    for (std::thread& t : threads) t.join();
  }
  int status = DKS_OK;
  for (int ik = 0; ik < ctx->nk && status == DKS_OK; ++ik)
    if (krc[ik] != DKS_OK) status = fail(krc[ik], "k-point " + std::to_string(ik) + ": " + kmsg[ik]);
  // a tensor-core kernel that gave up a bounded wait left its results incomplete
  if (status == DKS_OK && tc_mask() != 0 && tc_status_take() == DKS_ERR_TIMEOUT)
    status = fail(DKS_ERR_TIMEOUT, "a tensor-core contraction gave up a bounded wait");
  for (int ik = 0; ik < ctx->nk && status == DKS_OK; ++ik) {
    if (o64s[ik].neg) status = fail(DKS_ERR_NEG_STATE, "a returned eigenvalue lies below the gap midpoint");
    else if (!o64s[ik].converged) status = fail(DKS_ERR_NOT_CONVERGED, "n_iter exhausted");
  }
  if (report) {
    for (int ik = 0; ik < std::min(ctx->nk, 64); ++ik) {
      report->iterations[ik] = o32s[ik].iterations + o64s[ik].iterations;
      report->fp64_iterations[ik] = o64s[ik].iterations;
      report->max_residual[ik] = o64s[ik].max_res;
    }
    report->h_applications = happ.load();
    report->hist_len = (int)std::min<size_t>(hist.size(), 512);
    for (int i = 0; i < report->hist_len; ++i) report->res_history[i] = hist[i];
    report->status = status;
    report->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return status;
}

}  // extern "C"

// Autotuning of the H' application's launch parameters and contraction schedule.  The paper has
// no counterpart (its code ran on CPUs); the parameters are this implementation's: the byte budget
// of one chunk of FFT intermediates (how many bands' stick buffers share the L2-resident working
// set between the three FFT passes), the CTA size of the one-kernel plane FFT, whether the plane
// FFT runs as one kernel or as row and column kernels, and (complex64 blocks) whether the
// projector contractions run on the tensor cores or the CUDA cores.  dks_autotune times H' on a scratch block for every
// candidate with CUDA events on the caller's stream and keeps the fastest; dks_tune_set applies
// a stored choice (the Python layer caches choices per grid, basis size, block width, precision
// and device).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "dks_internal.h"

using namespace dks;

namespace {

bool valid_tuning(long long chunk, int threads, int split) {
  return chunk >= (1LL << 20) && chunk <= (1LL << 36) &&
         (threads == 0 || (threads >= 64 && threads <= 512 && threads % 32 == 0)) && (split == 0 || split == 1);
}

}  // namespace

int dks_tune_get(const dks_ctx* ctx, long long* fft_chunk_bytes, int* plane_threads, int* plane_split) {
  if (!ctx || !fft_chunk_bytes || !plane_threads || !plane_split)
    return fail(DKS_ERR_INVALID_ARG, "dks_tune_get: bad argument");
  *fft_chunk_bytes = (long long)ctx->chunk_budget;
  *plane_threads = ctx->plane_threads;
  *plane_split = ctx->plane_split;
  return DKS_OK;
}

int dks_tune_set(dks_ctx* ctx, long long fft_chunk_bytes, int plane_threads, int plane_split) {
  if (!ctx || !valid_tuning(fft_chunk_bytes, plane_threads, plane_split))
    return fail(DKS_ERR_INVALID_ARG,
                "dks_tune_set: need 1 MB <= chunk bytes <= 64 GB, plane threads 0 or a multiple of 32 in 64..512, "
                "split 0 or 1");
  ctx->chunk_budget = (size_t)fft_chunk_bytes;
  ctx->plane_threads = plane_threads;
  ctx->plane_split = plane_split;
  return DKS_OK;
}

int dks_tune_contractions_get(const dks_ctx* ctx, int* proj_tc) {
  if (!ctx || !proj_tc) return fail(DKS_ERR_INVALID_ARG, "dks_tune_contractions_get: bad argument");
  *proj_tc = ctx->tc_proj;
  return DKS_OK;
}

int dks_tune_contractions_set(dks_ctx* ctx, int proj_tc) {
  if (!ctx || proj_tc < -1 || proj_tc > 1)
    return fail(DKS_ERR_INVALID_ARG, "dks_tune_contractions_set: proj_tc must be -1, 0 or 1");
  ctx->tc_proj = proj_tc;
  return DKS_OK;
}

int dks_autotune(dks_ctx* ctx, int ik, int nb, int prec, void* stream, dks_tune_report* rep) {
  if (!ctx || ik < 0 || ik >= ctx->nk || nb < 1 || prec < 0 || prec > 2)
    return fail(DKS_ERR_INVALID_ARG, "dks_autotune: bad argument");
  if (rep) std::memset(rep, 0, sizeof(*rep));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t elems = (size_t)nb * ctx->ncomp * ctx->k[ik].npw;
  const size_t es = prec == DKS_PREC_FP32 ? sizeof(float2) : sizeof(double2);
  const long long chunks[4] = {16LL << 20, 32LL << 20, 64LL << 20, 128LL << 20};
  const int threads[4] = {0, 128, 256, 512};
  const size_t old_chunk = ctx->chunk_budget;
  const int old_threads = ctx->plane_threads, old_split = ctx->plane_split;
  // the one-kernel plane form is a candidate only where the plane fits one CTA
  const size_t es_s = prec == DKS_PREC_FP32 ? sizeof(float2) : sizeof(double2);
  const bool fits = (size_t)ctx->grid[0] * ctx->plane_ld * es_s <= 227 * 1024;
  void* buf = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  DKS_CUDA_TRY(cudaMallocAsync(&buf, 2 * elems * es, st));
  int rc = DKS_OK;
  double best_ms = 0.0;
  int best = -1, ncand = 0;
  long long cc[32];
  int ct[32], cs[32];
  double cms[32];
  auto body = [&]() -> int {
    DKS_CUDA_TRY(cudaMemsetAsync(buf, 0, 2 * elems * es, st));
    DKS_CUDA_TRY(cudaEventCreate(&e0));
    DKS_CUDA_TRY(cudaEventCreate(&e1));
    void* x = buf;
    void* hx = (char*)buf + elems * es;
    for (int sp = fits ? 0 : 1; sp < 2; ++sp)
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < (sp ? 1 : 4); ++b) {   // the CTA size belongs to the one-kernel form
          ctx->chunk_budget = (size_t)chunks[a];
          ctx->plane_threads = threads[b];
          ctx->plane_split = sp;
          DKS_TRY(dks_apply_H(ctx, ik, x, hx, nb, prec, st));   // warm-up (smem attributes, workspace)
          DKS_CUDA_TRY(cudaEventRecord(e0, st));
          for (int r = 0; r < 3; ++r) DKS_TRY(dks_apply_H(ctx, ik, x, hx, nb, prec, st));
          DKS_CUDA_TRY(cudaEventRecord(e1, st));
          DKS_CUDA_TRY(cudaEventSynchronize(e1));
          float ms = 0.0f;
          DKS_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
          cc[ncand] = chunks[a];
          ct[ncand] = threads[b];
          cs[ncand] = sp;
          cms[ncand] = ms / 3.0;
          if (best < 0 || cms[ncand] < best_ms) {
            best = ncand;
            best_ms = cms[ncand];
          }
          ++ncand;
        }
    return DKS_OK;
  };
  rc = body();
  // contraction schedule of the projector terms (complex64 blocks on a GB300): both timed at the
  // chosen FFT parameters
  int proj_best = -1;
  double proj_ms[2] = {0.0, 0.0};
  if (rc == DKS_OK && best >= 0 && prec == DKS_PREC_FP32 && ctx->nproj > 0 && tc_device()) {
    const int old_tc = ctx->tc_proj;
    ctx->chunk_budget = (size_t)cc[best];
    ctx->plane_threads = ct[best];
    ctx->plane_split = cs[best];
    void* x = buf;
    void* hx = (char*)buf + elems * es;
    for (int t = 0; t < 2 && rc == DKS_OK; ++t) {
      ctx->tc_proj = t;
      rc = dks_apply_H(ctx, ik, x, hx, nb, prec, st);
      if (rc == DKS_OK && cudaEventRecord(e0, st) != cudaSuccess) rc = fail(DKS_ERR_CUDA, "dks_autotune: event");
      for (int r = 0; r < 3 && rc == DKS_OK; ++r) rc = dks_apply_H(ctx, ik, x, hx, nb, prec, st);
      float ms = 0.0f;
      if (rc == DKS_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                           cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        rc = fail(DKS_ERR_CUDA, "dks_autotune: event timing");
      proj_ms[t] = ms / 3.0;
    }
    ctx->tc_proj = old_tc;
    if (rc == DKS_OK) proj_best = proj_ms[1] < proj_ms[0] ? 1 : 0;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(buf, st);
  cudaStreamSynchronize(st);
  if (rc != DKS_OK || best < 0) {
    ctx->chunk_budget = old_chunk;
    ctx->plane_threads = old_threads;
    ctx->plane_split = old_split;
    return rc != DKS_OK ? rc : fail(DKS_ERR_CUDA, "dks_autotune: no candidate timed");
  }
  ctx->chunk_budget = (size_t)cc[best];
  ctx->plane_threads = ct[best];
  ctx->plane_split = cs[best];
  if (proj_best >= 0) ctx->tc_proj = proj_best;
  if (rep) {
    rep->proj_tc = proj_best;
    rep->proj_ms[0] = proj_ms[0];
    rep->proj_ms[1] = proj_ms[1];
    rep->ncand = ncand;
    rep->best = best;
    for (int i = 0; i < ncand; ++i) {
      rep->chunk_bytes[i] = cc[i];
      rep->plane_threads[i] = ct[i];
      rep->plane_split[i] = cs[i];
      rep->ms[i] = cms[i];
    }
  }
  return DKS_OK;
}

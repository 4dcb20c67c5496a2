// Per-launch device timing (CUDA events on the launching stream) and launch counters.
// Counting is always on; event pairs are recorded only while profiling is enabled.
#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "dks_internal.h"

namespace dks {

namespace {
struct Rec {
  int cat;
  cudaEvent_t a, b;
  double bytes, flops;
};
std::mutex g_mu;
std::vector<cudaEvent_t> g_pool;
std::vector<Rec> g_recs;
bool g_on = false;
long long g_launch[P_NCAT] = {0};
const char* g_names[P_NCAT] = {"stick_inverse_fft",      "plane_fft_v",        "stick_forward_fft_dirac",
                               "dirac_only",             "proj_bh_x",          "proj_b_dz",
                               "gram",                   "rotate",             "rayleigh_ritz",
                               "col_stats",              "precond_teter",      "convert_gather",
                               "scf_grid",
                               "stick_inverse_fft_fp32", "plane_fft_v_fp32",   "stick_forward_fft_dirac_fp32",
                               "dirac_only_fp32",        "proj_bh_x_fp32",     "proj_b_dz_fp32",
                               "gram_fp32",              "rotate_fp32"};
cudaEvent_t take() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

Prof::Prof(int cat, cudaStream_t st, double bytes, double flops) : cat_(cat), st_(st), idx_(-1) {
  std::lock_guard<std::mutex> g(g_mu);
  ++g_launch[cat];
  if (!g_on) return;
  Rec r{cat, take(), take(), bytes, flops};
  cudaEventRecord(r.a, st);
  g_recs.push_back(r);
  idx_ = (long long)g_recs.size() - 1;
}

void Prof::count(int n) {
  std::lock_guard<std::mutex> g(g_mu);
  g_launch[cat_] += n;
}

Prof::~Prof() {
  if (idx_ < 0) return;
  std::lock_guard<std::mutex> g(g_mu);
  cudaEventRecord(g_recs[idx_].b, st_);
}

}  // namespace dks

using namespace dks;

extern "C" {

int dks_profile_ncat(void) { return P_NCAT; }

const char* dks_profile_name(int cat) { return (cat >= 0 && cat < P_NCAT) ? g_names[cat] : ""; }

int dks_profile_enable(int on) {
  std::lock_guard<std::mutex> g(g_mu);
  for (Rec& r : g_recs) {
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
  for (long long& c : g_launch) c = 0;
  g_on = on != 0;
  return DKS_OK;
}

int dks_profile_read(int ncat, double* ms, long long* launches, double* bytes, double* flops) {
  if (ncat < P_NCAT || !ms || !launches || !bytes || !flops)
    return fail(DKS_ERR_INVALID_ARG, "dks_profile_read: arrays of dks_profile_ncat() entries required");
  DKS_CUDA_TRY(cudaDeviceSynchronize());
  std::lock_guard<std::mutex> g(g_mu);
  for (int c = 0; c < ncat; ++c) {
    ms[c] = 0;
    bytes[c] = 0;
    flops[c] = 0;
    launches[c] = c < P_NCAT ? g_launch[c] : 0;
  }
  for (Rec& r : g_recs) {
    float t = 0;
    if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) ms[r.cat] += t;
    bytes[r.cat] += r.bytes;
    flops[r.cat] += r.flops;
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
  for (long long& c : g_launch) c = 0;
  return DKS_OK;
}

}  // extern "C"

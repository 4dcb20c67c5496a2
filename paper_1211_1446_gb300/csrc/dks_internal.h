// Internal declarations of the GB300 DKS / LOBPCG-F library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dks.h"

namespace dks {

constexpr int kMaxFftLen = 256;    // largest FFT axis length
constexpr int kMaxRadix = 8;       // radices 2, 3, 4, 5, 7, 8
constexpr int kMaxStages = 8;
constexpr int kMaxRR = 512;        // largest Rayleigh-Ritz pencil

// --------------------------------------------------------------- error state
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
#define DKS_CUDA_TRY(...)                                                                      \
  do {                                                                                         \
    cudaError_t e_ = (__VA_ARGS__);                                                            \
    if (e_ != cudaSuccess)                                                                     \
      return ::dks::fail(DKS_ERR_CUDA, std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_)); \
  } while (0)
#define DKS_TRY(...)                 \
  do {                               \
    int r_ = (__VA_ARGS__);          \
    if (r_ != DKS_OK) return r_;     \
  } while (0)

// --------------------------------------------------------------- FFT plans
// Mixed-radix in-place plan of one axis.  DIF stages run s = 0..nst-1 on blocks
// of length L_s (L_0 = N, L_{s+1} = L_s / R_s); DIT runs them in reverse.
struct AxisPlan {
  int n;
  int nst;
  int radix[kMaxStages];
  int blk[kMaxStages];   // L_s
};
bool make_axis_plan(int n, AxisPlan* p);
// position of frequency index k after the DIF stages (mixed-radix digit reversal)
std::vector<int> dif_positions(const AxisPlan& p);

// --------------------------------------------------------------- per-k basis
struct KPoint {
  int npw = 0;
  int nsticks = 0;
  double kcart[3] = {0, 0, 0};
  double ecut = 0;
  double qmax = 0;
  std::vector<int> miller;      // host npw*3, canonical order
  // device tables
  int* stick_start = nullptr;   // nsticks+1, pw offsets
  int* stick_plane = nullptr;   // nsticks, i1*LD + i2 (natural frequency position, padded rows)
  int* pw_stick = nullptr;      // npw
  int* pw_iz = nullptr;         // npw, i3 (natural)
  double* q = nullptr;          // npw*3 cartesian k+G (FP64)
  float* cq32 = nullptr;        // npw*6: c (k+G)_x, c (k+G)_y, c (k+G)_z as double-float (hi, lo) pairs
  double* ek = nullptr;         // npw, |k+G|^2/2
  double2* bt64 = nullptr;      // nproj x (2 npw) projector rows (beta, spin-major)
  float2* bt32 = nullptr;
  float4* btdf = nullptr;       // the same rows as double-float (re hi, re lo, im hi, im lo)
  // exact integer slices of bt64 for the refinement phase's projector contractions on the
  // tensor cores (oz_gemm.cu layout), made on first use; btoz_state 1 ready, -1 not held
  void* btoz = nullptr;
  int btoz_state = 0;
  double cshift = 0, omega = 1; // default filter constants
};

struct Workspace {
  void* ptr = nullptr;
  size_t bytes = 0;
};

// Execution state of one stream of work (one solve worker, or the context's own stream for the
// single-step entry points).  Never shared by two host threads at the same time.
struct Exec {
  Workspace ws_h;               // H' intermediates + projector coefficients
  Workspace ws_solve;           // solver blocks
  Workspace ws_oz;              // exact integer slices of x~ for the projector contractions
  bool df_gemm = false;         // complex128 projector contractions in double-float arithmetic
  cudaStream_t own = nullptr;   // stream created for a concurrent solve worker
};

}  // namespace dks

struct dks_ctx {
  int grid[3] = {0, 0, 0};
  int ng = 0;
  double c = 137.036;
  double lattice[9];
  double recip[9];
  double volume = 0;
  int nk = 0;
  dks::AxisPlan plan[3];
  int plane_ld = 0;              // row stride of an N1 x N2 plane in shared memory (N2 rounded up to odd)
  // device: twiddles exp(+2 pi i t / N_axis), t < N_axis
  double2* tw64[3] = {nullptr, nullptr, nullptr};
  float2* tw32[3] = {nullptr, nullptr, nullptr};
  float4* twdf[3] = {nullptr, nullptr, nullptr};   // double-float twiddles (re hi, re lo, im hi, im lo)
  // device: V / Ng in DIF-permuted layout [p3][p1*LD + p2], zero in the padding column
  double* vperm64 = nullptr;
  float* vperm32 = nullptr;
  float2* vpermdf = nullptr;    // double-float (hi, lo) copy
  double vmax = 0;
  bool has_v = false;
  int* posd[3] = {nullptr, nullptr, nullptr};   // device: DIF position of natural index i per axis
  double* vloc_dev = nullptr;   // device: the potential given at creation, natural grid order (or NULL)
  // projectors
  int nproj = 0;
  double dsum = 0;
  std::vector<double> dvec;     // host, per channel
  double* dvec_dev = nullptr;
  std::vector<dks::KPoint> k;
  // execution states owned by the context (grown on demand): exec[0] serves the single-step
  // entry points and serial solves, exec[1..] the concurrent k-point workers
  std::vector<dks::Exec*> exec;
  size_t chunk_budget = 64u << 20;   // bytes of FFT intermediates per chunk (L2-resident)
  int plane_threads = 0;             // CTA size of the plane FFT kernel (0: from the FFT plan)
  int plane_split = 0;               // 1: pass B as row / column kernels even when a plane fits one CTA
  int ncomp = 4;                     // components per column: 4 (DKS, Eq. vDKS) or 2 (KSSO two-spinors)
  int tc_proj = -1;                  // projector contractions of complex64 blocks: -1 follow the
                                     // process-wide mask, 0 CUDA cores, 1 tensor cores (tuner's choice)
  int device = 0;
  int num_sms = 0;
};

namespace dks {

// ---------------------------------------------------------------- profiling
enum ProfCat {
  P_STICK_INV, P_PLANE, P_STICK_FWD, P_DIRAC, P_PROJ_HN, P_PROJ_NN, P_GRAM, P_ROTATE, P_RR, P_STATS,
  P_PRECOND, P_MISC, P_SCF,
  // the same kernels launched on complex64 data (FP32 arithmetic)
  P_STICK_INV32, P_PLANE32, P_STICK_FWD32, P_DIRAC32, P_PROJ_HN32, P_PROJ_NN32, P_GRAM32, P_ROTATE32,
  P_NCAT
};
constexpr int kProf32 = P_STICK_INV32 - P_STICK_INV;   // offset of the complex64 variant
// RAII scope around one kernel launch: counts it, and while profiling is on records a
// CUDA event pair on the launching stream with the launch's algorithmic bytes and flops.
class Prof {
 public:
  Prof(int cat, cudaStream_t st, double bytes, double flops);
  ~Prof();
  // books n further kernel launches (negative: fewer) inside the same timed scope
  void count(int n);
 private:
  int cat_;
  cudaStream_t st_;
  long long idx_;
};

// Algorithmic real flops of one Rayleigh-Ritz step on an m x m Hermitian pencil for n Ritz
// pairs (Cholesky m^3/6, two triangular solves m^3/2 each, Householder tridiagonalisation
// 2m^3/3 complex multiply-adds; back-transformation m^2 n and the L^-H solve m^2 n / 2;
// 8 real flops per complex multiply-add).  The tridiagonal eigensolver is O(m n) and omitted.
inline double rr_flops(int m, int n) {
  const double md = m, nd = n;
  return 8.0 * (md * md * md * (1.0 / 6.0 + 1.0 + 2.0 / 3.0) + 1.5 * md * md * nd);
}

// NVTX range around a host scope (solves, phases, SCF iterations), for timeline tools; without
// a tool attached the calls return at once
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

int grow(Workspace& w, size_t bytes);
void release(Workspace& w);

// H' application on nb columns of k-point ik:
//   out = scale * (H' x - shift * x)          (beta == 0)
// x and out [nb][4][npw]; precision by template (double2 / float2).
template <typename V>
int apply_h(dks_ctx* ctx, Exec& ex, int ik, const V* x, V* out, int nb, double shift, double scale,
            cudaStream_t st);
Exec& exec0(dks_ctx* ctx);
// small two-spinors of nb columns from their large ones, Eq. (RKB); x complex128 (fp64) or complex64
int kinetic_balance(dks_ctx* ctx, int ik, void* x, int nb, bool fp64, cudaStream_t st);
// debug build: first failed device index check of the FFT kernels (then cleared); 0 otherwise
unsigned debug_check_take();
// rho (natural grid order) += sum_j occ[j] |psi_j(r)|^2 / vol over the columns of x (complex128)
int density_accumulate(dks_ctx* ctx, int ik, const double2* x, int nb, const double* occ, double* rho,
                       cudaStream_t st);

// kernels shared by the solver and the single-step entry points
template <typename Va, typename Vb = Va, bool Acc64 = false>
int gemm_hn(const Va* a, int lda, const Vb* b, int ldb, int k, int m, int n, double2* c,
            cudaStream_t st, int cat = P_GRAM, int ldc = 0, bool lower = false, int tc = -1);
// tc (complex64 operands only): -1 the process-wide tensor-core mask decides, 0 CUDA cores,
// 1 tensor cores where the device and the operands allow them
// c (m x n, col-major, leading dimension ldc or m) += a^H b, FP64 atomics; FP64 arithmetic when
// either operand is complex128 or Acc64; lower: only the block lower triangle (square results)
int mirror_lower(double2* c, int m, cudaStream_t st);   // upper triangle = conj of the lower
int set_diag_ramp(double2* a, int m, cudaStream_t st);  // a = diag(1, ..., m)
// block lower triangles of A += Z^H HZ and S += Z^H Z (m x m, column-major) from FP32 blocks in one pass
int gram_f32(const float2* z, const float2* hz, int ld, int k, int m, double2* a, double2* s, cudaStream_t st);
// double-float (FP32-pair) versions of the two contractions for complex128 data
int gemm_hn_df(const double2* a, int lda, const double2* b, int ldb, int k, int m, int n, double2* c,
               cudaStream_t st, int cat = P_GRAM, int ldc = 0, bool lower = false);
int gemm_nn_df(const double2* a, int lda, int k, int m, const double2* w, int ldw, const double* wscale,
               int n, double2* out, int ldo, double beta, cudaStream_t st, double alpha = 1.0,
               int cat = P_ROTATE);
// the same with operands already split into (re hi, re lo, im hi, im lo) quadruples
int gemm_hn_df(const float4* a, int lda, const float4* b, int ldb, int k, int m, int n, double2* c,
               cudaStream_t st, int cat = P_GRAM, int ldc = 0, bool lower = false);
int gemm_hn_df(const float4* a, int lda, const double2* b, int ldb, int k, int m, int n, double2* c,
               cudaStream_t st, int cat = P_GRAM, int ldc = 0, bool lower = false);
int gemm_nn_df(const float4* a, int lda, int k, int m, const double2* w, int ldw, const double* wscale,
               int n, double2* out, int ldo, double beta, cudaStream_t st, double alpha = 1.0,
               int cat = P_ROTATE);
int split_df(const double2* in, float4* out, size_t n, cudaStream_t st);
// block lower triangles of A += Z^H HZ and S += Z^H Z from double-float copies in one pass
int gram_df(const float4* z, const float4* hz, int ld, int k, int m, double2* a, double2* s, cudaStream_t st);
template <typename Va, typename Vo = Va>
int gemm_nn(const Va* a, int lda, int k, int m, const double2* w, int ldw, const double* wscale,
            int n, Vo* out, int ldo, double beta, cudaStream_t st, double alpha = 1.0,
            int cat = P_ROTATE, int tc = -1);
// out (k x n) = alpha * a (k x m) * (diag(wscale) w) + beta * out; wscale may be NULL;
// FP64 arithmetic when a or out is complex128
// columns of ncomp x npw elements (ncomp = 4: DKS four-spinors, 2: KSSO two-spinors)
template <typename V>
int col_stats(const V* x, const V* hx, const double* lam, const double* ek, int npw, int n,
              double* stats, cudaStream_t st, int ncomp = 4);  // stats[3j..]: |hx - lam x|^2, |x|^2, sum ek|x|^2
template <typename V, typename Vo = V>
int precond_apply(const V* x, const V* hx, const double* lam, const double* stats, const int* act,
                  int nact, const double* ek, int npw, int precond, Vo* y, cudaStream_t st, int ncomp = 4);
int rayleigh_ritz(const double2* a, const double2* s, int nz, int n, double2* v, double* lam,
                  int* info, double2* scratch, cudaStream_t st, double chol_tol = 1e-12,
                  double drop_tol = 1e-12);
size_t rr_scratch_elems(int nz);
// failure-detection test hook: polls of the first staging wait of the per-column Rayleigh-Ritz
// kernels, and the count (then cleared) of steps the single-CTA kernel redid after such a wait
// gave up
int rr_set_first_wait(unsigned polls);
int rr_timeout_redos_take(unsigned* out);
template <typename Vi, typename Vo>
int convert(const Vi* in, Vo* out, size_t n, cudaStream_t st);
int gather_cols(const double2* v, int ldv, int row0, int rows, const int* act, int nact,
                double2* out, cudaStream_t st);

// ---------------------------------------------------------------- tensor-core contractions
// complex64 contractions on tcgen05 with three BF16 slices per FP32 value (tc_gemm.cu); the
// bits select which of the FP32 contractions take that path (dks_tensor_cores)
constexpr int TC_ROTATE = DKS_TC_ROTATE, TC_GRAM = DKS_TC_GRAM, TC_PROJ_HN = DKS_TC_PROJ_HN,
              TC_PROJ_NN = DKS_TC_PROJ_NN, TC_FP64 = DKS_TC_FP64, TC_ALL = DKS_TC_ALL,
              TC_DEFAULT = DKS_TC_DEFAULT;
bool tc_enabled(int bit);            // bit selected and the device is a GB300 (sm_103)
bool tc_device();                    // the device is a GB300 (sm_103)
int tc_mask();
int tc_set(int mask, int kchunk);
int tc_get(int* mask, int* kchunk);
int tc_status_take();                // DKS_ERR_TIMEOUT when a tensor-core kernel gave up a wait (then cleared)
bool tc_nn_supported(const float2* a, int lda, int k, int m, int n);
bool tc_hn_supported(const float2* a, int lda, const float2* b, int ldb, int k);
// out (k x n) = alpha a (k x m) diag(wscale) w + beta out
int tc_gemm_nn(const float2* a, int lda, int k, int m, const double2* w, int ldw, const double* wscale, int n,
               float2* out, int ldo, double beta, cudaStream_t st, double alpha, int nsm);
// lower triangles of A = Z^H HZ and S = Z^H Z (m x m), written (not accumulated)
int tc_gram(const float2* z, const float2* hz, int ld, int k, int m, double2* a, double2* s, cudaStream_t st, int nsm);
// c = a^H b (m x n, ldc), or with conj_transpose_out c = b^H a (n x m, ldc), written
int tc_gemm_hn(const float2* a, int lda, const float2* b, int ldb, int k, int m, int n, double2* c, int ldc,
               bool conj_transpose_out, cudaStream_t st, int nsm);

// complex128 contractions on tcgen05 from exact integer slices (oz_gemm.cu): a block is sliced
// once (oz_split) into a buffer of oz_bytes(rows, ncol) bytes laid out by oz_layout
struct OzBlock {
  uint16_t* sl = nullptr;            // [7 slices][re, im][ncolp / 8][rowsp / 8][8 x 8] BF16
  int* ex = nullptr;                 // [rowsp / 128][ncolp] window exponents
  int rows = 0, rowsp = 0, ncol = 0, ncolp = 0;
};
size_t oz_bytes(int rows, int ncol);
int oz_layout(void* buf, int rows, int ncol, OzBlock* out);
// slices of the first ncol columns of a (rows x ncol, lda); ncol <= the block's capacity
int oz_split(const double2* a, long long lda, int ncol, const OzBlock& z, cudaStream_t st);
// lower triangles of A = Z^H HZ and S = Z^H Z over the first m columns (m x m, written)
int oz_gram(const OzBlock& z, const OzBlock& hz, int m, double2* a, double2* s, cudaStream_t st);
// out (rows x n, ldo) = alpha Z[:, c0 : c0 + m] W (+ beta out), W m x n complex128 (ldw)
int oz_rotate(const OzBlock& z, int c0, int m, const double2* w, int ldw, int n, double2* out, int ldo, double beta,
              cudaStream_t st, double alpha = 1.0, const double* wscale = nullptr, int cat = P_ROTATE);
// C = A^H B (m x n, ldc) over the first m columns of a and n of b, or with conj_transpose_out
// C = B^H A (n x m, ldc); written
int oz_gemm_hn(const OzBlock& a, int m, const OzBlock& b, int n, double2* c, int ldc, bool conj_transpose_out,
               cudaStream_t st, int cat = P_GRAM);
// the slices of a k-point's projector table (created on first use; false when they cannot be held)
bool projector_slices(dks_ctx* ctx, int ik, cudaStream_t st);
int oz_status_take();                // DKS_ERR_TIMEOUT when such a kernel gave up a wait (then cleared)

}  // namespace dks

/*
 * dks.h -- C ABI of the GB300 LOBPCG-F solver for the four-component
 * Dirac-Kohn-Sham (DKS) operator in a planewave basis.
 *
 * Method: Lin, Shao and E, "Efficient iterative method for solving the
 * Dirac-Kohn-Sham density functional theory", Algorithm 1 (LOBPCG-F) with the
 * filter f(E) = (E - C)^2 / Omega^2 of Eq. (filter), applied to the valence DKS
 * operator of Eq. (vDKS): the free Dirac operator of Eq. (2), a local potential
 * V(r) I4 and the spin-orbit projectors of Eq. (HGH), discretised by planewaves
 * (Sec. 2.3).  All energies are shifted by -mc^2 (Sec. 4): the library works
 * with H' = H - c^2, the positive band starts near 0 and the gap midpoint is
 * -c^2.
 *
 * Conventions shared by every entry point
 *  - Units: atomic units (bohr, Hartree), m = 1.
 *  - Basis of k-point ik: G = m1 b1 + m2 b2 + m3 b3 with |k+G|^2/2 <= ecut_k,
 *    in canonical order (Miller triples sorted lexicographically, signed).
 *    dks_basis() returns the Miller triples in that order.
 *  - Vector blocks: X[band][comp][pw], complex interleaved (re, im), contiguous,
 *    comp 0,1 the large two-spinor (spin up, down), comp 2,3 the small one
 *    (contexts of model DKS_MODEL_KSSO: comp 0,1 only, see dks_create_model).
 *    complex128 for DKS_PREC_FP64, complex64 for DKS_PREC_FP32.
 *  - Device pointers are CUDA device memory owned by the caller; host pointers
 *    are read during the call only.  `stream` is a cudaStream_t (NULL = legacy
 *    default stream).  Calls are asynchronous on `stream` unless stated.
 *  - Errors: every function returns DKS_OK (0) or a negative DKS_ERR_* code;
 *    dks_strerror() describes it and dks_last_error() gives detail for the
 *    calling thread.  Nothing is thrown across the ABI; no kernel traps.
 */
#ifndef DKS_H
#define DKS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DKS_OK 0
#define DKS_ERR_INVALID_ARG (-1)   /* bad pointer, size, index or option          */
#define DKS_ERR_CUDA (-2)          /* a CUDA runtime call failed                   */
#define DKS_ERR_OOM (-3)           /* device or host allocation failed             */
#define DKS_ERR_NOT_CONVERGED (-4) /* n_iter exhausted; partial results returned   */
#define DKS_ERR_NEG_STATE (-5)     /* a selected Ritz value is below the gap midpoint */
#define DKS_ERR_RANK (-6)          /* SVQB left fewer directions than the block    */
#define DKS_ERR_TIMEOUT (-7)       /* a bounded device wait gave up               */
#define DKS_ERR_GRID (-8)          /* a planewave sphere does not fit the FFT grid */
#define DKS_ERR_UNSUPPORTED (-9)   /* size outside the compiled limits             */

#define DKS_PREC_FP64 0  /* complex128 storage, FP64 arithmetic                      */
#define DKS_PREC_FP32 1  /* complex64 storage, FP32 arithmetic (FP64 Dirac 4x4 term) */
#define DKS_PREC_FP64_EMULATED 2 /* complex128 storage; the tall-skinny contractions (Gram,
                                    rotations, projectors) in double-float arithmetic on the
                                    FP32 units (~48-bit significand), everything else FP64   */

typedef struct dks_ctx dks_ctx; /* opaque; owns basis tables and workspace */

/* Cell, grid and k-points (Sec. 2.3, Sec. 4).  lattice rows are a1, a2, a3 in
 * bohr; grid = FFT grid (N1, N2, N3) used for wavefunctions and potential;
 * c = speed of light; kfrac = nk x 3 fractional k-points (host); ecut_k = nk
 * cutoffs in Ha (host) or NULL to use the `ecut` argument of dks_create. */
typedef struct {
  double lattice[9];
  int grid[3];
  double c;
  int nk;
  const double* kfrac;
  const double* ecut_k;
} dks_cell;

/* Local potential V(r) (Eq. vDKS: V_hxc + local pseudopotential) on the grid,
 * host FP64 array v_r[(i1*N2 + i2)*N3 + i3] = V(sum_i (i_i/N_i) a_i) in Ha.
 * v_r = NULL means V = 0. */
typedef struct {
  const double* v_r;
} dks_potentials;

/* Spin-orbit projectors of Eq. (HGH) (host arrays, nsite may be 0):
 *   beta_{s,l,j,mj}(q) = p_l(|q|) Omega_{j l mj}(qhat) exp(-i q.R_s) / sqrt(vol)
 *   p_l(q) = A_l q^l exp(-q^2 rl^2 / 2),  A_l = sqrt(2 (2 pi)^3 rl^(2l+3) / Gamma(l+3/2))
 * with Omega the spinor spherical harmonics (Condon-Shortley Y_lm coupled to
 * spin 1/2), l = 0..lmax[s] <= 2, j = l +- 1/2.  The operator is
 * I2 (x) sum D beta beta^H (identical on large and small two-spinors, since
 * the spin operator of Eq. (HGH) is diag(sigma, sigma)/2).
 *   pos[nsite*3]   cartesian positions (bohr)
 *   lmax[nsite]    highest l (-1 = no projector on this site)
 *   rl[nsite*3]    Gaussian width per l (bohr)
 *   d[nsite*3*2]   strength D per (l, jj) in Ha; jj = 0: j = l+1/2, jj = 1: j = l-1/2 */
typedef struct {
  int nsite;
  const double* pos;
  const int* lmax;
  const double* rl;
  const double* d;
} dks_projectors;

/* dks_create: build the planewave spheres, grid maps and projector tables for
 * every k-point and upload them with V(r) to the current CUDA device.
 * Synchronous.  Errors: INVALID_ARG, GRID (sphere touches the Nyquist plane
 * or leaves the grid), UNSUPPORTED (grid axis > 256 or plane too large),
 * OOM, CUDA.  *out is NULL on error. */
int dks_create(const dks_cell* cell, double ecut, const dks_potentials* pot,
               const dks_projectors* proj, dks_ctx** out);
void dks_destroy(dks_ctx* ctx);

/* Operator models.  DKS: the shifted four-component Dirac-Kohn-Sham H' of
 * Eq. (vDKS), columns [4][npw] (large then small two-spinor).  KSSO: the
 * two-component Kohn-Sham operator with spin-orbit coupling of the paper's KSSO
 * module (Sec. 4), |k+G|^2/2 + V + sum D beta beta^H on a two-spinor, columns
 * [2][npw], energies unshifted; its solve is Algorithm 1 without the filter
 * (standard LOBPCG), and dks_kinetic_balance does not apply to it. */
#define DKS_MODEL_DKS 0
#define DKS_MODEL_KSSO 1
/* dks_create for a given model (dks_create is model DKS).  Every entry point
 * taking a ctx then works on columns of dks_ncomp(ctx) x npw elements. */
int dks_create_model(const dks_cell* cell, double ecut, const dks_potentials* pot,
                     const dks_projectors* proj, int model, dks_ctx** out);
/* The FFT plan of one grid axis of length n (host only, no device needed; exposed so that the
 * plan can be checked): nst passes of the radices radix[0..nst-1] (each of 2, 3, 4, 5, 6, 7, 8,
 * product n, fewest passes), run as decimation-in-frequency passes in this order for the inverse
 * transform.  pos (int[n], or NULL): the position at which the DIF passes leave frequency k
 * (mixed-radix digit reversal; the real-space planes and V live in this order on the device).
 * radix needs room for 8 entries.  Errors: INVALID_ARG, UNSUPPORTED (n > 256 or a prime factor
 * above 7). */
int dks_fft_plan(int n, int* nst, int* radix, int* pos);

/* Components per column: 4 (DKS) or 2 (KSSO). */
int dks_ncomp(const dks_ctx* ctx, int* ncomp);

/* Basis size of k-point ik, and its Miller triples (host int[npw*3]). */
int dks_npw(const dks_ctx* ctx, int ik, int* npw);
int dks_basis(const dks_ctx* ctx, int ik, int* miller);
/* Number of projector channels: 2(l+1) + 2l per l on each site (18 for an s, p, d site). */
int dks_nproj(const dks_ctx* ctx, int* nproj);

/* Default filter constants for k-point ik (readings of Sec. 3.1, shifted units):
 *   C     = -(3c^2 + sqrt(c^2 qmax^2 + c^4)) / 2  (midpoint of the free negative band)
 *   Omega = E_upper - C,  E_upper = sqrt(c^2 qmax^2 + c^4) - c^2 + max|V| + sum|D|. */
int dks_filter_constants(const dks_ctx* ctx, int ik, double* C, double* Omega);

/* dks_apply_H: HX = H' X for nb bands of k-point ik (Eq. vDKS, Sec. 3.1
 * "matrix-free" Hx; the KSSO operator for a KSSO context).  X, HX: device,
 * [nb][ncomp][npw] (ncomp from dks_ncomp), precision `prec`; X and HX
 * must not overlap.  Uses ctx workspace (not reentrant per ctx).  Errors:
 * INVALID_ARG, CUDA. */
int dks_apply_H(dks_ctx* ctx, int ik, const void* X, void* HX, int nb, int prec, void* stream);

/* dks_kinetic_balance (DKS contexts only): Eq. (RKB) with p -> q = k+G and m = 1 (atomic units):
 * for every column of X [nb][4][npw] (device, precision `prec`), the small
 * two-spinor (components 2, 3) is overwritten by (sigma.q) phi / (2c), phi the
 * large two-spinor (components 0, 1, left unchanged), sigma.q =
 * [[q_z, q_x - i q_y], [q_x + i q_y, -q_z]].  This turns large components from
 * a two-component (KS/KSSO) calculation, or from an earlier solve, into a start
 * block X0 for dks_lobpcgf_solve (Sec. 3.1 on initial vectors, with N_init = 1).
 * In place; FP64 arithmetic for complex128, FP32 for complex64.  Errors:
 * INVALID_ARG, CUDA. */
int dks_kinetic_balance(dks_ctx* ctx, int ik, void* X, int nb, int prec, void* stream);

/* dks_filter: FY = f(H') Y = (H' - C)^2 Y / Omega^2 (Eq. filter), applied as
 * two passes of (H' - C)/Omega.  C and Omega in shifted units (see
 * dks_filter_constants).  Same layout and rules as dks_apply_H. */
int dks_filter(dks_ctx* ctx, int ik, const void* Y, void* FY, int nb, double C, double Omega,
               int prec, void* stream);

/* ---------------------------------------------------------------- solver */

#define DKS_MODE_FP64 0  /* plain FP64 LOBPCG-F                                        */
#define DKS_MODE_MIXED 1 /* FP32 H, Gram and rotations + FP64 small RR and residual
                            norms, then FP64 refinement iterations                     */
#define DKS_PRECOND_TETER 0
#define DKS_PRECOND_IDENTITY 1

typedef struct {
  int n_init;          /* initial filter steps N_init (Algorithm 1), default 3          */
  int n_iter;          /* maximum iterations N_iter, default 200                       */
  int nbuf;            /* extra columns iterated but not convergence-checked           */
  double C, Omega;     /* filter constants; NaN = dks_filter_constants                 */
  int mode;            /* DKS_MODE_*                                                   */
  double refine_tol;   /* MIXED: FP64 once max residual < refine_tol (1e-5) or stalls   */
  int precond;         /* DKS_PRECOND_*                                                */
  int use_filter;      /* 1 = LOBPCG-F; 0 = standard LOBPCG (Alg. 1 without F lines)  */
  const int* nev_k;    /* per-k wanted pairs (host, nk) or NULL = the nev argument     */
  void* stream;        /* cudaStream_t for all work                                    */
  double chol_tol;     /* Rayleigh-Ritz: SVQB when a Cholesky pivot^2 < chol_tol (1e-12) */
  double drop_tol;     /* SVQB drops directions below drop_tol * max eig (1e-12)        */
  int emulate_fp64;    /* MIXED: refinement contractions in double-float arithmetic on
                          the FP32 units (1, default) or native FP64 (0)                */
  int concurrency;     /* k-points solved at the same time, each on its own internal stream
                          and host thread (0 = min(nk, 4), bounded by free device memory);
                          with more than one, `stream` is synchronised first             */
  int solver;          /* DKS_SOLVER_LOBPCG (Algorithm 1, default) or DKS_SOLVER_DAVIDSON */
  int m_max;           /* DAVIDSON: largest basis, in columns (0 = 4 (nev + nbuf)); at
                          least 2 (nev + nbuf) and at most 512                           */
  int block;           /* LOBPCG: wanted pairs per band block (0 = all in one block).  With
                          nev_k > block the pairs are found block by block: each block
                          iterates its `block` wanted columns plus the nbuf buffer columns
                          and has the converged vectors of the earlier blocks projected out
                          of its filtered start block and of every filtered correction
                          (deflation); it starts from the previous block's buffer columns
                          followed by the next unused columns of X.  The Rayleigh-Ritz limit
                          then applies to block + nbuf, not to nev_k + nbuf               */
} dks_solve_opts;

/* Solvers.  LOBPCG: Algorithm 1 (LOBPCG-F with use_filter = 1).  DAVIDSON: block Davidson with
 * the same filter step (the paper notes that the filter carries over to Davidson-type
 * solvers, Sec. 3): a growing orthonormal basis V replaces [X, Y, P]; every iteration does
 * Rayleigh-Ritz on V, forms T = f(H) K(R) on the active columns (Algorithm 1's preconditioning and filter steps),
 * restarts V from the Ritz vectors when it would exceed m_max columns, projects T out of V
 * (twice), orthonormalises it and appends it.  Same options, modes and report otherwise. */
#define DKS_SOLVER_LOBPCG 0
#define DKS_SOLVER_DAVIDSON 1

typedef struct {
  int iterations[64];        /* per k (first 64 k-points)                         */
  int fp64_iterations[64];   /* iterations run in FP64 (MIXED: refinement only)   */
  double max_residual[64];   /* final max ||H'x - lambda x|| over checked columns */
  long long h_applications;  /* single-band H' applications, all k               */
  double shift;              /* c^2 removed from every eigenvalue                  */
  double seconds;            /* wall time of the call (host clock)                 */
  int status;                /* DKS_OK or the first error                          */
  int hist_len;              /* entries of res_history                             */
  double res_history[512];   /* k-point 0: max checked residual after each RR      */
} dks_solve_report;

void dks_solve_opts_default(dks_solve_opts* opts);

/* dks_lobpcgf_solve: Algorithm 1 for every k-point of ctx.
 *  nev      wanted eigenpairs per k (unless opts->nev_k)
 *  tol      convergence test: every checked column has ||H'x - lambda x||_2 < tol
 *           with ||x||_2 = 1 (FP64 norms)
 *  eig      host double[sum_k nev_k], ascending per k, shifted by -c^2
 *  X        host array of nk device pointers; X[ik] is complex128
 *           [nev_k + nbuf][4][npw_k]: the start block X0 on entry (N_init filter
 *           steps are applied to it), the eigenvectors on exit
 *  report   may be NULL
 * Synchronous (returns after the eigenvalues reach the host).  Returns
 * NOT_CONVERGED (results of the last iteration are still written), NEG_STATE,
 * RANK, INVALID_ARG, OOM or CUDA. */
int dks_lobpcgf_solve(dks_ctx* ctx, int nev, double tol, const dks_solve_opts* opts,
                      double* eig, void* const* X, dks_solve_report* report);

/* ------------------------------------------- single steps of Algorithm 1
 * Exposed so that each step can be checked on its own.  Column blocks are
 * [ncol][rows] complex (rows = 4 npw for DKS vectors), device memory. */

/* Algorithm 1's preconditioning step with the residual fused: for i < nact, column
 * j = act[i] (device int[nact]):  Y[i] = K(x_G) (HX[j] - lam[j] X[j]) with the
 * Teter-Payne-Allan factor K(x) = P/(P + 16x^4), P = 27+18x+12x^2+8x^3,
 * x_G = (|k+G|^2/2)/T_j, T_j = sum |k+G|^2/2 |X[j]|^2 / sum |X[j]|^2 over all four
 * components (precond = IDENTITY: K = 1).  lam: device double[ncols of X]. */
int dks_precond(dks_ctx* ctx, int ik, const void* X, const void* HX, const double* lam,
                const int* act, int nact, void* Y, int precond, int prec, void* stream);

/* Algorithm 1's projected pencil: A = Z^H HZ and S = Z^H Z for
 * Z, HZ [nz][rows]; A, S device double2 (complex128) nz x nz, column-major,
 * every entry computed (no symmetry assumed).  prec FP64: FP64 arithmetic;
 * FP64_EMULATED: complex128 data, double-float arithmetic; FP32: complex64
 * data, FP32 products per 32-deep k-tile summed into double-float totals. */
int dks_gram(const void* Z, const void* HZ, int rows, int nz, void* A, void* S, int prec,
             void* stream);

/* The solver's form of Algorithm 1's projected pencil: the block lower triangles of A =
 * Z^H HZ and S = Z^H Z in one fused pass over Z and HZ, then each strict upper
 * triangle set to the conjugate transpose of the lower one (A is Hermitian when
 * HZ = H' Z).  Arguments and layout as dks_gram; on return A[j][i] (column j,
 * row i) for i >= j is the exact-arithmetic entry up to rounding and A[i][j] =
 * conj(A[j][i]).  prec FP32: complex64 blocks; FP64_EMULATED: complex128 blocks
 * split once into double-float copies (2 x 32 nz rows bytes of device memory
 * allocated and freed on the stream per call); FP64: complex128 blocks, FP64
 * arithmetic, two lower-triangle passes.  Returns INVALID_ARG, OOM or CUDA. */
int dks_gram_hermitian(const void* Z, const void* HZ, int rows, int nz, void* A, void* S, int prec,
                       void* stream);

/* Algorithm 1's Rayleigh-Ritz step on the device in FP64: the n lowest pairs of A v = lam S v
 * (after diagonal scaling; Cholesky of S, or SVQB with drop tolerance
 * 1e-12 * max eig when the smallest Cholesky pivot^2 < 1e-12).  A, S device
 * complex128 nz x nz column-major; V device complex128 nz x n column-major;
 * lam device double[n] ascending; info device int[3] = {used SVQB, rank, eigensolver
 * status}: info[2] is 0, or nonzero when the single-CTA fallback's tridiagonal QL did not
 * converge within its sweep limit (the results it had are still written).  All three ints
 * are written, so info must hold at least 3.  nz <= 512.  Returns INVALID_ARG, UNSUPPORTED,
 * CUDA. */
int dks_rayleigh_ritz(const void* A, const void* S, int nz, int n, void* V, double* lam,
                      int* info, void* stream);

/* Allocation-free variant of dks_rayleigh_ritz (the paper has no counterpart: it exists for
 * callers that may not allocate device memory when they need the solve, e.g. a service whose
 * device memory all belongs to its own arena after start-up, or a host thread that must not
 * risk the device-wide synchronisation a cudaMalloc/cudaFree can cause).  Same arguments,
 * layout and results as dks_rayleigh_ritz; its scratch space is one file-scope device array of
 * about 1.6 MB per device, held from library load until process exit.  Limit:
 * nz <= DKS_RR_STATIC_MAX_NZ, larger pencils return DKS_ERR_UNSUPPORTED.  The first call on
 * each device caches the array's device address, so make it before any stream capture.  Every
 * call on a device shares the array (each call overwrites it completely before use); calls
 * whose executions overlap on the GPU race on it and must be ordered by the caller.  The array
 * used is the one of the current device, so `stream` must belong to the current device
 * (checked: a stream of another device returns DKS_ERR_INVALID_ARG).  info is int[3] as for
 * dks_rayleigh_ritz.  Calls no cudaMalloc, cudaFree or other allocating routine. */
#define DKS_RR_STATIC_MAX_NZ 128
int dks_rayleigh_ritz_static(const void* A, const void* S, int nz, int n, void* V, double* lam,
                             int* info, void* stream);

/* Failure-detection test hook for the bounded waits of the Rayleigh-Ritz step (no counterpart in
 * the paper).  The per-column kernels of the device Rayleigh-Ritz step stage the Cholesky factor
 * and the reflectors into shared memory with TMA bulk copies and wait for them on an mbarrier
 * for at most first_wait_polls polls (default 1 << 24); a wait that gives up lets the copy land
 * (a second wait with the full limit), sets a flag in device memory, and the single-CTA kernel
 * redoes the whole step.  first_wait_polls = 0 makes every such wait give up at once, so that
 * this path runs on every step; restore 1 << 24 afterwards.  redone (may be NULL) receives the
 * number of steps redone that way since the previous call, and the count is cleared.
 * Process-wide, current device.  Synchronous.  Returns DKS_OK or DKS_ERR_CUDA. */
int dks_debug_rr_wait(unsigned first_wait_polls, unsigned* redone);

/* Tensor cores for the complex64 contractions (the FP32 phase of the mixed mode and DKS_PREC_FP32
 * blocks).  The tall-skinny contractions that Algorithm 1 and Eq. (HGH) reduce to -- the
 * rotations X <- Z V and P <- [0, Y, P] V, the Gram matrices of the Rayleigh-Ritz pencil, and
 * the projector coefficients B^H x~ and update x~ += B D (B^H x~) -- can run on the GB300's
 * fifth-generation tensor cores (tcgen05 MMA, TMA-staged operands) instead of the FP32 CUDA
 * cores.  Each FP32 value is split exactly into three bfloat16 slices and every product is
 * formed from the six leading slice products (left-out terms below 2^-24 of the product), with
 * FP32 accumulation in tensor memory; the Gram and B^H x~ forms split the long index into
 * chunks of at most kchunk rows per FP32 accumulation and add the chunk partials in FP64 in a
 * fixed order.  mask: DKS_TC_* bits (DKS_TC_DEFAULT at load); kchunk <= 0 keeps the current chunk
 * length (default 512).
 * Process-wide; a device other than a GB300 (sm_103) keeps the CUDA-core kernels.  Operands
 * that are not 16-byte aligned or have an odd leading dimension also take the CUDA-core path.
 * Returns DKS_OK. */
#define DKS_TC_ROTATE 1   /* X <- Z V, P <- [0, Y, P] V, projections of earlier band blocks */
#define DKS_TC_GRAM 2     /* S = Z^H Z, A = Z^H HZ (and the other FP32 A^H B Gram forms)    */
#define DKS_TC_PROJ_HN 4  /* projector coefficients B^H x~                                  */
#define DKS_TC_PROJ_NN 8  /* projector update x~ += B (D B^H x~)                            */
/* complex128 blocks in double-float precision (the FP64 refinement phase of the mixed mode,
 * DKS_PREC_FP64_EMULATED): the Gram matrices A = Z^H HZ, S = Z^H Z and the rotations X <- Z V,
 * P <- [0, Y, P] V from exact integer slices -- per 128-row window and column an exponent E with
 * |Re|, |Im| < 2^(E-1), every value rounded to 56 fractional bits of 2^E and cut into seven
 * 8-bit digits held as bfloat16; the 28 digit products of levels 0..6 accumulate on the tensor
 * cores level by level, exactly in FP32 for levels 0..3, and the window sums are added in
 * double-float and FP64 (error near 2^-50 of the window maxima per product, deterministic).
 * The blocks are sliced once per iteration and the slices serve both the Gram matrices and the
 * rotations. */
#define DKS_TC_FP64 16
#define DKS_TC_ALL 31
/* default: the projector contractions of complex64 blocks and the refinement phase's
 * contractions.  The complex64 rotations and Gram matrices stay on the CUDA cores: on the
 * tensor cores they raise the residual floor of the FP32 phase (the residual H X - X Lambda is
 * formed from separately rotated X and HX blocks and the negative continuum amplifies what
 * their rounding leaves), which costs more FP64 iterations than the contraction saves. */
#define DKS_TC_DEFAULT (DKS_TC_PROJ_HN | DKS_TC_PROJ_NN | DKS_TC_FP64)
int dks_tensor_cores(int mask, int kchunk);
/* the current mask and chunk length */
int dks_tensor_cores_get(int* mask, int* kchunk);

/* Algorithm 1's rotations (X <- Z V, P <- [0, Y, P] V): OUT[j] = sum_i Z[i] W[i + ldw*j] (+ beta OUT[j]) for
 * j < n, i < nz; Z [nz][rows], OUT [n][rows] (precision prec), W device
 * complex128 column-major with leading dimension ldw (converted to prec). */
int dks_rotate(const void* Z, int rows, int nz, const void* W, int ldw, int n, void* OUT,
               double beta, int prec, void* stream);

/* Algorithm 1's residual norms: norms[j] = ||HX[j] - lam[j] X[j]||_2.  The residual and the sum over the
 * components of a planewave are formed in the storage precision (DKS_PREC_FP32: FP32,
 * otherwise FP64); the sum over planewaves is accumulated in FP64.  rows even (4 npw for
 * DKS four-spinors, 2 npw for KSSO two-spinors). */
int dks_residual_norms(const void* X, const void* HX, const double* lam, int rows, int n,
                       double* norms, int prec, void* stream);

/* ------------------------------------------------ self-consistent field (Sec. 2.1, Sec. 4.1)
 * The SCF loop around the eigensolver: density of the occupied states, Hartree and LDA
 * exchange-correlation potential, Anderson mixing with the Kerker preconditioner.
 * Grids are FP64 device arrays of Ng = N1 N2 N3 values f[(i1*N2 + i2)*N3 + i3] at
 * r = sum_i (i_i/N_i) a_i, the layout of dks_potentials::v_r; the caller owns them.  Along an
 * axis of length N, grid frequency index m stands for the signed integer m - N when 2m >= N
 * (the Nyquist index counts as -N/2), and G = m1 b1 + m2 b2 + m3 b3. */

/* dks_density: rho += sum_{j < nb} occ[j] psi_j(r)^dag psi_j(r) on the grid (Eq. density with
 * the magnetisation term dropped), psi_j(r) = vol^-1/2 sum_G X[j][comp][G] exp(i (k+G).r),
 * summed over the dks_ncomp(ctx) components.  X: device complex128 [nb][ncomp][npw] of k-point
 * ik; occ: host double[nb]; rho: device double[Ng], accumulated (zero it first; call once per
 * k-point with occ holding the k-point weights for a k-point sum).  FP64 transforms.  Uses
 * ctx workspace (not reentrant per ctx).  Errors: INVALID_ARG, UNSUPPORTED (plane too large
 * for shared memory), OOM, CUDA. */
int dks_density(dks_ctx* ctx, int ik, const void* X, int nb, const double* occ, double* rho, void* stream);

/* dks_hxc: vhxc = V_H + v_xc of the density rho (the Hartree-exchange-correlation potential of
 * Sec. 2.1).  V_H(G) = 4 pi rho(G) / |G|^2 for G != 0 and V_H(0) = 0 (a neutralising uniform
 * background), rho(G) the Fourier coefficients of rho on the grid; v_xc the spin-unpolarised
 * LDA: Dirac exchange plus the Perdew-Zunger (1981) fit of the Ceperley-Alder correlation;
 * grid points with rho <= 1e-30 get v_xc = 0.  rho, vhxc: device double[Ng], distinct.
 * energies: host double[2] = {E_H = 1/2 int rho V_H, E_xc = int rho eps_xc}, or NULL; when
 * given, the call synchronises `stream`.  Errors: INVALID_ARG, OOM, CUDA. */
int dks_hxc(dks_ctx* ctx, const double* rho, double* vhxc, double* energies, void* stream);

/* dks_set_potential: the context's local potential V(r) becomes v (device double[Ng], Ha) for
 * every later dks_apply_H, dks_filter and solve; the default filter constants follow the new
 * max|V| (dks_filter_constants).  The potential given at creation stays the context's
 * external part for dks_scf.  Synchronous.  Errors: INVALID_ARG, OOM, CUDA. */
int dks_set_potential(dks_ctx* ctx, const double* v, void* stream);

/* dks_update_potential: the SCF step V = V_loc + V_hxc(rho) in one call: dks_hxc of rho (device
 * double[Ng]) plus the potential given at creation (V_loc; zero if none), made the context's
 * potential as by dks_set_potential.  rho = NULL sets V = V_loc (the SCF's first potential).
 * energies: host double[2] = {E_H, E_xc} of rho (zeros for rho = NULL), or NULL.  Synchronous.
 * Errors: INVALID_ARG, OOM, CUDA. */
int dks_update_potential(dks_ctx* ctx, const double* rho, double* energies, void* stream);

/* dks_density_residual: *out = int |a - b| dr = (vol / Ng) sum_n |a_n - b_n| for two device
 * grids (the SCF convergence measure, in electrons).  Synchronous.  Errors: INVALID_ARG, CUDA. */
int dks_density_residual(dks_ctx* ctx, const double* a, const double* b, double* out, void* stream);

/* Anderson mixer of densities with the Kerker preconditioner (Sec. 4.1).  One step, given the
 * input density rho_in of the last potential and the output density rho_out of its solve:
 *   F = rho_out - rho_in; with the stored differences dR_j, dF_j of the last `history` steps,
 *   gamma = argmin_g |F - sum_j g_j dF_j|_2 (plain sum over grid points; directions whose
 *   singular value is below 1e-6 of the largest are left out),
 *   rho_next = rho_in - sum_j gamma_j dR_j + P (F - sum_j gamma_j dF_j),
 *   P: each Fourier component times alpha |G|^2 / (|G|^2 + q0^2) (0 at G = 0),
 * then (rho_in - previous rho_in, F - previous F) joins the history.  history = 0 gives
 * Kerker-preconditioned linear mixing.  0 <= history <= 16, alpha > 0, q0 >= 0. */
typedef struct dks_mixer dks_mixer;
int dks_mixer_create(dks_ctx* ctx, int history, double alpha, double q0, dks_mixer** out);
/* rho_in, rho_out, rho_next: device double[Ng]; rho_next may be rho_in, not rho_out.
 * Synchronous (the small least-squares problem is solved on the host).  The mixer keeps its
 * own device copies of the history.  Errors: INVALID_ARG, OOM, CUDA. */
int dks_mix(dks_mixer* mixer, const double* rho_in, const double* rho_out, double* rho_next, void* stream);
void dks_mixer_destroy(dks_mixer* mixer);

typedef struct {
  int nocc;            /* occupied states per k-point, one electron each (k-points weighted
                          1/nk); nocc <= nev_k                                          */
  int max_iter;        /* SCF iterations after the first solve (default 60)             */
  double tol;          /* stop when int |rho_out - rho_in| dr < tol electrons (1e-8)    */
  double alpha;        /* Kerker-Anderson mixing: alpha (0.5), q0 in 1/bohr (1.0),       */
  double kerker_q0;    /*   history (8)                                                  */
  int history;
  int n_init_warm;     /* N_init of the solves after the first (warm start from the
                          previous eigenvectors, default 1)                              */
  double solve_tol;    /* residual tolerance of every eigensolve (1e-8)                  */
  dks_solve_opts solve;/* options of the eigensolves (dks_solve_opts_default); its
                          n_init is the first solve's                                    */
} dks_scf_opts;

typedef struct {
  int iterations;            /* SCF iterations after the first solve                     */
  int converged;
  double residual;           /* int |rho_out - rho_in| dr of the last iteration           */
  double e_h, e_xc;          /* Hartree and xc energies of the last input density (Ha)    */
  long long solve_iterations;/* eigensolver iterations, all solves and k-points           */
  long long h_applications;  /* single-band H' applications, all solves                   */
  double seconds;            /* wall time of the call                                     */
  int status;                /* DKS_OK or the first error                                 */
  int hist_len;
  double res_history[128];   /* residual after each SCF iteration                         */
} dks_scf_report;

void dks_scf_opts_default(dks_scf_opts* opts);

/* dks_scf: the SCF loop.  The first solve uses the potential given at creation (V_loc);
 * then, until the residual is below tol or max_iter is reached:
 *   V = V_loc + V_hxc(rho_in) (dks_hxc), solve for nev_k pairs per k (warm start),
 *   rho_out = density of the nocc lowest (dks_density), residual, rho_in = mix(rho_in, rho_out);
 * the first rho_in is the density of the first solve.
 *  eig   host double[sum_k nev_k]: the last solve's eigenvalues (shifted as dks_lobpcgf_solve)
 *  X     as dks_lobpcgf_solve (start block in, last eigenvectors out)
 *  rho   device double[Ng] for the last rho_out, or NULL
 * On return the context's potential is the last V (dks_set_potential).  Synchronous.
 * Returns NOT_CONVERGED when max_iter ends the loop (results of the last iteration are
 * written), or the first error of a step; an eigensolve that ends NOT_CONVERGED does not stop
 * the loop. */
int dks_scf(dks_ctx* ctx, int nev, const dks_scf_opts* opts, double* eig, void* const* X, double* rho,
            dks_scf_report* report);

/* ------------------------------------------------ launch-parameter tuning (no counterpart in the
 * paper, whose code ran on CPUs).  Three parameters of this implementation's H' application:
 * the byte budget of one chunk of FFT intermediates (default 64 MB: how many bands' stick
 * buffers stay resident in L2 between the three FFT passes), the CTA size of the one-kernel
 * plane FFT (0 = from the FFT plan: two butterflies per thread and pass), and plane_split: 1 runs
 * the plane FFT as row and column kernels through an L2-resident plane buffer (always the case
 * for planes above one CTA's shared memory, N1 (N2 | 1) x 16 bytes > 227 KB for complex128).
 * Results never depend on them (every line transform is the same arithmetic); only the time
 * does.  Not reentrant per ctx (do not tune during a solve). */
typedef struct {
  int ncand;                  /* candidates timed                                     */
  int best;                   /* index of the fastest                                 */
  long long chunk_bytes[32];
  int plane_threads[32];
  int plane_split[32];
  double ms[32];              /* mean time of one H' application on the nb columns     */
  int proj_tc;                /* contraction schedule chosen for the projector terms of
                                 complex64 blocks: 0 CUDA cores, 1 tensor cores; -1 when not
                                 tuned (prec other than FP32, no projectors, not a GB300)  */
  double proj_ms[2];          /* H' time with each (at the chosen FFT parameters)       */
} dks_tune_report;
/* dks_autotune: times dks_apply_H on an nb-column scratch block of k-point ik in precision
 * prec (device memory allocated and freed on `stream`) for chunk budgets {16, 32, 64, 128} MB
 * x {one-kernel plane FFT with CTA sizes {plan, 128, 256, 512} (where the plane fits), split
 * plane FFT}, one warm-up and three timed applications each (CUDA events on `stream`), and keeps
 * the fastest.  Synchronous.  On error the previous parameters stay.  report may be NULL.
 * Errors: INVALID_ARG, OOM, CUDA. */
int dks_autotune(dks_ctx* ctx, int ik, int nb, int prec, void* stream, dks_tune_report* report);
/* Current parameters, and setting stored ones: 1 MB <= fft_chunk_bytes <= 64 GB; plane_threads 0
 * or a multiple of 32 in 64..512; plane_split 0 or 1.  Errors: INVALID_ARG. */
int dks_tune_get(const dks_ctx* ctx, long long* fft_chunk_bytes, int* plane_threads, int* plane_split);
int dks_tune_set(dks_ctx* ctx, long long fft_chunk_bytes, int plane_threads, int plane_split);
/* The context's contraction schedule for the projector terms of complex64 blocks (Eq. HGH:
 * B^H x~ and x~ += B D (B^H x~)): -1 follows the process-wide dks_tensor_cores mask (the
 * default), 0 the CUDA-core kernels, 1 the tcgen05 tensor-core kernels.  dks_autotune with
 * prec FP32 times both and sets it. */
int dks_tune_contractions_get(const dks_ctx* ctx, int* proj_tc);
int dks_tune_contractions_set(dks_ctx* ctx, int proj_tc);

/* ------------------------------------------------ instrumentation (no counterpart in the paper;
 * the solve report's phase timers of a production code).  Every kernel launch of the library is
 * counted per category; while profiling is enabled each launch is also bracketed by a CUDA event
 * pair on its own stream and tagged with its algorithmic bytes and flops (the minimum traffic and
 * work the launch must do, see the kernel comments).  Process-wide, thread-safe. */
int dks_profile_ncat(void);
const char* dks_profile_name(int cat);
/* enable (1) or disable (0) event recording; clears all counters and records */
int dks_profile_enable(int on);
/* synchronises the device, then per category c < ncat: ms[c] = summed event time,
 * launches[c], bytes[c], flops[c]; clears.  ncat must be >= dks_profile_ncat(). */
int dks_profile_read(int ncat, double* ms, long long* launches, double* bytes, double* flops);

/* dks_debug_check: *compiled = 1 in the debug build (libdks_debug.so, built with
 * `python -m paper_1211_1446_gb300.build --debug`), whose FFT kernels check every sphere <-> grid
 * and plane index before using it; *code = the first failed check since the last call (kernel
 * in the top byte: 1 stick inverse, 2 stick forward, 3 stick forward KSSO, 4 plane, 5 plane of
 * the density, 6 density gather; the item index in the low 24 bits), 0 when none, then cleared
 * (synchronises the device).  A failed check skips its access, so the results are wrong but no
 * memory outside the buffers is touched.  In the product build *compiled = 0, *code = 0 and no
 * device call is made. */
int dks_debug_check(int* compiled, unsigned* code);

const char* dks_strerror(int code);
const char* dks_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DKS_H */

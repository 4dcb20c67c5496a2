// Self-consistent field loop around the eigensolver (Sec. 2.1, DKS equations; Sec. 4.1, setup).
//
//   rho(r)  = sum_k w_k sum_{i occupied} psi_ik(r)^dag psi_ik(r)           Eq. (density), B_xc = 0
//   V_hxc   = V_H + v_xc,  V_H(G) = 4 pi rho(G) / |G|^2 (G != 0),             Sec. 2.1
//             v_xc the unpolarised LDA (Dirac exchange + Perdew-Zunger 1981 correlation)
//   mixing  Anderson with the Kerker preconditioner                          Sec. 4.1
//
// GPU design.  The density reuses the stick/plane inverse FFT of H' x (hx_kernels.cu) and sums
// |psi|^2 in shared memory.  Everything else works on the full N1 x N2 x N3 grid in FP64: the
// transforms of the density and of the mixing residual are direct DFTs along one axis at a time
// (one CTA per line, N <= 256, a few hundred MFLOP for the largest grids -- once per SCF
// iteration, against seconds of eigensolver work), the reciprocal-space factors and the LDA are
// one thread per grid point, reductions end in one atomic per warp.  The least-squares problem
// of the Anderson step (at most 16 unknowns) is solved on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "dks_internal.h"
#include "dks_kernels.cuh"

namespace dks {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxHistory = 16;
constexpr int kMaxPairs = kMaxHistory * (kMaxHistory + 1) / 2 + kMaxHistory;

struct Recip {
  double b[9];   // rows b1, b2, b3
};

__device__ __forceinline__ int signed_freq(int m, int n) { return 2 * m >= n ? m - n : m; }

__device__ __forceinline__ double warp_sum(double a) {
  for (int o = 16; o; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
  return a;
}

// direct DFT along one axis of a complex grid [n1][n2][n3], in place:
//   out[j] = sum_t in[t] w^(j t),  w = exp(-2 pi i / N) (fwd) or exp(+2 pi i / N)
// one CTA per line; tw[t] = exp(+2 pi i t / N)
__global__ void __launch_bounds__(128) k_dft_axis(double2* __restrict__ g, int n1, int n2, int n3, int axis,
                                                  const double2* __restrict__ tw, int fwd) {
  __shared__ double2 line[kMaxFftLen];
  const int n = axis == 0 ? n1 : axis == 1 ? n2 : n3;
  const int l = blockIdx.x;
  size_t base, stride;
  if (axis == 2) {
    base = (size_t)l * n3;
    stride = 1;
  } else if (axis == 1) {
    const int i1 = l / n3, i3 = l - i1 * n3;
    base = (size_t)i1 * n2 * n3 + i3;
    stride = n3;
  } else {
    base = l;
    stride = (size_t)n2 * n3;
  }
  for (int t = threadIdx.x; t < n; t += blockDim.x) line[t] = g[base + t * stride];
  __syncthreads();
  const double sgn = fwd ? -1.0 : 1.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double sr = 0.0, si = 0.0;
    int idx = 0;   // (j t) mod n
    for (int t = 0; t < n; ++t) {
      const double2 w = tw[idx];
      const double wi = sgn * w.y;
      const double2 v = line[t];
      sr = fma(v.x, w.x, fma(-v.y, wi, sr));
      si = fma(v.x, wi, fma(v.y, w.x, si));
      idx += j;
      if (idx >= n) idx -= n;
    }
    g[base + j * stride] = double2{sr, si};
  }
}

__global__ void k_real_to_complex(const double* __restrict__ r, double2* __restrict__ g, size_t ng) {
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < ng; n += (size_t)gridDim.x * blockDim.x)
    g[n] = double2{r[n], 0.0};
}

// g(G) *= scale * factor(G); mode 0: Hartree 4 pi / |G|^2 (0 at G = 0),
// mode 1: Kerker alpha |G|^2 / (|G|^2 + q0^2) (0 at G = 0)
__global__ void k_gfactor(double2* __restrict__ g, int n1, int n2, int n3, Recip rb, int mode, double alpha,
                          double q0sq, double scale) {
  const size_t ng = (size_t)n1 * n2 * n3;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < ng; n += (size_t)gridDim.x * blockDim.x) {
    const int i3 = (int)(n % n3);
    const size_t r = n / n3;
    const int i2 = (int)(r % n2), i1 = (int)(r / n2);
    const double m1 = signed_freq(i1, n1), m2 = signed_freq(i2, n2), m3 = signed_freq(i3, n3);
    const double gx = m1 * rb.b[0] + m2 * rb.b[3] + m3 * rb.b[6];
    const double gy = m1 * rb.b[1] + m2 * rb.b[4] + m3 * rb.b[7];
    const double gz = m1 * rb.b[2] + m2 * rb.b[5] + m3 * rb.b[8];
    const double g2 = gx * gx + gy * gy + gz * gz;
    double f = 0.0;
    if (g2 > 0.0) f = mode == 0 ? 4.0 * kPi / g2 : alpha * g2 / (g2 + q0sq);
    const double s = f * scale;
    g[n] = double2{g[n].x * s, g[n].y * s};
  }
}

// LDA, spin-unpolarised, in Hartree.  Exchange of the uniform gas, eps_x = -(3/4)(9/(4 pi^2))^(1/3)
// / r_s (the constant is 0.75 (9 / (4 pi^2))^(1/3)), v_x = 4/3 eps_x; correlation: the
// Perdew-Zunger (1981) fit of the Ceperley-Alder energies, v_c = eps_c - (r_s/3) d eps_c/d r_s.
struct XC {
  double eps, v;
};
__device__ __forceinline__ XC lda_pz81(double rho) {
  if (!(rho > 1e-30)) return XC{0.0, 0.0};
  const double rs = cbrt(3.0 / (4.0 * kPi * rho));
  const double ex = -0.4581652932831429 / rs;
  const double vx = (4.0 / 3.0) * ex;
  double ec, vc;
  if (rs < 1.0) {
    const double A = 0.0311, B = -0.048, C = 0.0020, D = -0.0116;
    const double lr = log(rs);
    ec = A * lr + B + C * rs * lr + D * rs;
    vc = ec - rs / 3.0 * (A / rs + C * lr + C + D);
  } else {
    const double gam = -0.1423, b1 = 1.0529, b2 = 0.3334;
    const double sq = sqrt(rs);
    const double den = 1.0 + b1 * sq + b2 * rs;
    ec = gam / den;
    vc = ec + rs / 3.0 * gam * (0.5 * b1 / sq + b2) / (den * den);
  }
  return XC{ex + ec, vx + vc};
}

// vhxc = Re(vh) + v_xc(rho); esum += {sum rho Re(vh), sum max(rho, 0) eps_xc}
__global__ void k_hxc_finish(const double* __restrict__ rho, const double2* __restrict__ vh,
                             double* __restrict__ vhxc, double* __restrict__ esum, size_t ng) {
  double eh = 0.0, exc = 0.0;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < ng; n += (size_t)gridDim.x * blockDim.x) {
    const double r = rho[n];
    const XC x = lda_pz81(r);
    const double v = vh[n].x;
    vhxc[n] = v + x.v;
    eh = fma(r, v, eh);
    exc = fma(fmax(r, 0.0), x.eps, exc);
  }
  eh = warp_sum(eh);
  exc = warp_sum(exc);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(esum, eh);
    atomicAdd(esum + 1, exc);
  }
}

// vperm[(p3[i3] N1 + p1[i1]) LD + p2[i2]] = v / Ng (FP64, FP32, double-float); max |v| as bits
__global__ void k_set_vperm(const double* __restrict__ v, int n1, int n2, int n3, int ld, const int* __restrict__ p1,
                            const int* __restrict__ p2, const int* __restrict__ p3, double ng_d,
                            double* __restrict__ vp64, float* __restrict__ vp32, float2* __restrict__ vpdf,
                            unsigned long long* __restrict__ vmax_bits) {
  const size_t ng = (size_t)n1 * n2 * n3;
  double m = 0.0;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < ng; n += (size_t)gridDim.x * blockDim.x) {
    const int i3 = (int)(n % n3);
    const size_t r = n / n3;
    const int i2 = (int)(r % n2), i1 = (int)(r / n2);
    const size_t at = ((size_t)p3[i3] * n1 + p1[i1]) * ld + p2[i2];
    const double d = v[n] / ng_d;
    vp64[at] = d;
    vp32[at] = (float)d;
    const float h = (float)d;
    vpdf[at] = float2{h, (float)(d - (double)h)};
    m = fmax(m, fabs(v[n]));
  }
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  // non-negative doubles order like their bit patterns
  if ((threadIdx.x & 31) == 0) atomicMax(vmax_bits, (unsigned long long)__double_as_longlong(m));
}

__global__ void k_axpy_grid(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out,
                            size_t ng) {
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < ng; n += (size_t)gridDim.x * blockDim.x)
    out[n] = a[n] + b[n];
}

// sum |a - b|
__global__ void k_absdiff_sum(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out,
                              size_t ng) {
  double s = 0.0;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < ng; n += (size_t)gridDim.x * blockDim.x)
    s += fabs(a[n] - b[n]);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

// ---------------------------------------------------------------- Anderson mixer kernels
// F = rho_out - rho_in; with a previous step: dR = rho_in - prev_in, dF = F - prev_F (into the
// history slot); then prev_in = rho_in, prev_F = F
__global__ void k_mix_prepare(const double* __restrict__ rin, const double* __restrict__ rout,
                              double* __restrict__ prev_in, double* __restrict__ prev_f, double* __restrict__ dr,
                              double* __restrict__ df, int has_prev, size_t ng) {
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < ng; n += (size_t)gridDim.x * blockDim.x) {
    const double ri = rin[n];
    const double f = rout[n] - ri;
    if (has_prev) {
      dr[n] = ri - prev_in[n];
      df[n] = f - prev_f[n];
    }
    prev_in[n] = ri;
    prev_f[n] = f;
  }
}

struct Pairs {
  int a[kMaxPairs], b[kMaxPairs];   // vector index: history slot, or -1 for F
};

// dots[p] += <v_a[p], v_b[p]> over the grid, one pair per blockIdx.y
__global__ void k_dots(const double* __restrict__ hist, const double* __restrict__ f, Pairs pr, size_t ng,
                       double* __restrict__ dots) {
  const int p = blockIdx.y;
  const double* x = pr.a[p] < 0 ? f : hist + (size_t)pr.a[p] * ng;
  const double* y = pr.b[p] < 0 ? f : hist + (size_t)pr.b[p] * ng;
  double s = 0.0;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < ng; n += (size_t)gridDim.x * blockDim.x)
    s = fma(x[n], y[n], s);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) atomicAdd(dots + p, s);
}

struct Gamma {
  double g[kMaxHistory];
};

// rho_next = rho_in - sum_j g_j dR_j;  cg = (F - sum_j g_j dF_j, 0)
__global__ void k_mix_combine(const double* __restrict__ rin, const double* __restrict__ f,
                              const double* __restrict__ dr, const double* __restrict__ df, int nh, Gamma gm,
                              size_t ng, double* rnext, double2* __restrict__ cg) {
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < ng; n += (size_t)gridDim.x * blockDim.x) {
    double r = rin[n], e = f[n];
#pragma unroll
    for (int j = 0; j < kMaxHistory; ++j) {   // fixed trip count keeps gm in registers
      if (j < nh) {
        r = fma(-gm.g[j], dr[(size_t)j * ng + n], r);
        e = fma(-gm.g[j], df[(size_t)j * ng + n], e);
      }
    }
    rnext[n] = r;
    cg[n] = double2{e, 0.0};
  }
}

__global__ void k_add_real(double* __restrict__ r, const double2* __restrict__ cg, size_t ng) {
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < ng; n += (size_t)gridDim.x * blockDim.x)
    r[n] += cg[n].x;
}

int grid_blocks(const dks_ctx* ctx, size_t ng) {
  return (int)std::max<size_t>(1, std::min<size_t>((ng + 255) / 256, (size_t)ctx->num_sms * 8));
}

// g -> sum over the grid of g exp(-+ i G.r): three axis passes
int dft3(dks_ctx* ctx, double2* g, bool fwd, cudaStream_t st) {
  const int n1 = ctx->grid[0], n2 = ctx->grid[1], n3 = ctx->grid[2];
  const size_t ng = (size_t)ctx->ng;
  for (int a = 0; a < 3; ++a) {
    const int axis = fwd ? 2 - a : a;
    const int n = ctx->grid[axis];
    Prof pr(P_SCF, st, 32.0 * ng, 8.0 * ng * n);
    k_dft_axis<<<(unsigned)(ng / n), 128, 0, st>>>(g, n1, n2, n3, axis, ctx->tw64[axis], fwd ? 1 : 0);
  }
  DKS_CUDA_TRY(cudaGetLastError());
  return DKS_OK;
}

Recip recip_of(const dks_ctx* ctx) {
  Recip r;
  std::memcpy(r.b, ctx->recip, sizeof(r.b));
  return r;
}

// symmetric eigen-decomposition by cyclic Jacobi rotations (n <= 16): a (row-major n x n) is
// destroyed, w gets the eigenvalues, v (row-major) the eigenvectors as columns
void jacobi_eig(std::vector<double>& a, int n, std::vector<double>& w, std::vector<double>& v) {
  v.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) v[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const double x = a[(size_t)i * n + j] * a[(size_t)i * n + j];
        tot += x;
        if (i != j) off += x;
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = a[(size_t)p * n + q];
        if (apq == 0.0) continue;
        const double th = (a[(size_t)q * n + q] - a[(size_t)p * n + p]) / (2.0 * apq);
        const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {   // columns p, q
          const double akp = a[(size_t)k * n + p], akq = a[(size_t)k * n + q];
          a[(size_t)k * n + p] = c * akp - s * akq;
          a[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {   // rows p, q
          const double apk = a[(size_t)p * n + k], aqk = a[(size_t)q * n + k];
          a[(size_t)p * n + k] = c * apk - s * aqk;
          a[(size_t)q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = v[(size_t)k * n + p], vkq = v[(size_t)k * n + q];
          v[(size_t)k * n + p] = c * vkp - s * vkq;
          v[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = a[(size_t)i * n + i];
}

}  // namespace

// vhxc = V_H + v_xc of rho; esum_dev (2 doubles, device) receives {sum rho V_H, sum rho eps_xc}
static int hxc_potential(dks_ctx* ctx, const double* rho, double* vhxc, double2* cg, double* esum_dev, cudaStream_t st) {
  const size_t ng = (size_t)ctx->ng;
  const int blocks = grid_blocks(ctx, ng);
  {
    Prof pr(P_SCF, st, 24.0 * ng, 0.0);
    k_real_to_complex<<<blocks, 256, 0, st>>>(rho, cg, ng);
  }
  DKS_TRY(dft3(ctx, cg, true, st));
  {
    Prof pr(P_SCF, st, 32.0 * ng, 12.0 * ng);
    k_gfactor<<<blocks, 256, 0, st>>>(cg, ctx->grid[0], ctx->grid[1], ctx->grid[2], recip_of(ctx), 0, 0.0, 0.0,
                                      1.0 / (double)ng);
  }
  DKS_TRY(dft3(ctx, cg, false, st));
  DKS_CUDA_TRY(cudaMemsetAsync(esum_dev, 0, 2 * sizeof(double), st));
  {
    Prof pr(P_SCF, st, 32.0 * ng, 40.0 * ng);
    k_hxc_finish<<<blocks, 256, 0, st>>>(rho, cg, vhxc, esum_dev, ng);
  }
  DKS_CUDA_TRY(cudaGetLastError());
  return DKS_OK;
}

static int set_potential(dks_ctx* ctx, const double* v, cudaStream_t st) {
  const int n1 = ctx->grid[0], n2 = ctx->grid[1], n3 = ctx->grid[2], ld = ctx->plane_ld;
  const size_t nvp = (size_t)n3 * n1 * ld;
  if (!ctx->vperm64) {
    DKS_CUDA_TRY(cudaMalloc((void**)&ctx->vperm64, nvp * sizeof(double)));
    DKS_CUDA_TRY(cudaMalloc((void**)&ctx->vperm32, nvp * sizeof(float)));
    DKS_CUDA_TRY(cudaMalloc((void**)&ctx->vpermdf, nvp * sizeof(float2)));
    DKS_CUDA_TRY(cudaMemsetAsync(ctx->vperm64, 0, nvp * sizeof(double), st));   // padding column stays 0
    DKS_CUDA_TRY(cudaMemsetAsync(ctx->vperm32, 0, nvp * sizeof(float), st));
    DKS_CUDA_TRY(cudaMemsetAsync(ctx->vpermdf, 0, nvp * sizeof(float2), st));
  }
  unsigned long long* vmax_dev = nullptr;
  DKS_CUDA_TRY(cudaMallocAsync((void**)&vmax_dev, sizeof(unsigned long long), st));
  DKS_CUDA_TRY(cudaMemsetAsync(vmax_dev, 0, sizeof(unsigned long long), st));
  const size_t ng = (size_t)ctx->ng;
  {
    Prof pr(P_SCF, st, 8.0 * ng + 14.0 * ng, 2.0 * ng);
    k_set_vperm<<<grid_blocks(ctx, ng), 256, 0, st>>>(v, n1, n2, n3, ld, ctx->posd[0], ctx->posd[1], ctx->posd[2],
                                                       (double)ng, ctx->vperm64, ctx->vperm32, ctx->vpermdf,
                                                       vmax_dev);
  }
  unsigned long long bits = 0;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, vmax_dev, sizeof(bits), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(vmax_dev, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(DKS_ERR_CUDA, std::string("set_potential: ") + cudaGetErrorString(e));
  double vmax;
  std::memcpy(&vmax, &bits, sizeof(vmax));
  ctx->vmax = vmax;
  ctx->has_v = true;
  // default filter constants follow max|V| (C does not depend on V)
  const double c = ctx->c;
  for (KPoint& kp : ctx->k) {
    const double emax = -2.0 * kp.cshift - 3.0 * c * c;
    kp.omega = (emax - c * c) + ctx->vmax + ctx->dsum - kp.cshift;
  }
  return DKS_OK;
}

}  // namespace dks

using namespace dks;

struct dks_mixer {
  dks_ctx* ctx = nullptr;
  int m = 0;
  double alpha = 0.5, q0 = 1.0;
  int nh = 0, next = 0;
  bool has_prev = false;
  double* dr = nullptr;       // m x Ng
  double* df = nullptr;       // m x Ng
  double* prev_in = nullptr;  // Ng
  double* prev_f = nullptr;   // Ng: F of the latest step
  double2* cg = nullptr;      // Ng complex work grid
  double* dots = nullptr;     // kMaxPairs
};

void dks_mixer_destroy(dks_mixer* mx) {
  if (!mx) return;
  cudaFree(mx->dr);
  cudaFree(mx->df);
  cudaFree(mx->prev_in);
  cudaFree(mx->prev_f);
  cudaFree(mx->cg);
  cudaFree(mx->dots);
  delete mx;
}

int dks_mixer_create(dks_ctx* ctx, int history, double alpha, double q0, dks_mixer** out) {
  if (!out) return fail(DKS_ERR_INVALID_ARG, "dks_mixer_create: out is NULL");
  *out = nullptr;
  if (!ctx || history < 0 || history > kMaxHistory || !(alpha > 0) || !(q0 >= 0) || !std::isfinite(alpha) ||
      !std::isfinite(q0))
    return fail(DKS_ERR_INVALID_ARG, "dks_mixer_create: need 0 <= history <= 16, alpha > 0, q0 >= 0");
  dks_mixer* mx = new (std::nothrow) dks_mixer();
  if (!mx) return fail(DKS_ERR_OOM, "host allocation");
  mx->ctx = ctx;
  mx->m = history;
  mx->alpha = alpha;
  mx->q0 = q0;
  const size_t ng = (size_t)ctx->ng;
  cudaError_t e = cudaSuccess;
  if (history) {
    e = cudaMalloc((void**)&mx->dr, (size_t)history * ng * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&mx->df, (size_t)history * ng * sizeof(double));
  }
  if (e == cudaSuccess) e = cudaMalloc((void**)&mx->prev_in, ng * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&mx->prev_f, ng * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&mx->cg, ng * sizeof(double2));
  if (e == cudaSuccess) e = cudaMalloc((void**)&mx->dots, kMaxPairs * sizeof(double));
  if (e != cudaSuccess) {
    dks_mixer_destroy(mx);
    return fail(e == cudaErrorMemoryAllocation ? DKS_ERR_OOM : DKS_ERR_CUDA,
                std::string("dks_mixer_create: ") + cudaGetErrorString(e));
  }
  *out = mx;
  return DKS_OK;
}

int dks_mix(dks_mixer* mx, const double* rho_in, const double* rho_out, double* rho_next, void* stream) {
  if (!mx || !rho_in || !rho_out || !rho_next || rho_next == rho_out)
    return fail(DKS_ERR_INVALID_ARG, "dks_mix: bad argument (rho_next may alias rho_in only)");
  dks_ctx* ctx = mx->ctx;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t ng = (size_t)ctx->ng;
  const int blocks = grid_blocks(ctx, ng);
  const bool add = mx->has_prev && mx->m > 0;
  const int slot = mx->next;
  {
    Prof pr(P_SCF, st, (add ? 7.0 : 4.0) * 8.0 * ng, 3.0 * ng);
    k_mix_prepare<<<blocks, 256, 0, st>>>(rho_in, rho_out, mx->prev_in, mx->prev_f,
                                          add ? mx->dr + (size_t)slot * ng : nullptr,
                                          add ? mx->df + (size_t)slot * ng : nullptr, add ? 1 : 0, ng);
  }
  DKS_CUDA_TRY(cudaGetLastError());
  if (add) {
    mx->next = (mx->next + 1) % mx->m;
    mx->nh = std::min(mx->nh + 1, mx->m);
  }
  mx->has_prev = true;
  const int nh = mx->nh;
  Gamma gm;
  for (int j = 0; j < kMaxHistory; ++j) gm.g[j] = 0.0;
  if (nh > 0) {
    // Gram matrix of the dF_j and right-hand side <dF_j, F>
    Pairs pr;
    int np = 0;
    for (int i = 0; i < nh; ++i)
      for (int j = i; j < nh; ++j) {
        pr.a[np] = i;
        pr.b[np++] = j;
      }
    for (int i = 0; i < nh; ++i) {
      pr.a[np] = i;
      pr.b[np++] = -1;
    }
    DKS_CUDA_TRY(cudaMemsetAsync(mx->dots, 0, np * sizeof(double), st));
    {
      Prof p(P_SCF, st, 16.0 * ng * np, 2.0 * ng * np);
      const int bx = std::max(1, std::min(blocks, (4 * ctx->num_sms + np - 1) / np));
      k_dots<<<dim3(bx, np), 256, 0, st>>>(mx->df, mx->prev_f, pr, ng, mx->dots);
    }
    DKS_CUDA_TRY(cudaGetLastError());
    std::vector<double> h(np);
    DKS_CUDA_TRY(cudaMemcpyAsync(h.data(), mx->dots, np * sizeof(double), cudaMemcpyDeviceToHost, st));
    DKS_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<double> a((size_t)nh * nh), rhs(nh), w, v;
    int k = 0;
    for (int i = 0; i < nh; ++i)
      for (int j = i; j < nh; ++j) {
        a[(size_t)i * nh + j] = a[(size_t)j * nh + i] = h[k++];
      }
    for (int i = 0; i < nh; ++i) rhs[i] = h[k++];
    // least squares through the normal equations, pseudo-inverse: eigenvalues of the Gram
    // matrix below 1e-12 of the largest (singular values below 1e-6) are left out
    jacobi_eig(a, nh, w, v);
    double wmax = 0.0;
    for (double x : w) wmax = std::max(wmax, x);
    for (int l = 0; l < nh; ++l) {
      if (!(w[l] > 1e-12 * wmax)) continue;
      double c = 0.0;
      for (int i = 0; i < nh; ++i) c += v[(size_t)i * nh + l] * rhs[i];
      c /= w[l];
      for (int i = 0; i < nh; ++i) gm.g[i] += c * v[(size_t)i * nh + l];
    }
  }
  {
    Prof pr(P_SCF, st, (2.0 + 2.0 * nh) * 8.0 * ng + 24.0 * ng, 4.0 * nh * ng);
    k_mix_combine<<<blocks, 256, 0, st>>>(rho_in, mx->prev_f, mx->dr, mx->df, nh, gm, ng, rho_next, mx->cg);
  }
  DKS_TRY(dft3(ctx, mx->cg, true, st));
  {
    Prof pr(P_SCF, st, 32.0 * ng, 12.0 * ng);
    k_gfactor<<<blocks, 256, 0, st>>>(mx->cg, ctx->grid[0], ctx->grid[1], ctx->grid[2], recip_of(ctx), 1,
                                      mx->alpha, mx->q0 * mx->q0, 1.0 / (double)ng);
  }
  DKS_TRY(dft3(ctx, mx->cg, false, st));
  {
    Prof pr(P_SCF, st, 32.0 * ng, ng);
    k_add_real<<<blocks, 256, 0, st>>>(rho_next, mx->cg, ng);
  }
  DKS_CUDA_TRY(cudaGetLastError());
  DKS_CUDA_TRY(cudaStreamSynchronize(st));
  return DKS_OK;
}

int dks_density(dks_ctx* ctx, int ik, const void* X, int nb, const double* occ, double* rho, void* stream) {
  if (!ctx || ik < 0 || ik >= ctx->nk || nb < 0 || (nb && (!X || !occ || !rho)))
    return fail(DKS_ERR_INVALID_ARG, "dks_density: bad argument");
  return density_accumulate(ctx, ik, (const double2*)X, nb, occ, rho, (cudaStream_t)stream);
}

int dks_hxc(dks_ctx* ctx, const double* rho, double* vhxc, double* energies, void* stream) {
  if (!ctx || !rho || !vhxc || rho == vhxc) return fail(DKS_ERR_INVALID_ARG, "dks_hxc: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t ng = (size_t)ctx->ng;
  void* tmp = nullptr;
  DKS_CUDA_TRY(cudaMallocAsync(&tmp, ng * sizeof(double2) + 2 * sizeof(double), st));
  double2* cg = (double2*)tmp;
  double* esum = (double*)(cg + ng);
  int rc = hxc_potential(ctx, rho, vhxc, cg, esum, st);
  double e[2] = {0.0, 0.0};
  if (rc == DKS_OK && energies) {
    cudaError_t err = cudaMemcpyAsync(e, esum, sizeof(e), cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) rc = fail(DKS_ERR_CUDA, std::string("dks_hxc: ") + cudaGetErrorString(err));
    const double dv = ctx->volume / (double)ng;
    energies[0] = 0.5 * dv * e[0];
    energies[1] = dv * e[1];
  }
  cudaFreeAsync(tmp, st);
  return rc;
}

int dks_set_potential(dks_ctx* ctx, const double* v, void* stream) {
  if (!ctx || !v) return fail(DKS_ERR_INVALID_ARG, "dks_set_potential: bad argument");
  return set_potential(ctx, v, (cudaStream_t)stream);
}

int dks_update_potential(dks_ctx* ctx, const double* rho, double* energies, void* stream) {
  if (!ctx) return fail(DKS_ERR_INVALID_ARG, "dks_update_potential: ctx is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t ng = (size_t)ctx->ng;
  void* tmp = nullptr;
  DKS_CUDA_TRY(cudaMallocAsync(&tmp, ng * (sizeof(double2) + sizeof(double)) + 2 * sizeof(double), st));
  double2* cg = (double2*)tmp;
  double* v = (double*)(cg + ng);
  double* esum = v + ng;
  auto body = [&]() -> int {
    if (rho) {
      DKS_TRY(hxc_potential(ctx, rho, v, cg, esum, st));
      if (ctx->vloc_dev) {
        Prof pr(P_SCF, st, 24.0 * ng, (double)ng);
        k_axpy_grid<<<grid_blocks(ctx, ng), 256, 0, st>>>(ctx->vloc_dev, v, v, ng);
        DKS_CUDA_TRY(cudaGetLastError());
      }
    } else if (ctx->vloc_dev) {
      DKS_CUDA_TRY(cudaMemcpyAsync(v, ctx->vloc_dev, ng * sizeof(double), cudaMemcpyDeviceToDevice, st));
    } else {
      DKS_CUDA_TRY(cudaMemsetAsync(v, 0, ng * sizeof(double), st));
    }
    DKS_TRY(set_potential(ctx, v, st));   // synchronises st
    if (energies) {
      energies[0] = energies[1] = 0.0;
      if (rho) {
        double e[2];
        DKS_CUDA_TRY(cudaMemcpyAsync(e, esum, sizeof(e), cudaMemcpyDeviceToHost, st));
        DKS_CUDA_TRY(cudaStreamSynchronize(st));
        const double dv = ctx->volume / (double)ng;
        energies[0] = 0.5 * dv * e[0];
        energies[1] = dv * e[1];
      }
    }
    return DKS_OK;
  };
  const int rc = body();
  cudaFreeAsync(tmp, st);
  return rc;
}

int dks_density_residual(dks_ctx* ctx, const double* a, const double* b, double* out, void* stream) {
  if (!ctx || !a || !b || !out) return fail(DKS_ERR_INVALID_ARG, "dks_density_residual: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t ng = (size_t)ctx->ng;
  double* sum = nullptr;
  DKS_CUDA_TRY(cudaMallocAsync((void**)&sum, sizeof(double), st));
  double h = 0.0;
  cudaError_t e = cudaMemsetAsync(sum, 0, sizeof(double), st);
  if (e == cudaSuccess) {
    Prof pr(P_SCF, st, 16.0 * ng, 2.0 * ng);
    k_absdiff_sum<<<grid_blocks(ctx, ng), 256, 0, st>>>(a, b, sum, ng);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, sum, sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(sum, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(DKS_ERR_CUDA, std::string("dks_density_residual: ") + cudaGetErrorString(e));
  *out = h * ctx->volume / (double)ng;
  return DKS_OK;
}

void dks_scf_opts_default(dks_scf_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->nocc = 0;
  o->max_iter = 60;
  o->tol = 1e-8;
  o->alpha = 0.5;
  o->kerker_q0 = 1.0;
  o->history = 8;
  o->n_init_warm = 1;
  o->solve_tol = 1e-8;
  dks_solve_opts_default(&o->solve);
}

int dks_scf(dks_ctx* ctx, int nev, const dks_scf_opts* o, double* eig, void* const* X, double* rho,
            dks_scf_report* rep) {
  const auto t0 = std::chrono::steady_clock::now();
  if (rep) std::memset(rep, 0, sizeof(*rep));
  if (!ctx || !o || !eig || !X || o->nocc < 1 || o->max_iter < 0 || !(o->tol > 0) || !(o->solve_tol > 0) ||
      o->n_init_warm < 0)
    return fail(DKS_ERR_INVALID_ARG, "dks_scf: bad argument (nocc >= 1, tol > 0, solve_tol > 0)");
  for (int ik = 0; ik < ctx->nk; ++ik) {
    const int nv = o->solve.nev_k ? o->solve.nev_k[ik] : nev;
    if (o->nocc > nv) return fail(DKS_ERR_INVALID_ARG, "dks_scf: nocc exceeds the wanted pairs of a k-point");
  }
  cudaStream_t st = (cudaStream_t)o->solve.stream;
  const size_t ng = (size_t)ctx->ng;
  dks_mixer* mx = nullptr;
  DKS_TRY(dks_mixer_create(ctx, o->history, o->alpha, o->kerker_q0, &mx));
  void* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, 4 * ng * sizeof(double) + ng * sizeof(double2) + 4 * sizeof(double));
  if (e != cudaSuccess) {
    dks_mixer_destroy(mx);
    return fail(DKS_ERR_OOM, std::string("dks_scf: ") + cudaGetErrorString(e));
  }
  double* vext = (double*)buf;    // V_loc
  double* rin = vext + ng;
  double* rout = rin + ng;
  double* vtot = rout + ng;
  double2* cg = (double2*)(vtot + ng);
  double* small = (double*)(cg + ng);   // [0..1] energies, [2] residual
  const int blocks = grid_blocks(ctx, ng);
  const std::vector<double> occ(o->nocc, 1.0 / ctx->nk);
  dks_solve_opts so = o->solve;
  dks_solve_report srep;
  int rc = DKS_OK, final_rc = DKS_OK;
  auto run_solve = [&](int n_init) -> int {
    so.n_init = n_init;
    const int r = dks_lobpcgf_solve(ctx, nev, o->solve_tol, &so, eig, X, &srep);
    if (rep) {
      for (int ik = 0; ik < std::min(ctx->nk, 64); ++ik) rep->solve_iterations += srep.iterations[ik];
      rep->h_applications += srep.h_applications;
    }
    return r == DKS_ERR_NOT_CONVERGED ? DKS_OK : r;
  };
  auto density_of = [&](double* out) -> int {
    DKS_CUDA_TRY(cudaMemsetAsync(out, 0, ng * sizeof(double), st));
    for (int ik = 0; ik < ctx->nk; ++ik) DKS_TRY(density_accumulate(ctx, ik, (const double2*)X[ik], o->nocc,
                                                                    occ.data(), out, st));
    return DKS_OK;
  };
  auto body = [&]() -> int {
    if (ctx->vloc_dev)
      DKS_CUDA_TRY(cudaMemcpyAsync(vext, ctx->vloc_dev, ng * sizeof(double), cudaMemcpyDeviceToDevice, st));
    else
      DKS_CUDA_TRY(cudaMemsetAsync(vext, 0, ng * sizeof(double), st));
    DKS_TRY(set_potential(ctx, vext, st));
    DKS_TRY(run_solve(o->solve.n_init));
    DKS_TRY(density_of(rin));
    final_rc = DKS_ERR_NOT_CONVERGED;
    for (int it = 1; it <= o->max_iter; ++it) {
      NvtxRange nvtx("SCF iteration");
      DKS_TRY(hxc_potential(ctx, rin, vtot, cg, small, st));
      {
        Prof pr(P_SCF, st, 24.0 * ng, ng);
        k_axpy_grid<<<blocks, 256, 0, st>>>(vext, vtot, vtot, ng);
      }
      DKS_CUDA_TRY(cudaGetLastError());
      DKS_TRY(set_potential(ctx, vtot, st));
      DKS_TRY(run_solve(o->n_init_warm));
      DKS_TRY(density_of(rout));
      DKS_CUDA_TRY(cudaMemsetAsync(small + 2, 0, sizeof(double), st));
      {
        Prof pr(P_SCF, st, 16.0 * ng, 2.0 * ng);
        k_absdiff_sum<<<blocks, 256, 0, st>>>(rout, rin, small + 2, ng);
      }
      DKS_CUDA_TRY(cudaGetLastError());
      double hs[3];
      DKS_CUDA_TRY(cudaMemcpyAsync(hs, small, sizeof(hs), cudaMemcpyDeviceToHost, st));
      DKS_CUDA_TRY(cudaStreamSynchronize(st));
      const double dv = ctx->volume / (double)ng;
      const double res = dv * hs[2];
      if (rep) {
        rep->iterations = it;
        rep->residual = res;
        rep->e_h = 0.5 * dv * hs[0];
        rep->e_xc = dv * hs[1];
        if (rep->hist_len < 128) rep->res_history[rep->hist_len++] = res;
      }
      if (res < o->tol) {
        final_rc = DKS_OK;
        if (rep) rep->converged = 1;
        break;
      }
      DKS_TRY(dks_mix(mx, rin, rout, rin, st));
    }
    if (rho) {
      // the last rho_out (or the first density when max_iter is 0)
      DKS_CUDA_TRY(cudaMemcpyAsync(rho, o->max_iter ? rout : rin, ng * sizeof(double), cudaMemcpyDeviceToDevice,
                                   st));
      DKS_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return DKS_OK;
  };
  rc = body();
  cudaStreamSynchronize(st);
  cudaFree(buf);
  dks_mixer_destroy(mx);
  if (rc == DKS_OK) rc = final_rc;
  if (rep) {
    rep->status = rc;
    rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return rc;
}

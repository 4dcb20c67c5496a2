// C ABI: context creation (planewave spheres, FFT plans, projector tables),
// H' application, filter and the single-step entry points of Algorithm 1.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "dks_internal.h"

namespace dks {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int grow(Workspace& w, size_t bytes) {
  if (bytes <= w.bytes) return DKS_OK;
  if (w.ptr) cudaFree(w.ptr);
  w.ptr = nullptr;
  w.bytes = 0;
  cudaError_t e = cudaMalloc(&w.ptr, bytes);
  if (e != cudaSuccess) {
    w.ptr = nullptr;
    return fail(DKS_ERR_OOM, std::string("workspace of ") + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
  }
  w.bytes = bytes;
  return DKS_OK;
}

Exec& exec0(dks_ctx* ctx) {
  if (ctx->exec.empty()) ctx->exec.push_back(new Exec());
  return *ctx->exec[0];
}

void release(Workspace& w) {
  if (w.ptr) cudaFree(w.ptr);
  w.ptr = nullptr;
  w.bytes = 0;
}

// fewest passes over the radices {8, 7, 6, 5, 4, 3, 2}; among equal counts the larger radix first
static int plan_passes(int n, int* best_first) {
  if (n == 1) return 0;
  const int radices[] = {8, 7, 6, 5, 4, 3, 2};
  int best = 1 << 20;
  *best_first = 0;
  for (int r : radices) {
    if (n % r) continue;
    int dummy = 0;
    const int c = 1 + plan_passes(n / r, &dummy);
    if (c < best) {
      best = c;
      *best_first = r;
    }
  }
  return best;
}

bool make_axis_plan(int n, AxisPlan* p) {
  if (n < 1 || n > kMaxFftLen) return false;
  p->n = n;
  p->nst = 0;
  int rest = n, len = n;
  while (rest > 1) {
    int r = 0;
    if (plan_passes(rest, &r) >= (1 << 20) || !r || p->nst >= kMaxStages) return false;
    p->radix[p->nst] = r;
    p->blk[p->nst] = len;
    ++p->nst;
    len /= r;
    rest /= r;
  }
  return true;
}

// pos(k): DIF maps frequency k = m + R k' of a block of length L to position m (L/R) + pos_{L/R}(k')
std::vector<int> dif_positions(const AxisPlan& p) {
  std::vector<int> pos(p.n);
  for (int k = 0; k < p.n; ++k) {
    int kk = k, at = 0;
    for (int s = 0; s < p.nst; ++s) {
      const int r = p.radix[s], sub = p.blk[s] / r;
      at += (kk % r) * sub;
      kk /= r;
    }
    pos[k] = at;
  }
  return pos;
}

// complex spherical harmonics, Condon-Shortley phase, l <= 2, unit vector u
static std::complex<double> ylm(int l, int m, const double u[3]) {
  const double pi = 3.14159265358979323846;
  const std::complex<double> xp(u[0], u[1]), xm(u[0], -u[1]);
  const double z = u[2];
  if (std::abs(m) > l) return 0.0;
  switch (l) {
    case 0: return 0.5 / std::sqrt(pi);
    case 1:
      if (m == 0) return std::sqrt(3.0 / (4 * pi)) * z;
      return m > 0 ? -std::sqrt(3.0 / (8 * pi)) * xp : std::sqrt(3.0 / (8 * pi)) * xm;
    default:
      if (m == 0) return std::sqrt(5.0 / (16 * pi)) * (3 * z * z - 1);
      if (m == 1) return -std::sqrt(15.0 / (8 * pi)) * z * xp;
      if (m == -1) return std::sqrt(15.0 / (8 * pi)) * z * xm;
      if (m == 2) return std::sqrt(15.0 / (32 * pi)) * xp * xp;
      return std::sqrt(15.0 / (32 * pi)) * xm * xm;
  }
}

// spinor spherical harmonic Omega_{j l mj}: j2 = 2j, mj2 = 2mj; returns (up, down)
static void spinor_ylm(int j2, int l, int mj2, const double u[3], std::complex<double> out[2]) {
  const double mj = 0.5 * mj2, d = 2.0 * l + 1.0;
  const int m_up = (mj2 - 1) / 2;   // mj2 is odd, so this division is exact
  const int m_dn = m_up + 1;
  double a_up, a_dn;
  if (j2 == 2 * l + 1) {
    a_up = std::sqrt((l + mj + 0.5) / d);
    a_dn = std::sqrt((l - mj + 0.5) / d);
  } else {
    a_up = -std::sqrt((l - mj + 0.5) / d);
    a_dn = std::sqrt((l + mj + 0.5) / d);
  }
  out[0] = a_up * ylm(l, m_up, u);
  out[1] = a_dn * ylm(l, m_dn, u);
}

static double radial_norm(int l, double r) {
  const double twopi3 = std::pow(2.0 * 3.14159265358979323846, 3);
  return std::sqrt(2.0 * twopi3 * std::pow(r, 2 * l + 3) / std::tgamma(l + 1.5));
}

template <typename T>
static int upload(T** dst, const T* src, size_t n) {
  if (!n) {
    *dst = nullptr;
    return DKS_OK;
  }
  DKS_CUDA_TRY(cudaMalloc((void**)dst, n * sizeof(T)));
  DKS_CUDA_TRY(cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice));
  return DKS_OK;
}

struct Channel {
  int site, l, jj, j2, mj2;
};

static int build_k(dks_ctx* ctx, const double kfrac[3], double ecut, const dks_projectors* proj,
                   const std::vector<Channel>& chans, KPoint& kp) {
  const double* B = ctx->recip;
  for (int a = 0; a < 3; ++a) kp.kcart[a] = kfrac[0] * B[a] + kfrac[1] * B[3 + a] + kfrac[2] * B[6 + a];
  kp.ecut = ecut;
  const double knorm = std::sqrt(kp.kcart[0] * kp.kcart[0] + kp.kcart[1] * kp.kcart[1] + kp.kcart[2] * kp.kcart[2]);
  const double gmax = std::sqrt(2.0 * ecut);
  int lim[3];
  for (int i = 0; i < 3; ++i) {
    const double* a = ctx->lattice + 3 * i;
    const double an = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    lim[i] = (int)std::floor((knorm + gmax) * an / (2.0 * 3.14159265358979323846)) + 1;
  }
  std::vector<int> mil;
  std::vector<double> q;
  for (int m1 = -lim[0]; m1 <= lim[0]; ++m1)
    for (int m2 = -lim[1]; m2 <= lim[1]; ++m2)
      for (int m3 = -lim[2]; m3 <= lim[2]; ++m3) {
        double v[3];
        for (int a = 0; a < 3; ++a) v[a] = kp.kcart[a] + (m1 * B[a] + m2 * B[3 + a] + m3 * B[6 + a]);
        if (0.5 * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) <= ecut) {
          mil.push_back(m1);
          mil.push_back(m2);
          mil.push_back(m3);
          q.insert(q.end(), v, v + 3);
        }
      }
  const int npw = (int)(mil.size() / 3);
  if (npw == 0) return fail(DKS_ERR_INVALID_ARG, "empty planewave sphere");
  for (int p = 0; p < npw; ++p)
    for (int a = 0; a < 3; ++a)
      if (std::abs(mil[3 * p + a]) > (ctx->grid[a] - 1) / 2)
        return fail(DKS_ERR_GRID, "planewave sphere does not fit the FFT grid along axis " + std::to_string(a));
  kp.npw = npw;
  kp.miller = mil;
  std::vector<int> sstart, splane, pstick(npw), piz(npw);
  std::vector<double> ek(npw);
  double qmax2 = 0;
  for (int p = 0; p < npw; ++p) {
    if (p == 0 || mil[3 * p] != mil[3 * p - 3] || mil[3 * p + 1] != mil[3 * p - 2]) {
      sstart.push_back(p);
      const int i1 = ((mil[3 * p] % ctx->grid[0]) + ctx->grid[0]) % ctx->grid[0];
      const int i2 = ((mil[3 * p + 1] % ctx->grid[1]) + ctx->grid[1]) % ctx->grid[1];
      splane.push_back(i1 * ctx->plane_ld + i2);
    }
    pstick[p] = (int)sstart.size() - 1;
    piz[p] = ((mil[3 * p + 2] % ctx->grid[2]) + ctx->grid[2]) % ctx->grid[2];
    const double q2 = q[3 * p] * q[3 * p] + q[3 * p + 1] * q[3 * p + 1] + q[3 * p + 2] * q[3 * p + 2];
    ek[p] = 0.5 * q2;
    qmax2 = std::max(qmax2, q2);
  }
  kp.nsticks = (int)sstart.size();
  sstart.push_back(npw);
  kp.qmax = std::sqrt(qmax2);
  DKS_TRY(upload(&kp.stick_start, sstart.data(), sstart.size()));
  DKS_TRY(upload(&kp.stick_plane, splane.data(), splane.size()));
  DKS_TRY(upload(&kp.pw_stick, pstick.data(), pstick.size()));
  DKS_TRY(upload(&kp.pw_iz, piz.data(), piz.size()));
  DKS_TRY(upload(&kp.q, q.data(), q.size()));
  std::vector<float> cq(6 * (size_t)npw);
  for (size_t e = 0; e < 3 * (size_t)npw; ++e) {
    const double v = ctx->c * q[e];
    const float h = (float)v;
    cq[2 * e] = h;
    cq[2 * e + 1] = (float)(v - (double)h);
  }
  DKS_TRY(upload(&kp.cq32, cq.data(), cq.size()));
  DKS_TRY(upload(&kp.ek, ek.data(), ek.size()));
  // projector rows beta_c[(spin*npw + p)]
  if (!chans.empty()) {
    const size_t rows = (size_t)2 * npw;
    std::vector<double2> bt(chans.size() * rows);
    std::vector<float2> bt32(chans.size() * rows);
    const double inv_sqrt_vol = 1.0 / std::sqrt(ctx->volume);
    for (size_t c = 0; c < chans.size(); ++c) {
      const Channel& ch = chans[c];
      const double* R = proj->pos + 3 * ch.site;
      const double rl = proj->rl[3 * ch.site + ch.l];
      const double an = radial_norm(ch.l, rl);
      for (int p = 0; p < npw; ++p) {
        const double* v = &q[3 * p];
        const double qn = std::sqrt(2.0 * ek[p]);
        double u[3] = {0, 0, 1};
        if (qn > 0) u[0] = v[0] / qn, u[1] = v[1] / qn, u[2] = v[2] / qn;
        const double rad = an * std::pow(qn, ch.l) * std::exp(-0.5 * qn * qn * rl * rl) * inv_sqrt_vol;
        const double arg = -(v[0] * R[0] + v[1] * R[1] + v[2] * R[2]);
        const std::complex<double> phase(std::cos(arg), std::sin(arg));
        std::complex<double> om[2];
        spinor_ylm(ch.j2, ch.l, ch.mj2, u, om);
        for (int s = 0; s < 2; ++s) {
          const std::complex<double> val = rad * phase * om[s];
          bt[c * rows + (size_t)s * npw + p] = double2{val.real(), val.imag()};
          bt32[c * rows + (size_t)s * npw + p] = float2{(float)val.real(), (float)val.imag()};
        }
      }
    }
    DKS_TRY(upload(&kp.bt64, bt.data(), bt.size()));
    DKS_TRY(upload(&kp.bt32, bt32.data(), bt32.size()));
    std::vector<float4> btd(bt.size());
    for (size_t e = 0; e < bt.size(); ++e) {
      const float rh = (float)bt[e].x, ih = (float)bt[e].y;
      btd[e] = float4{rh, (float)(bt[e].x - (double)rh), ih, (float)(bt[e].y - (double)ih)};
    }
    DKS_TRY(upload(&kp.btdf, btd.data(), btd.size()));
  }
  // default filter constants (shifted units)
  const double c = ctx->c;
  const double emax = std::sqrt(c * c * qmax2 + c * c * c * c);
  kp.cshift = -(3.0 * c * c + emax) / 2.0;
  const double eupper = (emax - c * c) + ctx->vmax + ctx->dsum;
  kp.omega = eupper - kp.cshift;
  return DKS_OK;
}

static void free_ctx(dks_ctx* ctx) {
  if (!ctx) return;
  for (int a = 0; a < 3; ++a) {
    cudaFree(ctx->tw64[a]);
    cudaFree(ctx->tw32[a]);
    cudaFree(ctx->twdf[a]);
  }
  cudaFree(ctx->vperm64);
  cudaFree(ctx->vperm32);
  cudaFree(ctx->vpermdf);
  cudaFree(ctx->vloc_dev);
  for (int a = 0; a < 3; ++a) cudaFree(ctx->posd[a]);
  cudaFree(ctx->dvec_dev);
  for (KPoint& kp : ctx->k) {
    cudaFree(kp.stick_start);
    cudaFree(kp.stick_plane);
    cudaFree(kp.pw_stick);
    cudaFree(kp.pw_iz);
    cudaFree(kp.q);
    cudaFree(kp.cq32);
    cudaFree(kp.ek);
    cudaFree(kp.bt64);
    cudaFree(kp.bt32);
    cudaFree(kp.btdf);
    if (kp.btoz) cudaFree(kp.btoz);
  }
  for (Exec* e : ctx->exec) {
    release(e->ws_h);
    release(e->ws_solve);
    release(e->ws_oz);
    if (e->own) cudaStreamDestroy(e->own);
    delete e;
  }
  delete ctx;
}

}  // namespace dks

using namespace dks;

extern "C" {

const char* dks_strerror(int code) {
  switch (code) {
    case DKS_OK: return "ok";
    case DKS_ERR_INVALID_ARG: return "invalid argument";
    case DKS_ERR_CUDA: return "CUDA runtime error";
    case DKS_ERR_OOM: return "out of memory";
    case DKS_ERR_NOT_CONVERGED: return "not converged within n_iter";
    case DKS_ERR_NEG_STATE: return "a selected Ritz value lies below the gap midpoint";
    case DKS_ERR_RANK: return "subspace rank fell below the block size";
    case DKS_ERR_TIMEOUT: return "bounded device wait gave up";
    case DKS_ERR_GRID: return "planewave sphere does not fit the FFT grid";
    case DKS_ERR_UNSUPPORTED: return "size outside the compiled limits";
    default: return "unknown error";
  }
}

const char* dks_last_error(void) { return g_last_error.c_str(); }

int dks_create(const dks_cell* cell, double ecut, const dks_potentials* pot, const dks_projectors* proj,
               dks_ctx** out) {
  if (!out) return fail(DKS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!cell || !cell->kfrac || cell->nk < 1 || !(cell->c > 0))
    return fail(DKS_ERR_INVALID_ARG, "cell: need kfrac, nk >= 1 and c > 0");
  if (!cell->ecut_k && !(ecut > 0)) return fail(DKS_ERR_INVALID_ARG, "ecut must be positive");
  dks_ctx* ctx = new (std::nothrow) dks_ctx();
  if (!ctx) return fail(DKS_ERR_OOM, "host allocation");
  int rc = DKS_OK;
  auto bail = [&](int code) {
    free_ctx(ctx);
    return code;
  };
  cudaGetDevice(&ctx->device);
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
  ctx->c = cell->c;
  ctx->nk = cell->nk;
  std::memcpy(ctx->lattice, cell->lattice, sizeof(ctx->lattice));
  for (int a = 0; a < 3; ++a) {
    ctx->grid[a] = cell->grid[a];
    if (!make_axis_plan(cell->grid[a], &ctx->plan[a]))
      return bail(fail(DKS_ERR_UNSUPPORTED, "grid axis must be <= 256 with factors 2, 3, 5, 7"));
  }
  ctx->ng = ctx->grid[0] * ctx->grid[1] * ctx->grid[2];
  ctx->plane_ld = ctx->grid[1] | 1;
  // planes above one CTA's shared memory run pass B as row and column kernels (hx_kernels.cu)
  // reciprocal rows: b_i = 2 pi (A^-1)^T rows
  const double* A = ctx->lattice;
  const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                     A[2] * (A[3] * A[7] - A[4] * A[6]);
  if (!(std::fabs(det) > 0)) return bail(fail(DKS_ERR_INVALID_ARG, "singular lattice"));
  ctx->volume = std::fabs(det);
  const double tp = 2.0 * 3.14159265358979323846 / det;
  // b1 = 2pi (a2 x a3)/det etc.
  const double* a1 = A;
  const double* a2 = A + 3;
  const double* a3 = A + 6;
  double* Bm = ctx->recip;
  Bm[0] = tp * (a2[1] * a3[2] - a2[2] * a3[1]);
  Bm[1] = tp * (a2[2] * a3[0] - a2[0] * a3[2]);
  Bm[2] = tp * (a2[0] * a3[1] - a2[1] * a3[0]);
  Bm[3] = tp * (a3[1] * a1[2] - a3[2] * a1[1]);
  Bm[4] = tp * (a3[2] * a1[0] - a3[0] * a1[2]);
  Bm[5] = tp * (a3[0] * a1[1] - a3[1] * a1[0]);
  Bm[6] = tp * (a1[1] * a2[2] - a1[2] * a2[1]);
  Bm[7] = tp * (a1[2] * a2[0] - a1[0] * a2[2]);
  Bm[8] = tp * (a1[0] * a2[1] - a1[1] * a2[0]);
  // twiddles
  for (int a = 0; a < 3; ++a) {
    const int n = ctx->grid[a];
    std::vector<double2> tw(n);
    std::vector<float2> tw32(n);
    for (int t = 0; t < n; ++t) {
      const double ang = 2.0 * 3.14159265358979323846 * t / n;
      tw[t] = double2{std::cos(ang), std::sin(ang)};
      tw32[t] = float2{(float)tw[t].x, (float)tw[t].y};
    }
    std::vector<float4> twd(n);
    for (int t = 0; t < n; ++t) {
      const float rh = (float)tw[t].x, ih = (float)tw[t].y;
      twd[t] = float4{rh, (float)(tw[t].x - (double)rh), ih, (float)(tw[t].y - (double)ih)};
    }
    if ((rc = upload(&ctx->tw64[a], tw.data(), n))) return bail(rc);
    if ((rc = upload(&ctx->tw32[a], tw32.data(), n))) return bail(rc);
    if ((rc = upload(&ctx->twdf[a], twd.data(), n))) return bail(rc);
  }
  // DIF positions of the natural grid indices (density and potential updates on the device)
  for (int a = 0; a < 3; ++a) {
    const std::vector<int> pa = dif_positions(ctx->plan[a]);
    if ((rc = upload(&ctx->posd[a], pa.data(), pa.size()))) return bail(rc);
  }
  // potential in DIF order, scaled by 1/Ng
  ctx->has_v = pot && pot->v_r;
  if (ctx->has_v) {
    if ((rc = upload(&ctx->vloc_dev, pot->v_r, (size_t)ctx->ng))) return bail(rc);
    const int n1 = ctx->grid[0], n2 = ctx->grid[1], n3 = ctx->grid[2];
    const std::vector<int> p1 = dif_positions(ctx->plan[0]), p2 = dif_positions(ctx->plan[1]),
                           p3 = dif_positions(ctx->plan[2]);
    const int ld = ctx->plane_ld;
    const size_t nvp = (size_t)n3 * n1 * ld;
    std::vector<double> vp(nvp, 0.0);
    std::vector<float> vp32(nvp, 0.0f);
    std::vector<float2> vpdf(nvp, float2{0.0f, 0.0f});
    for (int i1 = 0; i1 < n1; ++i1)
      for (int i2 = 0; i2 < n2; ++i2)
        for (int i3 = 0; i3 < n3; ++i3) {
          const double v = pot->v_r[((size_t)i1 * n2 + i2) * n3 + i3];
          ctx->vmax = std::max(ctx->vmax, std::fabs(v));
          const size_t at = ((size_t)p3[i3] * n1 + p1[i1]) * ld + p2[i2];
          vp[at] = v / ctx->ng;
          vp32[at] = (float)(v / ctx->ng);
          const float h = (float)vp[at];
          vpdf[at] = float2{h, (float)(vp[at] - (double)h)};
        }
    if ((rc = upload(&ctx->vperm64, vp.data(), vp.size()))) return bail(rc);
    if ((rc = upload(&ctx->vperm32, vp32.data(), vp32.size()))) return bail(rc);
    if ((rc = upload(&ctx->vpermdf, vpdf.data(), vpdf.size()))) return bail(rc);
  }
  // projector channels
  std::vector<Channel> chans;
  if (proj && proj->nsite > 0) {
    if (!proj->pos || !proj->lmax || !proj->rl || !proj->d)
      return bail(fail(DKS_ERR_INVALID_ARG, "projectors: NULL array"));
    for (int s = 0; s < proj->nsite; ++s) {
      if (proj->lmax[s] > 2) return bail(fail(DKS_ERR_UNSUPPORTED, "projectors: lmax > 2"));
      for (int l = 0; l <= proj->lmax[s]; ++l) {
        if (!(proj->rl[3 * s + l] > 0)) return bail(fail(DKS_ERR_INVALID_ARG, "projectors: rl must be > 0"));
        for (int jj = 0; jj < 2; ++jj) {
          const int j2 = jj == 0 ? 2 * l + 1 : 2 * l - 1;
          if (j2 < 0) continue;
          const double dv = proj->d[(3 * s + l) * 2 + jj];
          ctx->dsum += std::fabs(dv);
          for (int mj2 = -j2; mj2 <= j2; mj2 += 2) {
            chans.push_back(Channel{s, l, jj, j2, mj2});
            ctx->dvec.push_back(dv);
          }
        }
      }
    }
  }
  ctx->nproj = (int)chans.size();
  if (ctx->nproj && (rc = upload(&ctx->dvec_dev, ctx->dvec.data(), ctx->dvec.size()))) return bail(rc);
  ctx->k.resize(cell->nk);
  for (int ik = 0; ik < cell->nk; ++ik) {
    const double ek = cell->ecut_k ? cell->ecut_k[ik] : ecut;
    if (!(ek > 0)) return bail(fail(DKS_ERR_INVALID_ARG, "ecut_k must be positive"));
    if ((rc = build_k(ctx, cell->kfrac + 3 * ik, ek, proj, chans, ctx->k[ik]))) return bail(rc);
  }
  *out = ctx;
  return DKS_OK;
}

void dks_destroy(dks_ctx* ctx) { free_ctx(ctx); }

int dks_debug_check(int* compiled, unsigned* code) {
  if (!compiled || !code) return fail(DKS_ERR_INVALID_ARG, "dks_debug_check: NULL output");
#ifdef DKS_DEBUG
  *compiled = 1;
  *code = debug_check_take();
#else
  *compiled = 0;
  *code = 0u;
#endif
  return DKS_OK;
}

int dks_fft_plan(int n, int* nst, int* radix, int* pos) {
  if (!nst || !radix) return fail(DKS_ERR_INVALID_ARG, "dks_fft_plan: NULL output");
  AxisPlan p;
  if (!make_axis_plan(n, &p)) return fail(DKS_ERR_UNSUPPORTED, "axis length must be <= 256 with factors 2, 3, 5, 7");
  *nst = p.nst;
  for (int i = 0; i < p.nst; ++i) radix[i] = p.radix[i];
  if (pos) {
    const std::vector<int> v = dif_positions(p);
    for (int k = 0; k < n; ++k) pos[k] = v[k];
  }
  return DKS_OK;
}

int dks_create_model(const dks_cell* cell, double ecut, const dks_potentials* pot, const dks_projectors* proj,
                     int model, dks_ctx** out) {
  if (model != DKS_MODEL_DKS && model != DKS_MODEL_KSSO) {
    if (out) *out = nullptr;
    return fail(DKS_ERR_INVALID_ARG, "dks_create_model: unknown model");
  }
  const int rc = dks_create(cell, ecut, pot, proj, out);
  if (rc == DKS_OK && model == DKS_MODEL_KSSO) (*out)->ncomp = 2;
  return rc;
}

int dks_ncomp(const dks_ctx* ctx, int* ncomp) {
  if (!ctx || !ncomp) return fail(DKS_ERR_INVALID_ARG, "dks_ncomp: bad argument");
  *ncomp = ctx->ncomp;
  return DKS_OK;
}

int dks_npw(const dks_ctx* ctx, int ik, int* npw) {
  if (!ctx || !npw || ik < 0 || ik >= ctx->nk) return fail(DKS_ERR_INVALID_ARG, "dks_npw: bad argument");
  *npw = ctx->k[ik].npw;
  return DKS_OK;
}

int dks_basis(const dks_ctx* ctx, int ik, int* miller) {
  if (!ctx || !miller || ik < 0 || ik >= ctx->nk) return fail(DKS_ERR_INVALID_ARG, "dks_basis: bad argument");
  std::memcpy(miller, ctx->k[ik].miller.data(), ctx->k[ik].miller.size() * sizeof(int));
  return DKS_OK;
}

int dks_nproj(const dks_ctx* ctx, int* nproj) {
  if (!ctx || !nproj) return fail(DKS_ERR_INVALID_ARG, "dks_nproj: bad argument");
  *nproj = ctx->nproj;
  return DKS_OK;
}

int dks_filter_constants(const dks_ctx* ctx, int ik, double* C, double* Omega) {
  if (!ctx || !C || !Omega || ik < 0 || ik >= ctx->nk)
    return fail(DKS_ERR_INVALID_ARG, "dks_filter_constants: bad argument");
  *C = ctx->k[ik].cshift;
  *Omega = ctx->k[ik].omega;
  return DKS_OK;
}

int dks_apply_H(dks_ctx* ctx, int ik, const void* X, void* HX, int nb, int prec, void* stream) {
  if (!ctx || ik < 0 || ik >= ctx->nk || nb < 0 || (nb && (!X || !HX)) || prec < 0 || prec > 2)
    return fail(DKS_ERR_INVALID_ARG, "dks_apply_H: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  Exec& ex = exec0(ctx);
  if (prec != DKS_PREC_FP32) {
    ex.df_gemm = prec == DKS_PREC_FP64_EMULATED;
    const int rc = apply_h<double2>(ctx, ex, ik, (const double2*)X, (double2*)HX, nb, 0.0, 1.0, st);
    ex.df_gemm = false;
    return rc;
  }
  return apply_h<float2>(ctx, ex, ik, (const float2*)X, (float2*)HX, nb, 0.0, 1.0, st);
}

int dks_kinetic_balance(dks_ctx* ctx, int ik, void* X, int nb, int prec, void* stream) {
  if (!ctx || ik < 0 || ik >= ctx->nk || nb < 0 || (nb && !X) || prec < 0 || prec > 2 || ctx->ncomp != 4)
    return fail(DKS_ERR_INVALID_ARG, "dks_kinetic_balance: bad argument (DKS contexts only)");
  return kinetic_balance(ctx, ik, X, nb, prec != DKS_PREC_FP32, (cudaStream_t)stream);
}

int dks_filter(dks_ctx* ctx, int ik, const void* Y, void* FY, int nb, double C, double Omega, int prec,
               void* stream) {
  if (!ctx || ik < 0 || ik >= ctx->nk || nb < 0 || (nb && (!Y || !FY)) || (prec != 0 && prec != 1) ||
      !(Omega != 0) || !std::isfinite(C) || !std::isfinite(Omega))
    return fail(DKS_ERR_INVALID_ARG, "dks_filter: bad argument");
  if (!nb) return DKS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t elems = (size_t)nb * ctx->ncomp * ctx->k[ik].npw;
  const size_t es = prec == DKS_PREC_FP64 ? sizeof(double2) : sizeof(float2);
  void* tmp = nullptr;
  DKS_CUDA_TRY(cudaMallocAsync(&tmp, elems * es, st));
  int rc;
  Exec& ex = exec0(ctx);
  if (prec == DKS_PREC_FP64) {
    rc = apply_h<double2>(ctx, ex, ik, (const double2*)Y, (double2*)tmp, nb, C, 1.0 / Omega, st);
    if (!rc) rc = apply_h<double2>(ctx, ex, ik, (const double2*)tmp, (double2*)FY, nb, C, 1.0 / Omega, st);
  } else {
    rc = apply_h<float2>(ctx, ex, ik, (const float2*)Y, (float2*)tmp, nb, C, 1.0 / Omega, st);
    if (!rc) rc = apply_h<float2>(ctx, ex, ik, (const float2*)tmp, (float2*)FY, nb, C, 1.0 / Omega, st);
  }
  cudaFreeAsync(tmp, st);
  return rc;
}

int dks_precond(dks_ctx* ctx, int ik, const void* X, const void* HX, const double* lam, const int* act, int nact,
                void* Y, int precond, int prec, void* stream) {
  if (!ctx || ik < 0 || ik >= ctx->nk || nact < 0 || (nact && (!X || !HX || !lam || !act || !Y)) || prec < 0 ||
      prec > 2)
    return fail(DKS_ERR_INVALID_ARG, "dks_precond: bad argument");
  if (!nact) return DKS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const KPoint& kp = ctx->k[ik];
  // statistics are needed for every column an active index may name: take max(act)+1 from the host? no --
  // compute them for the gathered columns only through a small index-free pass over all columns up to
  // the largest index, which the caller bounds by the buffer it passed.
  int ncol = 0;
  std::vector<int> hact(nact);
  DKS_CUDA_TRY(cudaMemcpyAsync(hact.data(), act, nact * sizeof(int), cudaMemcpyDeviceToHost, st));
  DKS_CUDA_TRY(cudaStreamSynchronize(st));
  for (int v : hact) {
    if (v < 0) return fail(DKS_ERR_INVALID_ARG, "dks_precond: negative column index");
    ncol = std::max(ncol, v + 1);
  }
  double* stats = nullptr;
  DKS_CUDA_TRY(cudaMallocAsync((void**)&stats, (size_t)3 * ncol * sizeof(double), st));
  int rc;
  if (prec != DKS_PREC_FP32) {
    rc = col_stats<double2>((const double2*)X, nullptr, nullptr, kp.ek, kp.npw, ncol, stats, st, ctx->ncomp);
    if (!rc) rc = precond_apply<double2>((const double2*)X, (const double2*)HX, lam, stats, act, nact, kp.ek, kp.npw,
                                         precond, (double2*)Y, st, ctx->ncomp);
  } else {
    rc = col_stats<float2>((const float2*)X, nullptr, nullptr, kp.ek, kp.npw, ncol, stats, st, ctx->ncomp);
    if (!rc) rc = precond_apply<float2>((const float2*)X, (const float2*)HX, lam, stats, act, nact, kp.ek, kp.npw,
                                        precond, (float2*)Y, st, ctx->ncomp);
  }
  cudaFreeAsync(stats, st);
  return rc;
}

int dks_gram(const void* Z, const void* HZ, int rows, int nz, void* A, void* S, int prec, void* stream) {
  if (rows <= 0 || nz <= 0 || !Z || !HZ || !A || !S) return fail(DKS_ERR_INVALID_ARG, "dks_gram: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  DKS_CUDA_TRY(cudaMemsetAsync(A, 0, (size_t)nz * nz * sizeof(double2), st));
  DKS_CUDA_TRY(cudaMemsetAsync(S, 0, (size_t)nz * nz * sizeof(double2), st));
  if (prec == DKS_PREC_FP64_EMULATED) {
    DKS_TRY(gemm_hn_df((const double2*)Z, rows, (const double2*)HZ, rows, rows, nz, nz, (double2*)A, st));
    DKS_TRY(gemm_hn_df((const double2*)Z, rows, (const double2*)Z, rows, rows, nz, nz, (double2*)S, st));
  } else if (prec == DKS_PREC_FP64) {
    DKS_TRY(gemm_hn<double2>((const double2*)Z, rows, (const double2*)HZ, rows, rows, nz, nz, (double2*)A, st));
    DKS_TRY(gemm_hn<double2>((const double2*)Z, rows, (const double2*)Z, rows, rows, nz, nz, (double2*)S, st));
  } else {
    DKS_TRY(gemm_hn<float2>((const float2*)Z, rows, (const float2*)HZ, rows, rows, nz, nz, (double2*)A, st));
    DKS_TRY(gemm_hn<float2>((const float2*)Z, rows, (const float2*)Z, rows, rows, nz, nz, (double2*)S, st));
  }
  return DKS_OK;
}

int dks_gram_hermitian(const void* Z, const void* HZ, int rows, int nz, void* A, void* S, int prec, void* stream) {
  if (rows <= 0 || nz <= 0 || !Z || !HZ || !A || !S)
    return fail(DKS_ERR_INVALID_ARG, "dks_gram_hermitian: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  DKS_CUDA_TRY(cudaMemsetAsync(A, 0, (size_t)nz * nz * sizeof(double2), st));
  DKS_CUDA_TRY(cudaMemsetAsync(S, 0, (size_t)nz * nz * sizeof(double2), st));
  if (prec == DKS_PREC_FP64_EMULATED && tc_enabled(TC_FP64)) {
    // exact integer slices of Z and HZ on the tensor cores
    const size_t ob = (oz_bytes(rows, nz) + 255) / 256 * 256;
    unsigned char* buf = nullptr;
    if (cudaMallocAsync((void**)&buf, 2 * ob, st) != cudaSuccess) {
      cudaGetLastError();
      return fail(DKS_ERR_OOM, "dks_gram_hermitian: no device memory for the slices");
    }
    OzBlock oz, ozh;
    oz_layout(buf, rows, nz, &oz);
    oz_layout(buf + ob, rows, nz, &ozh);
    int rc = oz_split((const double2*)Z, rows, nz, oz, st);
    if (!rc) rc = oz_split((const double2*)HZ, rows, nz, ozh, st);
    if (!rc) rc = oz_gram(oz, ozh, nz, (double2*)A, (double2*)S, st);
    cudaFreeAsync(buf, st);
    DKS_TRY(rc);
  } else if (prec == DKS_PREC_FP64_EMULATED) {
    const size_t n = (size_t)nz * rows;
    float4* zs = nullptr;
    if (cudaMallocAsync((void**)&zs, 2 * n * sizeof(float4), st) != cudaSuccess) {
      cudaGetLastError();
      return fail(DKS_ERR_OOM, "dks_gram_hermitian: no device memory for the double-float copies");
    }
    int rc = split_df((const double2*)Z, zs, n, st);
    if (!rc) rc = split_df((const double2*)HZ, zs + n, n, st);
    if (!rc) rc = gram_df(zs, zs + n, rows, rows, nz, (double2*)A, (double2*)S, st);
    cudaFreeAsync(zs, st);
    DKS_TRY(rc);
  } else if (prec == DKS_PREC_FP64) {
    DKS_TRY(gemm_hn<double2>((const double2*)Z, rows, (const double2*)HZ, rows, rows, nz, nz, (double2*)A, st,
                             P_GRAM, 0, true));
    DKS_TRY(gemm_hn<double2>((const double2*)Z, rows, (const double2*)Z, rows, rows, nz, nz, (double2*)S, st,
                             P_GRAM, 0, true));
  } else {
    DKS_TRY(gram_f32((const float2*)Z, (const float2*)HZ, rows, rows, nz, (double2*)A, (double2*)S, st));
  }
  DKS_TRY(mirror_lower((double2*)A, nz, st));
  return mirror_lower((double2*)S, nz, st);
}

int dks_rayleigh_ritz(const void* A, const void* S, int nz, int n, void* V, double* lam, int* info, void* stream) {
  if (!A || !S || !V || !lam || !info) return fail(DKS_ERR_INVALID_ARG, "dks_rayleigh_ritz: NULL pointer");
  if (nz <= 0 || n <= 0 || n > nz) return fail(DKS_ERR_INVALID_ARG, "dks_rayleigh_ritz: need 0 < n <= nz");
  if (nz > kMaxRR) return fail(DKS_ERR_UNSUPPORTED, "dks_rayleigh_ritz: nz above 512");
  cudaStream_t st = (cudaStream_t)stream;
  double2* scr = nullptr;
  DKS_CUDA_TRY(cudaMallocAsync((void**)&scr, rr_scratch_elems(nz) * sizeof(double2), st));
  const int rc = rayleigh_ritz((const double2*)A, (const double2*)S, nz, n, (double2*)V, lam, info, scr, st);
  cudaFreeAsync(scr, st);
  return rc;
}

int dks_rotate(const void* Z, int rows, int nz, const void* W, int ldw, int n, void* OUT, double beta, int prec,
               void* stream) {
  if (rows <= 0 || nz <= 0 || n <= 0 || ldw < nz || !Z || !W || !OUT)
    return fail(DKS_ERR_INVALID_ARG, "dks_rotate: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == DKS_PREC_FP64_EMULATED && tc_enabled(TC_FP64)) {
    // exact integer slices of Z on the tensor cores
    void* buf = nullptr;
    if (cudaMallocAsync(&buf, oz_bytes(rows, nz), st) != cudaSuccess) {
      cudaGetLastError();
      return fail(DKS_ERR_OOM, "dks_rotate: no device memory for the slices");
    }
    OzBlock oz;
    oz_layout(buf, rows, nz, &oz);
    int rc = oz_split((const double2*)Z, rows, nz, oz, st);
    if (!rc) rc = oz_rotate(oz, 0, nz, (const double2*)W, ldw, n, (double2*)OUT, rows, beta, st);
    cudaFreeAsync(buf, st);
    return rc;
  }
  if (prec == DKS_PREC_FP64_EMULATED)
    return gemm_nn_df((const double2*)Z, rows, rows, nz, (const double2*)W, ldw, nullptr, n, (double2*)OUT, rows,
                      beta, st);
  if (prec == DKS_PREC_FP64)
    return gemm_nn<double2>((const double2*)Z, rows, rows, nz, (const double2*)W, ldw, nullptr, n, (double2*)OUT,
                            rows, beta, st);
  return gemm_nn<float2>((const float2*)Z, rows, rows, nz, (const double2*)W, ldw, nullptr, n, (float2*)OUT, rows,
                         beta, st);
}

int dks_debug_rr_wait(unsigned first_wait_polls, unsigned* redone) {
  if (redone) DKS_TRY(rr_timeout_redos_take(redone));
  return rr_set_first_wait(first_wait_polls);
}

int dks_tensor_cores(int mask, int kchunk) {
  if (mask < 0 || mask > DKS_TC_ALL) return fail(DKS_ERR_INVALID_ARG, "dks_tensor_cores: mask outside DKS_TC_ALL");
  return tc_set(mask, kchunk);
}

int dks_tensor_cores_get(int* mask, int* kchunk) { return tc_get(mask, kchunk); }

int dks_residual_norms(const void* X, const void* HX, const double* lam, int rows, int n, double* norms, int prec,
                       void* stream) {
  if (rows <= 0 || rows % 2 || n <= 0 || !X || !HX || !lam || !norms || prec < 0 || prec > 2)
    return fail(DKS_ERR_INVALID_ARG, "dks_residual_norms: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  const int nc = rows % 4 ? 2 : 4;   // the column sums do not depend on the grouping of rows
  double* stats = nullptr;
  double* ek = nullptr;
  DKS_CUDA_TRY(cudaMallocAsync((void**)&stats, (size_t)3 * n * sizeof(double), st));
  DKS_CUDA_TRY(cudaMallocAsync((void**)&ek, (size_t)(rows / nc) * sizeof(double), st));
  DKS_CUDA_TRY(cudaMemsetAsync(ek, 0, (size_t)(rows / nc) * sizeof(double), st));
  int rc = prec != DKS_PREC_FP32
               ? col_stats<double2>((const double2*)X, (const double2*)HX, lam, ek, rows / nc, n, stats, st, nc)
               : col_stats<float2>((const float2*)X, (const float2*)HX, lam, ek, rows / nc, n, stats, st, nc);
  if (!rc) {
    // norms[j] = sqrt(stats[3j])
    std::vector<double> h((size_t)3 * n);
    cudaError_t e = cudaMemcpyAsync(h.data(), stats, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = fail(DKS_ERR_CUDA, cudaGetErrorString(e));
    std::vector<double> nr(n);
    for (int j = 0; j < n; ++j) nr[j] = std::sqrt(h[3 * j]);
    if (!rc) {
      e = cudaMemcpyAsync(norms, nr.data(), n * sizeof(double), cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) rc = fail(DKS_ERR_CUDA, cudaGetErrorString(e));
    }
  }
  cudaFreeAsync(stats, st);
  cudaFreeAsync(ek, st);
  return rc;
}

}  // extern "C"

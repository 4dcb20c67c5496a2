// H' x for the shifted valence DKS operator (Eq. vDKS, Sec. 3.1 "matrix-free Hx").
//
//   H' x = [[0, c s.q], [c s.q, -2c^2]] x          free Dirac term per planewave (Eq. 2)
//        + FFT^-1 . V(r) . FFT x                     local potential, one grid per component
//        + (I2 (x) B D B^H) x                         spin-orbit projectors (Eq. HGH)
//
// GPU layout.  x[band][comp][pw] with planewaves in canonical order, so each
// (m1, m2) "stick" along the third axis is a contiguous run of planewaves.  The
// 3D transform of one field (band, comp) runs in three passes that keep all
// intermediates in a stick-compressed buffer T[field][p3][stick] sized to stay
// resident in the 129 MB L2:
//   pass A  scatter the stick into a zeroed length-N3 line in shared memory,
//           inverse FFT along axis 3 (DIF, natural in -> digit-reversed out)
//   pass B  one (field, plane) per CTA: scatter the sticks into an N1 x N2 plane
//           in shared memory, inverse 2D FFT (DIF), multiply by V/Ng stored in
//           the same digit-reversed order, forward 2D FFT (DIT, digit-reversed in
//           -> natural out), gather the sticks back (in place in T)
//   pass C  four components of one band per CTA: forward FFT along axis 3 (DIT),
//           gather to the sphere, add the Dirac 4x4 term computed in FP64 and the
//           optional filter shift, scale, store
// Pairing DIF for the inverse with DIT for the forward transform removes every
// digit-reversal permutation: the real-space planes simply live in permuted
// order, and V is uploaded in that order.
// The projector term is two tall-skinny contractions over 2*npw rows with
// x viewed as [2*nb][2*npw] (large and small two-spinors as separate columns).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <type_traits>

#include "dks_internal.h"
#include "dks_kernels.cuh"
#include "fft_device.cuh"

namespace dks {

template <typename V> __device__ __forceinline__ V vzero() { return V{0, 0}; }
template <> __device__ __forceinline__ cdf vzero<cdf>() { return cdf{{0.f, 0.f}, {0.f, 0.f}}; }

// ---------------------------------------------------------------------------
// pass A: sphere -> stick lines, inverse FFT along axis 3
// ---------------------------------------------------------------------------
template <typename Vg, typename V>
__global__ void __launch_bounds__(256) k_stick_inverse(
    const Vg* __restrict__ x, Vg* __restrict__ t, int npw, int nsticks, const int* __restrict__ stick_start,
    const int* __restrict__ pw_stick, const int* __restrict__ pw_iz, AxisPlan p3,
    const V* __restrict__ tw3, int spb, int ls) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* line = reinterpret_cast<V*>(smem_raw);   // spb lines of stride ls (odd)
  const int n3 = p3.n;
  const int s0 = blockIdx.x * spb;
  const int ns = min(spb, nsticks - s0);
  const int f = blockIdx.y;
  for (int e = threadIdx.x; e < spb * ls; e += blockDim.x) line[e] = vzero<V>();
  __syncthreads();
  const Vg* xf = x + (size_t)f * npw;
  const int q0 = stick_start[s0], q1 = stick_start[s0 + ns];
  for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
    const int sl = pw_stick[q] - s0, iz = pw_iz[q];
    if (dks_ok(sl >= 0 && sl < ns && iz >= 0 && iz < n3, kChkStickInverse | (q & 0xffffff)))
      line[sl * ls + iz] = to_s<V>(xf[q]);
  }
  __syncthreads();
  fft_lines<V, false, false>(line, ns, ls, 1, p3, tw3);
  Vg* tf = t + (size_t)f * n3 * nsticks;
  const float rns = __fdividef(1.0f, (float)ns);
  for (int e = threadIdx.x; e < ns * n3; e += blockDim.x) {
    const int z = qdiv(e, ns, rns), s = e - z * ns;
    tf[(size_t)z * nsticks + s0 + s] = to_g(line[s * ls + z]);
  }
}

// ---------------------------------------------------------------------------
// pass B: one plane of one field: 2D inverse FFT, x V/Ng, 2D forward FFT
// ---------------------------------------------------------------------------
template <typename Vg, typename V>
__device__ __forceinline__ void plane_body(Vg* __restrict__ t, int nsticks, const int* __restrict__ stick_plane,
                                           const AxisPlan& p1, const AxisPlan& p2, int ld, int n3,
                                           const V* __restrict__ tw1, const V* __restrict__ tw2,
                                           const typename RealOf<V>::T* __restrict__ vperm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* plane = reinterpret_cast<V*>(smem_raw);   // n1 rows of stride ld (odd), position i1*ld + i2
  const int n1 = p1.n, n2 = p2.n, np = n1 * ld;
  const int z = blockIdx.x, f = blockIdx.y;
  for (int e = threadIdx.x; e < np; e += blockDim.x) plane[e] = vzero<V>();
  __syncthreads();
  Vg* row = t + ((size_t)f * n3 + z) * nsticks;
  for (int s = threadIdx.x; s < nsticks; s += blockDim.x)
    if (dks_ok(stick_plane[s] >= 0 && stick_plane[s] < np, kChkPlane | (s & 0xffffff)))
      plane[stick_plane[s]] = to_s<V>(row[s]);
  __syncthreads();
  fft_lines<V, false, false>(plane, n1, ld, 1, p2, tw2);   // along axis 2 (contiguous)
  fft_lines<V, false, false>(plane, n2, 1, ld, p1, tw1);   // along axis 1
  const typename RealOf<V>::T* vz = vperm + (size_t)z * np;   // zero in the padding column
  for (int e = threadIdx.x; e < np; e += blockDim.x) plane[e] = cscale(plane[e], vz[e]);
  __syncthreads();
  fft_lines<V, true, true>(plane, n2, 1, ld, p1, tw1);
  fft_lines<V, true, true>(plane, n1, ld, 1, p2, tw2);
  for (int s = threadIdx.x; s < nsticks; s += blockDim.x)
    if (dks_ok(stick_plane[s] >= 0 && stick_plane[s] < np, kChkPlane | (s & 0xffffff)))
      row[s] = to_g(plane[stick_plane[s]]);
}
template <typename Vg, typename V>
__global__ void __launch_bounds__(512) k_plane(Vg* __restrict__ t, int nsticks,
                                               const int* __restrict__ stick_plane, AxisPlan p1,
                                               AxisPlan p2, int ld, int n3, const V* __restrict__ tw1,
                                               const V* __restrict__ tw2,
                                               const typename RealOf<V>::T* __restrict__ vperm) {
  plane_body<Vg, V>(t, nsticks, stick_plane, p1, p2, ld, n3, tw1, tw2, vperm);
}
// the same for 128-thread CTAs of complex64 planes, compiled for ten resident CTAs per SM: the
// plane passes are latency-bound, and the register budget of the general form (one CTA of up
// to 512 threads) leaves eight
template <typename Vg, typename V>
__global__ void __launch_bounds__(128, 10) k_plane128(Vg* __restrict__ t, int nsticks,
                                                      const int* __restrict__ stick_plane, AxisPlan p1,
                                                      AxisPlan p2, int ld, int n3, const V* __restrict__ tw1,
                                                      const V* __restrict__ tw2,
                                                      const typename RealOf<V>::T* __restrict__ vperm) {
  plane_body<Vg, V>(t, nsticks, stick_plane, p1, p2, ld, n3, tw1, tw2, vperm);
}

// ---------------------------------------------------------------------------
// pass B split in three kernels, for planes too large for one CTA's shared memory (N1 LD
// sizeof(Vs) above the 227 KB limit, e.g. 120 x 121 complex128) or when chosen by the tuner.
// The plane of one (field, p3) goes through an L2-resident buffer P[field][p3][i1][LD] (rows in
// natural i1 order before the column transform, in DIF position order after it); every line
// transform is the same fft_lines call as in k_plane, so the results are the same bit for bit.
//   B1  rows r0 .. r0+nr-1: scatter their sticks, inverse FFT along axis 2     -> P
//   B2  columns c0 .. c0+nc-1 (DIF positions along axis 2): inverse FFT along axis 1,
//       x V/Ng, forward FFT along axis 1                                       -> P
//   B3  rows: forward FFT along axis 2, gather the sticks                      -> T
// ---------------------------------------------------------------------------
template <typename Vg, typename Vs>
__global__ void __launch_bounds__(256) k_plane_rows_inv(const Vg* __restrict__ t, Vs* __restrict__ pbuf, int nsticks,
                                                        const int* __restrict__ stick_plane, AxisPlan p2, int ld,
                                                        int n1, int n3, const Vs* __restrict__ tw2, int rpb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Vs* rows = reinterpret_cast<Vs*>(smem_raw);   // rpb rows of stride ld
  const int z = blockIdx.x, f = blockIdx.y, r0 = blockIdx.z * rpb;
  const int nr = min(rpb, n1 - r0);
  for (int e = threadIdx.x; e < nr * ld; e += blockDim.x) rows[e] = vzero<Vs>();
  __syncthreads();
  const Vg* src = t + ((size_t)f * n3 + z) * nsticks;
  const int lo = r0 * ld, hi = (r0 + nr) * ld;   // stick_plane = i1 LD + i2
  for (int s = threadIdx.x; s < nsticks; s += blockDim.x) {
    const int pos = stick_plane[s];
    if (pos >= lo && pos < hi) rows[pos - lo] = to_s<Vs>(src[s]);
  }
  __syncthreads();
  fft_lines<Vs, false, false>(rows, nr, ld, 1, p2, tw2);
  Vs* out = pbuf + (((size_t)f * n3 + z) * n1 + r0) * ld;
  for (int e = threadIdx.x; e < nr * ld; e += blockDim.x) out[e] = rows[e];
}

template <typename Vs>
__global__ void __launch_bounds__(256) k_plane_cols_v(Vs* __restrict__ pbuf, AxisPlan p1, int ld, int n2, int n3,
                                                      const Vs* __restrict__ tw1,
                                                      const typename RealOf<Vs>::T* __restrict__ vperm, int cpb,
                                                      int ls1) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Vs* cols = reinterpret_cast<Vs*>(smem_raw);   // cpb lines of stride ls1 (odd), element i1
  const int n1 = p1.n;
  const int z = blockIdx.x, f = blockIdx.y, c0 = blockIdx.z * cpb;
  const int ncl = min(cpb, n2 - c0);
  Vs* pl = pbuf + ((size_t)f * n3 + z) * (size_t)n1 * ld;
  const float rc = __fdividef(1.0f, (float)ncl);
  for (int e = threadIdx.x; e < n1 * ncl; e += blockDim.x) {
    const int i = qdiv(e, ncl, rc), c = e - i * ncl;
    cols[c * ls1 + i] = pl[(size_t)i * ld + c0 + c];
  }
  __syncthreads();
  fft_lines<Vs, false, false>(cols, ncl, ls1, 1, p1, tw1);
  const typename RealOf<Vs>::T* vz = vperm + (size_t)z * n1 * ld;
  for (int e = threadIdx.x; e < n1 * ncl; e += blockDim.x) {
    const int i = qdiv(e, ncl, rc), c = e - i * ncl;
    cols[c * ls1 + i] = cscale(cols[c * ls1 + i], vz[(size_t)i * ld + c0 + c]);
  }
  __syncthreads();
  fft_lines<Vs, true, true>(cols, ncl, ls1, 1, p1, tw1);
  for (int e = threadIdx.x; e < n1 * ncl; e += blockDim.x) {
    const int i = qdiv(e, ncl, rc), c = e - i * ncl;
    pl[(size_t)i * ld + c0 + c] = cols[c * ls1 + i];
  }
}

template <typename Vg, typename Vs>
__global__ void __launch_bounds__(256) k_plane_rows_fwd(Vg* __restrict__ t, const Vs* __restrict__ pbuf, int nsticks,
                                                        const int* __restrict__ stick_plane, AxisPlan p2, int ld,
                                                        int n1, int n3, const Vs* __restrict__ tw2, int rpb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Vs* rows = reinterpret_cast<Vs*>(smem_raw);
  const int z = blockIdx.x, f = blockIdx.y, r0 = blockIdx.z * rpb;
  const int nr = min(rpb, n1 - r0);
  const Vs* in = pbuf + (((size_t)f * n3 + z) * n1 + r0) * ld;
  for (int e = threadIdx.x; e < nr * ld; e += blockDim.x) rows[e] = in[e];
  __syncthreads();
  fft_lines<Vs, true, true>(rows, nr, ld, 1, p2, tw2);
  Vg* dst = t + ((size_t)f * n3 + z) * nsticks;
  const int lo = r0 * ld, hi = (r0 + nr) * ld;
  for (int s = threadIdx.x; s < nsticks; s += blockDim.x) {
    const int pos = stick_plane[s];
    if (pos >= lo && pos < hi) dst[s] = to_g(rows[pos - lo]);
  }
}

// density from the split plane: after B1, per (p3, column block) the inverse FFT along axis 1 of
// every field it owns and the weighted sum of |psi|^2, added into the DIF-ordered planes
__global__ void __launch_bounds__(256) k_plane_cols_density(const double2* __restrict__ pbuf, AxisPlan p1, int ld,
                                                            int n2, int n3, const double2* __restrict__ tw1,
                                                            const double* __restrict__ wfield, int nf, int fper,
                                                            int cpb, int ls1, double* __restrict__ rho_perm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n1 = p1.n;
  const int z = blockIdx.x, c0 = blockIdx.y * cpb, f0 = blockIdx.z * fper, f1 = min(nf, f0 + fper);
  const int ncl = min(cpb, n2 - c0);
  double2* cols = reinterpret_cast<double2*>(smem_raw);
  double* acc = reinterpret_cast<double*>(cols + (size_t)cpb * ls1);
  const float rc = __fdividef(1.0f, (float)ncl);
  for (int e = threadIdx.x; e < n1 * ncl; e += blockDim.x) acc[e] = 0.0;
  for (int f = f0; f < f1; ++f) {
    const double2* pl = pbuf + ((size_t)f * n3 + z) * (size_t)n1 * ld;
    for (int e = threadIdx.x; e < n1 * ncl; e += blockDim.x) {
      const int i = qdiv(e, ncl, rc), c = e - i * ncl;
      cols[c * ls1 + i] = pl[(size_t)i * ld + c0 + c];
    }
    __syncthreads();
    fft_lines<double2, false, false>(cols, ncl, ls1, 1, p1, tw1);
    const double w = wfield[f];
    for (int e = threadIdx.x; e < n1 * ncl; e += blockDim.x) {
      const int i = qdiv(e, ncl, rc), c = e - i * ncl;
      const double2 v = cols[c * ls1 + i];
      acc[e] = fma(w, fma(v.x, v.x, v.y * v.y), acc[e]);
    }
    __syncthreads();
  }
  double* out = rho_perm + (size_t)z * n1 * ld;
  for (int e = threadIdx.x; e < n1 * ncl; e += blockDim.x) {
    const int i = qdiv(e, ncl, rc), c = e - i * ncl;
    if (acc[e] != 0.0) atomicAdd(out + (size_t)i * ld + c0 + c, acc[e]);
  }
}

// ---------------------------------------------------------------------------
// electron density (Eq. density): pass A as above, then per plane the inverse 2D FFT of
// every field and the weighted sum of |psi|^2 over the fields, FP64 throughout.  The sum
// stays in shared memory across the fields a CTA owns; the planes are in the DIF-permuted
// order of the potential ([p3][p1*LD + p2]).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) k_plane_density(const double2* __restrict__ t, int nsticks,
                                                       const int* __restrict__ stick_plane, AxisPlan p1,
                                                       AxisPlan p2, int ld, int n3, const double2* __restrict__ tw1,
                                                       const double2* __restrict__ tw2,
                                                       const double* __restrict__ wfield, int nf, int fper,
                                                       double* __restrict__ rho_perm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n1 = p1.n, n2 = p2.n, np = n1 * ld;
  double2* plane = reinterpret_cast<double2*>(smem_raw);
  double* acc = reinterpret_cast<double*>(plane + np);
  const int z = blockIdx.x;
  const int f0 = blockIdx.y * fper, f1 = min(nf, f0 + fper);
  for (int e = threadIdx.x; e < np; e += blockDim.x) acc[e] = 0.0;
  for (int f = f0; f < f1; ++f) {
    for (int e = threadIdx.x; e < np; e += blockDim.x) plane[e] = double2{0.0, 0.0};
    __syncthreads();
    const double2* row = t + ((size_t)f * n3 + z) * nsticks;
    for (int s = threadIdx.x; s < nsticks; s += blockDim.x)
      if (dks_ok(stick_plane[s] >= 0 && stick_plane[s] < np, kChkPlaneDensity | (s & 0xffffff)))
        plane[stick_plane[s]] = row[s];
    __syncthreads();
    fft_lines<double2, false, false>(plane, n1, ld, 1, p2, tw2);
    fft_lines<double2, false, false>(plane, n2, 1, ld, p1, tw1);
    const double w = wfield[f];
    for (int e = threadIdx.x; e < np; e += blockDim.x) {
      const double2 v = plane[e];
      acc[e] = fma(w, fma(v.x, v.x, v.y * v.y), acc[e]);
    }
    __syncthreads();
  }
  double* out = rho_perm + (size_t)z * np;
  for (int e = threadIdx.x; e < np; e += blockDim.x)
    if (acc[e] != 0.0) atomicAdd(out + e, acc[e]);
}

// rho[(i1 N2 + i2) N3 + i3] += scale * rho_perm[(p3[i3] N1 + p1[i1]) LD + p2[i2]]
__global__ void k_unpermute_add(const double* __restrict__ rho_perm, double* __restrict__ rho, int n1, int n2,
                                int n3, int ld, const int* __restrict__ p1, const int* __restrict__ p2,
                                const int* __restrict__ p3, double scale) {
  const size_t ng = (size_t)n1 * n2 * n3;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < ng; n += (size_t)gridDim.x * blockDim.x) {
    const int i3 = (int)(n % n3);
    const size_t r = n / n3;
    const int i2 = (int)(r % n2), i1 = (int)(r / n2);
    const size_t at = ((size_t)p3[i3] * n1 + p1[i1]) * ld + p2[i2];
    if (dks_ok(at < (size_t)n3 * n1 * ld, kChkUnpermute | (unsigned)(n & 0xffffff))) rho[n] += scale * rho_perm[at];
  }
}

// ---------------------------------------------------------------------------
// pass C: forward FFT along axis 3, gather, Dirac term (FP64), shift, scale
// ---------------------------------------------------------------------------
__device__ __forceinline__ void dirac4(const double2 xv[4], double qx, double qy, double qz, double c,
                                       double diag_small, double shift, double2 h[4]) {
  // [[0, c s.q], [c s.q, -2c^2]] x - shift x ;  s.q = [[qz, qx - i qy], [qx + i qy, -qz]]
  const double2 qm = {c * qx, -c * qy};   // c (qx - i qy)
  const double2 qp = {c * qx, c * qy};    // c (qx + i qy)
  const double cz = c * qz;
  double2 a = cmul(qm, xv[3]);
  h[0] = {cz * xv[2].x + a.x - shift * xv[0].x, cz * xv[2].y + a.y - shift * xv[0].y};
  a = cmul(qp, xv[2]);
  h[1] = {a.x - cz * xv[3].x - shift * xv[1].x, a.y - cz * xv[3].y - shift * xv[1].y};
  a = cmul(qm, xv[1]);
  h[2] = {cz * xv[0].x + a.x + (diag_small - shift) * xv[2].x,
          cz * xv[0].y + a.y + (diag_small - shift) * xv[2].y};
  a = cmul(qp, xv[0]);
  h[3] = {a.x - cz * xv[1].x + (diag_small - shift) * xv[3].x,
          a.y - cz * xv[1].y + (diag_small - shift) * xv[3].y};
}

// sum_k c_k x_k for four double-float constants c_k = (h, l) and FP32 values x_k: exact FP32
// products with their rounding errors, two-sum of the leading parts; result as (hi, lo)
__device__ __forceinline__ dfl dsum4(float c1h, float c1l, float x1, float c2h, float c2l, float x2, float c3h,
                                     float c3l, float x3, float c4h, float c4l, float x4) {
  float s = c1h * x1;
  float r = fmaf(c1l, x1, fmaf(c1h, x1, -s));
  auto add = [&](float ch, float cl, float x) {
    const float p = ch * x;
    const float e = fmaf(cl, x, fmaf(ch, x, -p));
    const float t = s + p;
    const float bb = t - s;
    r += ((s - (t - bb)) + (p - bb)) + e;
    s = t;
  };
  add(c2h, c2l, x2);
  add(c3h, c3l, x3);
  add(c4h, c4l, x4);
  return dfl{s, r};
}

template <typename Vg, typename V>
__global__ void __launch_bounds__(256) k_stick_forward(
    const Vg* __restrict__ t, const Vg* __restrict__ x, Vg* __restrict__ out, int npw, int nsticks,
    const int* __restrict__ stick_start, const int* __restrict__ pw_stick, const int* __restrict__ pw_iz,
    AxisPlan p3, const V* __restrict__ tw3, const double* __restrict__ q, const float* __restrict__ cq32,
    double c, double shift, double scale, int spb, int ls) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* line = reinterpret_cast<V*>(smem_raw);   // 4*spb lines of stride ls (odd)
  const int n3 = p3.n;
  const int s0 = blockIdx.x * spb;
  const int ns = min(spb, nsticks - s0);
  const int b = blockIdx.y;
  const float rns = __fdividef(1.0f, (float)ns);
  for (int a = 0; a < 4; ++a) {
    const Vg* ta = t + (size_t)(b * 4 + a) * n3 * nsticks + s0;
    for (int e = threadIdx.x; e < ns * n3; e += blockDim.x) {
      const int z = qdiv(e, ns, rns), s = e - z * ns;
      line[(a * spb + s) * ls + z] = to_s<V>(ta[(size_t)z * nsticks + s]);
    }
  }
  __syncthreads();
  fft_lines<V, true, true>(line, 4 * spb, ls, 1, p3, tw3);
  const size_t fo = (size_t)b * 4 * npw;
  const int q0 = stick_start[s0], q1 = stick_start[s0 + ns];
  if constexpr (std::is_same<Vg, float2>::value && std::is_same<V, float2>::value) {
    // FP32 blocks: the large components in FP32; the small components, where c s.q x_L and
    // (2c^2 + shift) x_S nearly cancel, as double-float sums of exact products
    const double kd = 2.0 * c * c + shift;
    const float kh = (float)kd, kl = (float)(kd - (double)kh), sh = (float)shift, sc = (float)scale;
    for (int p = q0 + threadIdx.x; p < q1; p += blockDim.x) {
      const int s = pw_stick[p] - s0, iz = pw_iz[p];
      if (!dks_ok(s >= 0 && s < ns && iz >= 0 && iz < p3.n, kChkStickForward | (p & 0xffffff))) continue;
      const float2 x0 = x[fo + p], x1 = x[fo + (size_t)npw + p], x2 = x[fo + 2 * (size_t)npw + p],
                   x3 = x[fo + 3 * (size_t)npw + p];
      const float* cq = cq32 + 6 * (size_t)p;
      const float cxh = cq[0], cxl = cq[1], cyh = cq[2], cyl = cq[3], czh = cq[4], czl = cq[5];
      float2 h[4];
      h[0] = float2{czh * x2.x + cxh * x3.x + cyh * x3.y - sh * x0.x, czh * x2.y + cxh * x3.y - cyh * x3.x - sh * x0.y};
      h[1] = float2{cxh * x2.x - cyh * x2.y - czh * x3.x - sh * x1.x, cxh * x2.y + cyh * x2.x - czh * x3.y - sh * x1.y};
      const dfl h2r = dsum4(czh, czl, x0.x, cxh, cxl, x1.x, cyh, cyl, x1.y, -kh, -kl, x2.x);
      const dfl h2i = dsum4(czh, czl, x0.y, cxh, cxl, x1.y, -cyh, -cyl, x1.x, -kh, -kl, x2.y);
      const dfl h3r = dsum4(cxh, cxl, x0.x, -cyh, -cyl, x0.y, -czh, -czl, x1.x, -kh, -kl, x3.x);
      const dfl h3i = dsum4(cxh, cxl, x0.y, cyh, cyl, x0.x, -czh, -czl, x1.y, -kh, -kl, x3.y);
      const float2 l2 = line[(2 * spb + s) * ls + iz], l3 = line[(3 * spb + s) * ls + iz];
      h[2] = float2{h2r.h + (h2r.l + l2.x), h2i.h + (h2i.l + l2.y)};
      h[3] = float2{h3r.h + (h3r.l + l3.x), h3i.h + (h3i.l + l3.y)};
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const float2 loc = line[(a * spb + s) * ls + iz];
        h[a] = float2{h[a].x + loc.x, h[a].y + loc.y};
      }
#pragma unroll
      for (int a = 0; a < 4; ++a) out[fo + (size_t)a * npw + p] = float2{sc * h[a].x, sc * h[a].y};
    }
    return;
  }
  const double diag_small = -2.0 * c * c;
  for (int p = q0 + threadIdx.x; p < q1; p += blockDim.x) {
    const int s = pw_stick[p] - s0, iz = pw_iz[p];
    if (!dks_ok(s >= 0 && s < ns && iz >= 0 && iz < p3.n, kChkStickForward | (p & 0xffffff))) continue;
    double2 xv[4], h[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) xv[a] = to_d2(x[fo + (size_t)a * npw + p]);
    dirac4(xv, q[3 * p], q[3 * p + 1], q[3 * p + 2], c, diag_small, shift, h);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const double2 loc = to_d2(line[(a * spb + s) * ls + iz]);
      out[fo + (size_t)a * npw + p] = from_d2<Vg>({scale * (h[a].x + loc.x), scale * (h[a].y + loc.y)});
    }
  }
}

// KSSO two-spinors: forward z-transform of the V psi sticks of both components, gathered onto
// the sphere, plus the kinetic term: out = scale ((|k+G|^2/2 - shift) x + V psi)
template <typename Vg, typename V>
__global__ void __launch_bounds__(256) k_stick_forward_ks(
    const Vg* __restrict__ t, const Vg* __restrict__ x, Vg* __restrict__ out, int npw, int nsticks,
    const int* __restrict__ stick_start, const int* __restrict__ pw_stick, const int* __restrict__ pw_iz,
    AxisPlan p3, const V* __restrict__ tw3, const double* __restrict__ ek, double shift, double scale, int spb,
    int ls) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* line = reinterpret_cast<V*>(smem_raw);   // 2*spb lines of stride ls (odd)
  const int n3 = p3.n;
  const int s0 = blockIdx.x * spb;
  const int ns = min(spb, nsticks - s0);
  const int b = blockIdx.y;
  const float rns = __fdividef(1.0f, (float)ns);
  for (int a = 0; a < 2; ++a) {
    const Vg* ta = t + (size_t)(b * 2 + a) * n3 * nsticks + s0;
    for (int e = threadIdx.x; e < ns * n3; e += blockDim.x) {
      const int z = qdiv(e, ns, rns), s = e - z * ns;
      line[(a * spb + s) * ls + z] = to_s<V>(ta[(size_t)z * nsticks + s]);
    }
  }
  __syncthreads();
  fft_lines<V, true, true>(line, 2 * spb, ls, 1, p3, tw3);
  const size_t fo = (size_t)b * 2 * npw;
  const int q0 = stick_start[s0], q1 = stick_start[s0 + ns];
  for (int p = q0 + threadIdx.x; p < q1; p += blockDim.x) {
    const int s = pw_stick[p] - s0, iz = pw_iz[p];
    if (!dks_ok(s >= 0 && s < ns && iz >= 0 && iz < p3.n, kChkStickForwardKs | (p & 0xffffff))) continue;
    if constexpr (std::is_same<Vg, float2>::value && std::is_same<V, float2>::value) {
      const float kin = (float)(ek[p] - shift), sc = (float)scale;
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const float2 xv = x[fo + (size_t)a * npw + p], loc = line[(a * spb + s) * ls + iz];
        out[fo + (size_t)a * npw + p] = float2{sc * fmaf(kin, xv.x, loc.x), sc * fmaf(kin, xv.y, loc.y)};
      }
    } else {
      const double kin = ek[p] - shift;
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const double2 xv = to_d2(x[fo + (size_t)a * npw + p]), loc = to_d2(line[(a * spb + s) * ls + iz]);
        out[fo + (size_t)a * npw + p] = from_d2<Vg>({scale * fma(kin, xv.x, loc.x), scale * fma(kin, xv.y, loc.y)});
      }
    }
  }
}

// KSSO kinetic term alone (no local potential on the grid): fields of npw planewaves
template <typename V>
__global__ void k_kinetic_only(const V* __restrict__ x, V* __restrict__ out, int npw, int nfields,
                               const double* __restrict__ ek, double shift, double scale) {
  const size_t total = (size_t)nfields * npw;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(e % npw);
    const double k = scale * (ek[p] - shift);
    const double2 xv = to_d2(x[e]);
    out[e] = from_d2<V>({k * xv.x, k * xv.y});
  }
}

// Dirac term alone (no local potential on the grid)
template <typename V>
__global__ void k_dirac_only(const V* __restrict__ x, V* __restrict__ out, int npw, int nb,
                             const double* __restrict__ q, double c, double shift, double scale) {
  const size_t total = (size_t)nb * npw;
  const double diag_small = -2.0 * c * c;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t b = e / npw;
    const int p = (int)(e - b * npw);
    const size_t fo = b * 4 * npw;
    double2 xv[4], h[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) xv[a] = to_d2(x[fo + (size_t)a * npw + p]);
    dirac4(xv, q[3 * p], q[3 * p + 1], q[3 * p + 2], c, diag_small, shift, h);
#pragma unroll
    for (int a = 0; a < 4; ++a)
      out[fo + (size_t)a * npw + p] = from_d2<V>({scale * h[a].x, scale * h[a].y});
  }
}

// Eq. (RKB) in the planewave basis (p -> q = k+G, m = 1): small = (sigma.q) large / (2c).
// Complex128 data: FP64 arithmetic with q; complex64 data: FP32 arithmetic with the leading
// parts of c q (scaled by 1 / (2 c^2)).
__device__ __forceinline__ void kb_spinor(double qx, double qy, double qz, double2 u, double2 d, double2& s0,
                                          double2& s1) {
  s0 = double2{qz * u.x + qx * d.x + qy * d.y, qz * u.y + qx * d.y - qy * d.x};
  s1 = double2{qx * u.x - qy * u.y - qz * d.x, qx * u.y + qy * u.x - qz * d.y};
}
__device__ __forceinline__ void kb_spinor(float qx, float qy, float qz, float2 u, float2 d, float2& s0,
                                          float2& s1) {
  s0 = float2{qz * u.x + qx * d.x + qy * d.y, qz * u.y + qx * d.y - qy * d.x};
  s1 = float2{qx * u.x - qy * u.y - qz * d.x, qx * u.y + qy * u.x - qz * d.y};
}
__global__ void k_kinetic_balance64(double2* __restrict__ x, int npw, int nb, const double* __restrict__ q,
                                    double c) {
  const size_t total = (size_t)nb * npw;
  const double h = 0.5 / c;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t b = e / npw;
    const int p = (int)(e - b * npw);
    double2* xb = x + b * 4 * npw + p;
    double2 s0, s1;
    kb_spinor(h * q[3 * p], h * q[3 * p + 1], h * q[3 * p + 2], xb[0], xb[npw], s0, s1);
    xb[2 * (size_t)npw] = s0;
    xb[3 * (size_t)npw] = s1;
  }
}
__global__ void k_kinetic_balance32(float2* __restrict__ x, int npw, int nb, const float* __restrict__ cq,
                                    float h) {
  const size_t total = (size_t)nb * npw;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t b = e / npw;
    const int p = (int)(e - b * npw);
    float2* xb = x + b * 4 * npw + p;
    float2 s0, s1;
    kb_spinor(h * cq[6 * p], h * cq[6 * p + 2], h * cq[6 * p + 4], xb[0], xb[npw], s0, s1);
    xb[2 * (size_t)npw] = s0;
    xb[3 * (size_t)npw] = s1;
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <typename V>
static int set_smem(const void* fn, size_t bytes) {
  if (bytes > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return fail(DKS_ERR_CUDA, std::string("smem attribute: ") + cudaGetErrorString(e));
  }
  return DKS_OK;
}

static int pick_spb(int n3, size_t elem, int lines_per_stick, size_t target) {
  int spb = 32;
  while (spb > 1 && (size_t)spb * n3 * elem * lines_per_stick > target) spb >>= 1;
  return spb;
}

// Pass B in one kernel needs the whole N1 x LD plane in shared memory; larger planes (or a
// tuner's choice, ctx->plane_split) take the three-kernel form through the buffer P.
static bool split_plane(const dks_ctx* ctx, size_t elem) {
  return ctx->plane_split || (size_t)ctx->grid[0] * ctx->plane_ld * elem > 227 * 1024;
}
// rows (or columns) of a plane per CTA in the split form: about 64 KB of shared memory
static int lines_per_cta(int nlines, int line_stride, size_t elem, size_t extra_per_line = 0) {
  return std::max(1, std::min(nlines, (int)((64 * 1024) / (line_stride * elem + extra_per_line))));
}

// The three FFT passes over chunks of bands.  Vg is the storage type (global memory), Vs the
// arithmetic type of the transforms in shared memory: the same type, or double-float (cdf) for
// complex128 data in the emulated-FP64 mode.
template <typename Vg, typename Vs>
static int fft_local(dks_ctx* ctx, const KPoint& kp, const Vg* x, Vg* out, int nb, int chunk, Vg* tbuf, void* pbufv,
                     double shift, double scale, cudaStream_t st) {
  const bool fp64 = sizeof(Vg) == sizeof(double2);
  const bool df = !std::is_same<Vg, Vs>::value;
  const int npw = kp.npw, n3 = ctx->grid[2];
  const size_t field_elems = (size_t)kp.nsticks * n3;
  const Vs* tw1 = df ? (const Vs*)ctx->twdf[0] : fp64 ? (const Vs*)ctx->tw64[0] : (const Vs*)ctx->tw32[0];
  const Vs* tw2 = df ? (const Vs*)ctx->twdf[1] : fp64 ? (const Vs*)ctx->tw64[1] : (const Vs*)ctx->tw32[1];
  const Vs* tw3 = df ? (const Vs*)ctx->twdf[2] : fp64 ? (const Vs*)ctx->tw64[2] : (const Vs*)ctx->tw32[2];
  using VR = typename RealOf<Vs>::T;
  const VR* vp = df ? (const VR*)ctx->vpermdf : fp64 ? (const VR*)ctx->vperm64 : (const VR*)ctx->vperm32;
  const int ls = n3 | 1;                      // odd line stride: conflict-free shared memory
  const int ld = ctx->plane_ld;
  const int nc = ctx->ncomp;                   // fields per band: 4 (DKS) or 2 (KSSO)
  const int spb_a = pick_spb(ls, sizeof(Vs), 1, 32 * 1024);
  const int spb_c = pick_spb(ls, sizeof(Vs), nc, 64 * 1024);
  const size_t sm_a = (size_t)spb_a * ls * sizeof(Vs);
  const size_t sm_b = (size_t)ctx->grid[0] * ld * sizeof(Vs);
  const size_t sm_c = (size_t)nc * spb_c * ls * sizeof(Vs);
  // threads of the plane kernel: the largest pass has N1 N2 / (smallest radix) butterflies;
  int rmin = 8;
  for (int a = 0; a < 2; ++a)
    for (int i = 0; i < ctx->plan[a].nst; ++i) rmin = std::min(rmin, ctx->plan[a].radix[i]);
  // two butterflies per thread and pass (independent work for latency hiding, more CTAs per SM)
  const int nbf = ctx->grid[0] * ctx->grid[1] / rmin;
  const int tb_plane =
      ctx->plane_threads > 0 ? ctx->plane_threads : std::min(512, std::max(128, (nbf / 2 + 31) / 32 * 32));
  DKS_TRY(set_smem<Vs>((const void*)k_stick_inverse<Vg, Vs>, sm_a));
  const bool split = split_plane(ctx, sizeof(Vs));
  Vs* pbuf = reinterpret_cast<Vs*>(pbufv);
  const int n1 = ctx->grid[0], n2 = ctx->grid[1], ls1 = n1 | 1;
  const int rpb = lines_per_cta(n1, ld, sizeof(Vs)), cpb = lines_per_cta(n2, ls1, sizeof(Vs));
  const size_t sm_r = (size_t)rpb * ld * sizeof(Vs), sm_cv = (size_t)cpb * ls1 * sizeof(Vs);
  if (split) {
    if (!pbuf) return fail(DKS_ERR_INVALID_ARG, "split plane FFT without its buffer");
    DKS_TRY(set_smem<Vs>((const void*)k_plane_rows_inv<Vg, Vs>, sm_r));
    DKS_TRY(set_smem<Vs>((const void*)k_plane_cols_v<Vs>, sm_cv));
    DKS_TRY(set_smem<Vs>((const void*)k_plane_rows_fwd<Vg, Vs>, sm_r));
  } else {
    DKS_TRY(set_smem<Vs>((const void*)k_plane<Vg, Vs>, sm_b));
    if constexpr (std::is_same<Vs, float2>::value) DKS_TRY(set_smem<Vs>((const void*)k_plane128<Vg, Vs>, sm_b));
  }
  DKS_TRY(set_smem<Vs>(nc == 4 ? (const void*)k_stick_forward<Vg, Vs> : (const void*)k_stick_forward_ks<Vg, Vs>,
                       sm_c));
  const int cat32 = fp64 ? 0 : kProf32;
  for (int b0 = 0; b0 < nb; b0 += chunk) {
    const int nbc = std::min(chunk, nb - b0);
    const Vg* xb = x + (size_t)b0 * nc * npw;
    const double nf = (double)nc * nbc, es = (double)sizeof(Vg);
    const double tb = nf * (double)field_elems * es;          // one pass over the stick buffer
    const double f3 = 5.0 * n3 * std::log2((double)n3) * kp.nsticks * nf;
    {
      Prof pr(P_STICK_INV + cat32, st, nf * npw * es + tb, f3);
      dim3 ga((kp.nsticks + spb_a - 1) / spb_a, nc * nbc);
      k_stick_inverse<Vg, Vs><<<ga, 256, sm_a, st>>>(xb, tbuf, npw, kp.nsticks, kp.stick_start, kp.pw_stick,
                                                     kp.pw_iz, ctx->plan[2], tw3, spb_a, ls);
    }
    {
      const double nn = (double)ctx->grid[0] * ctx->grid[1];
      Prof pr(P_PLANE + cat32, st, 2.0 * tb + (double)ctx->ng * es / 2,
              nf * n3 * (10.0 * nn * std::log2(nn) + 2.0 * nn));
      if (split) {
        pr.count(2);
        const int nfi = nc * nbc;
        const dim3 g1(n3, nfi, (n1 + rpb - 1) / rpb), g2(n3, nfi, (n2 + cpb - 1) / cpb);
        k_plane_rows_inv<Vg, Vs><<<g1, 256, sm_r, st>>>(tbuf, pbuf, kp.nsticks, kp.stick_plane, ctx->plan[1], ld, n1,
                                                        n3, tw2, rpb);
        k_plane_cols_v<Vs><<<g2, 256, sm_cv, st>>>(pbuf, ctx->plan[0], ld, n2, n3, tw1, vp, cpb, ls1);
        k_plane_rows_fwd<Vg, Vs><<<g1, 256, sm_r, st>>>(tbuf, pbuf, kp.nsticks, kp.stick_plane, ctx->plan[1], ld, n1,
                                                        n3, tw2, rpb);
      } else {
        dim3 gb(n3, nc * nbc);
        bool launched = false;
        if constexpr (std::is_same<Vs, float2>::value) {
          if (tb_plane == 128) {
            k_plane128<Vg, Vs><<<gb, 128, sm_b, st>>>(tbuf, kp.nsticks, kp.stick_plane, ctx->plan[0],
                                                      ctx->plan[1], ld, n3, tw1, tw2, vp);
            launched = true;
          }
        }
        if (!launched)
          k_plane<Vg, Vs><<<gb, tb_plane, sm_b, st>>>(tbuf, kp.nsticks, kp.stick_plane, ctx->plan[0],
                                                      ctx->plan[1], ld, n3, tw1, tw2, vp);
      }
    }
    {
      Prof pr(P_STICK_FWD + cat32, st, tb + 2.0 * nf * npw * es + 24.0 * npw,
              f3 + (nc == 4 ? 64.0 : 8.0) * nbc * npw);
      dim3 gc((kp.nsticks + spb_c - 1) / spb_c, nbc);
      if (nc == 4)
        k_stick_forward<Vg, Vs><<<gc, 256, sm_c, st>>>(tbuf, xb, out + (size_t)b0 * 4 * npw, npw, kp.nsticks,
                                                       kp.stick_start, kp.pw_stick, kp.pw_iz, ctx->plan[2], tw3,
                                                       kp.q, kp.cq32, ctx->c, shift, scale, spb_c, ls);
      else
        k_stick_forward_ks<Vg, Vs><<<gc, 256, sm_c, st>>>(tbuf, xb, out + (size_t)b0 * 2 * npw, npw, kp.nsticks,
                                                          kp.stick_start, kp.pw_stick, kp.pw_iz, ctx->plan[2], tw3,
                                                          kp.ek, shift, scale, spb_c, ls);
    }
  }
  DKS_CUDA_TRY(cudaGetLastError());
  return DKS_OK;
}

template <typename V>
int apply_h(dks_ctx* ctx, Exec& ex, int ik, const V* x, V* out, int nb, double shift, double scale,
            cudaStream_t st) {
  if (nb <= 0) return DKS_OK;
  KPoint& kp = ctx->k[ik];
  const int npw = kp.npw;
  const bool fp64 = sizeof(V) == sizeof(double2);
  const int n3 = ctx->grid[2];
  const int nc = ctx->ncomp;
  const int ncol = nb * nc / 2;   // projector columns x~: two-spinors of 2 npw rows
  const size_t zp_elems = (size_t)ctx->nproj * ncol;
  const size_t field_elems = (size_t)kp.nsticks * n3;
  // split pass B: one N1 x LD plane per (field, p3) in the buffer P (the arithmetic type of the
  // transforms has the size of V: complex128 and double-float pairs are both 16 bytes)
  const size_t plane_elems = split_plane(ctx, sizeof(V)) ? (size_t)n3 * ctx->grid[0] * ctx->plane_ld : 0;
  // chunk of bands whose intermediates stay within the L2-resident budget
  int chunk = (int)std::max<size_t>(1, ctx->chunk_budget / (nc * (field_elems + plane_elems) * sizeof(V)));
  chunk = std::min(chunk, nb);
  const size_t zp_bytes = ((zp_elems * sizeof(double2) + 255) / 256) * 256;
  const size_t t_bytes = ctx->has_v ? ((nc * chunk * field_elems * sizeof(V) + 255) / 256) * 256 : 0;
  const size_t p_bytes = ctx->has_v ? nc * chunk * plane_elems * sizeof(V) : 0;
  DKS_TRY(grow(ex.ws_h, zp_bytes + t_bytes + p_bytes + 256));
  double2* zp = reinterpret_cast<double2*>(ex.ws_h.ptr);
  V* tbuf = reinterpret_cast<V*>(reinterpret_cast<char*>(ex.ws_h.ptr) + zp_bytes);
  void* pbuf = p_bytes ? reinterpret_cast<char*>(ex.ws_h.ptr) + zp_bytes + t_bytes : nullptr;
  const V* bt = nullptr;
  // refinement phase with DKS_TC_FP64: both projector contractions from exact integer slices of
  // x~ (made here) and of the projector table (made once per k-point)
  const bool ozp = fp64 && ex.df_gemm && ctx->nproj && tc_enabled(TC_FP64) && projector_slices(ctx, ik, st);
  OzBlock bto;
  if (ozp) DKS_TRY(oz_layout(kp.btoz, 2 * npw, ctx->nproj, &bto));
  if (ctx->nproj) {
    bt = fp64 ? reinterpret_cast<const V*>(kp.bt64) : reinterpret_cast<const V*>(kp.bt32);
    DKS_CUDA_TRY(cudaMemsetAsync(zp, 0, zp_elems * sizeof(double2), st));
    // Z = B^H x~ : (nproj x 2npw) (2npw x 2nb)
    if (ozp) {
      // x~ (2 npw x ncol) as the A operand, the table as B: Z = (x~^H B)^H
      DKS_TRY(grow(ex.ws_oz, oz_bytes(2 * npw, ncol)));
      OzBlock xo;
      DKS_TRY(oz_layout(ex.ws_oz.ptr, 2 * npw, ncol, &xo));
      DKS_TRY(oz_split((const double2*)x, 2 * npw, ncol, xo, st));
      DKS_TRY(oz_gemm_hn(xo, ncol, bto, ctx->nproj, zp, ctx->nproj, true, st, P_PROJ_HN));
    } else if (fp64 && ex.df_gemm)
      DKS_TRY(gemm_hn_df(kp.btdf, 2 * npw, (const double2*)x, 2 * npw, 2 * npw, ctx->nproj, ncol, zp, st,
                         P_PROJ_HN));
    else
      DKS_TRY(gemm_hn<V>(bt, 2 * npw, x, 2 * npw, 2 * npw, ctx->nproj, ncol, zp, st, P_PROJ_HN, 0, false,
                         ctx->tc_proj));
  }
  if (ctx->has_v) {
    bool done = false;
    if constexpr (std::is_same<V, double2>::value) {
      if (ex.df_gemm) {
        DKS_TRY((fft_local<double2, cdf>(ctx, kp, x, out, nb, chunk, tbuf, pbuf, shift, scale, st)));
        done = true;
      }
    }
    if (!done) DKS_TRY((fft_local<V, V>(ctx, kp, x, out, nb, chunk, tbuf, pbuf, shift, scale, st)));
  } else if (nc == 4) {
    const int blocks = std::max(1, std::min(ctx->num_sms * 8, (int)(((size_t)nb * npw + 255) / 256)));
    Prof pr(P_DIRAC + (fp64 ? 0 : kProf32), st, 8.0 * nb * npw * sizeof(V) + 24.0 * npw, 64.0 * nb * npw);
    k_dirac_only<V><<<blocks, 256, 0, st>>>(x, out, npw, nb, kp.q, ctx->c, shift, scale);
  } else {
    const int blocks = std::max(1, std::min(ctx->num_sms * 8, (int)(((size_t)2 * nb * npw + 255) / 256)));
    Prof pr(P_DIRAC + (fp64 ? 0 : kProf32), st, 4.0 * nb * npw * sizeof(V) + 8.0 * npw, 8.0 * nb * npw);
    k_kinetic_only<V><<<blocks, 256, 0, st>>>(x, out, npw, 2 * nb, kp.ek, shift, scale);
  }
  DKS_CUDA_TRY(cudaGetLastError());
  if (ctx->nproj) {
    // out~ += B (scale D Z)
    if (ozp)
      DKS_TRY(oz_rotate(bto, 0, ctx->nproj, zp, ctx->nproj, ncol, (double2*)out, 2 * npw, 1.0, st, scale,
                        ctx->dvec_dev, P_PROJ_NN));
    else if (fp64 && ex.df_gemm)
      DKS_TRY(gemm_nn_df(kp.btdf, 2 * npw, 2 * npw, ctx->nproj, zp, ctx->nproj, ctx->dvec_dev, ncol,
                         (double2*)out, 2 * npw, 1.0, st, scale, P_PROJ_NN));
    else
      DKS_TRY(gemm_nn<V>(bt, 2 * npw, 2 * npw, ctx->nproj, zp, ctx->nproj, ctx->dvec_dev, ncol, out, 2 * npw,
                         1.0, st, scale, P_PROJ_NN, ctx->tc_proj));
  }
  return DKS_OK;
}

int density_accumulate(dks_ctx* ctx, int ik, const double2* x, int nb, const double* occ, double* rho,
                       cudaStream_t st) {
  if (nb <= 0) return DKS_OK;
  KPoint& kp = ctx->k[ik];
  Exec& ex = exec0(ctx);
  const int npw = kp.npw, nc = ctx->ncomp;
  const int n1 = ctx->grid[0], n2 = ctx->grid[1], n3 = ctx->grid[2], ld = ctx->plane_ld;
  const size_t field_elems = (size_t)kp.nsticks * n3;
  const size_t np = (size_t)n1 * ld;
  const size_t sm_b = np * (sizeof(double2) + sizeof(double));
  // one plane per CTA (the plane and its |psi|^2 sum in shared memory), or the split form: rows
  // by k_plane_rows_inv into the buffer P, then columns by k_plane_cols_density
  const bool split = ctx->plane_split || sm_b > 227 * 1024;
  const size_t plane_elems = split ? (size_t)n3 * np : 0;
  int chunk = (int)std::max<size_t>(1, ctx->chunk_budget / (nc * (field_elems + plane_elems) * sizeof(double2)));
  chunk = std::min(chunk, nb);
  const size_t perm_bytes = ((n3 * np * sizeof(double) + 255) / 256) * 256;
  const size_t w_bytes = ((nc * (size_t)nb * sizeof(double) + 255) / 256) * 256;
  const size_t t_bytes = ((nc * (size_t)chunk * field_elems * sizeof(double2) + 255) / 256) * 256;
  DKS_TRY(grow(ex.ws_h, perm_bytes + w_bytes + t_bytes + nc * (size_t)chunk * plane_elems * sizeof(double2)));
  double* rho_perm = reinterpret_cast<double*>(ex.ws_h.ptr);
  double* wf = reinterpret_cast<double*>(reinterpret_cast<char*>(ex.ws_h.ptr) + perm_bytes);
  double2* tbuf = reinterpret_cast<double2*>(reinterpret_cast<char*>(ex.ws_h.ptr) + perm_bytes + w_bytes);
  double2* pbuf = reinterpret_cast<double2*>(reinterpret_cast<char*>(ex.ws_h.ptr) + perm_bytes + w_bytes + t_bytes);
  const int ls1 = n1 | 1;
  const int rpb = lines_per_cta(n1, ld, sizeof(double2));
  const int cpb = lines_per_cta(n2, ls1, sizeof(double2), (size_t)n1 * sizeof(double));
  const size_t sm_r = (size_t)rpb * ld * sizeof(double2);
  const size_t sm_cd = (size_t)cpb * (ls1 * sizeof(double2) + n1 * sizeof(double));
  std::vector<double> wh((size_t)nc * nb);
  for (int b = 0; b < nb; ++b)
    for (int c = 0; c < nc; ++c) wh[(size_t)b * nc + c] = occ[b];
  DKS_CUDA_TRY(cudaMemcpyAsync(wf, wh.data(), wh.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  DKS_CUDA_TRY(cudaMemsetAsync(rho_perm, 0, n3 * np * sizeof(double), st));
  const int ls = n3 | 1;
  const int spb_a = pick_spb(ls, sizeof(double2), 1, 32 * 1024);
  const size_t sm_a = (size_t)spb_a * ls * sizeof(double2);
  DKS_TRY(set_smem<double2>((const void*)k_stick_inverse<double2, double2>, sm_a));
  if (split) {
    DKS_TRY(set_smem<double2>((const void*)k_plane_rows_inv<double2, double2>, sm_r));
    DKS_TRY(set_smem<double2>((const void*)k_plane_cols_density, sm_cd));
  } else {
    DKS_TRY(set_smem<double2>((const void*)k_plane_density, sm_b));
  }
  int rmin = 8;
  for (int a = 0; a < 2; ++a)
    for (int i = 0; i < ctx->plan[a].nst; ++i) rmin = std::min(rmin, ctx->plan[a].radix[i]);
  const int nbf = n1 * n2 / rmin;
  const int tb_plane = std::min(512, std::max(128, (nbf / 2 + 31) / 32 * 32));
  for (int b0 = 0; b0 < nb; b0 += chunk) {
    const int nbc = std::min(chunk, nb - b0);
    const int nf = nc * nbc;
    const double es = sizeof(double2), tb = (double)nf * field_elems * es;
    {
      Prof pr(P_STICK_INV, st, (double)nf * npw * es + tb, 5.0 * n3 * std::log2((double)n3) * kp.nsticks * nf);
      dim3 ga((kp.nsticks + spb_a - 1) / spb_a, nf);
      k_stick_inverse<double2, double2><<<ga, 256, sm_a, st>>>(x + (size_t)b0 * nc * npw, tbuf, npw, kp.nsticks,
                                                               kp.stick_start, kp.pw_stick, kp.pw_iz, ctx->plan[2],
                                                               ctx->tw64[2], spb_a, ls);
    }
    {
      // split the fields of a plane over enough CTAs to fill the GPU twice; atomics combine them
      const int nsplit = std::max(1, std::min(nf, (2 * ctx->num_sms + n3 - 1) / n3));
      const int fper = (nf + nsplit - 1) / nsplit;
      const double nn = (double)n1 * n2;
      Prof pr(P_SCF, st, tb + 2.0 * n3 * np * sizeof(double), nf * n3 * (5.0 * nn * std::log2(nn) + 3.0 * nn));
      if (split) {
        pr.count(1);
        const dim3 g1(n3, nf, (n1 + rpb - 1) / rpb);
        k_plane_rows_inv<double2, double2><<<g1, 256, sm_r, st>>>(tbuf, pbuf, kp.nsticks, kp.stick_plane,
                                                                  ctx->plan[1], ld, n1, n3, ctx->tw64[1], rpb);
        const dim3 g2(n3, (n2 + cpb - 1) / cpb, (nf + fper - 1) / fper);
        k_plane_cols_density<<<g2, 256, sm_cd, st>>>(pbuf, ctx->plan[0], ld, n2, n3, ctx->tw64[0],
                                                     wf + (size_t)b0 * nc, nf, fper, cpb, ls1, rho_perm);
      } else {
        dim3 gb(n3, (nf + fper - 1) / fper);
        k_plane_density<<<gb, tb_plane, sm_b, st>>>(tbuf, kp.nsticks, kp.stick_plane, ctx->plan[0], ctx->plan[1], ld,
                                                    n3, ctx->tw64[0], ctx->tw64[1], wf + (size_t)b0 * nc, nf, fper,
                                                    rho_perm);
      }
    }
  }
  {
    const size_t ng = (size_t)ctx->ng;
    Prof pr(P_SCF, st, 3.0 * ng * sizeof(double), 2.0 * ng);
    const int blocks = (int)std::min<size_t>((ng + 255) / 256, (size_t)ctx->num_sms * 8);
    k_unpermute_add<<<blocks, 256, 0, st>>>(rho_perm, rho, n1, n2, n3, ld, ctx->posd[0], ctx->posd[1], ctx->posd[2],
                                            1.0 / ctx->volume);
  }
  DKS_CUDA_TRY(cudaGetLastError());
  return DKS_OK;
}

// the first failed index check of this file's kernels since the last call, then cleared
// (debug build; 0 in the product build)
unsigned debug_check_take() {
#ifdef DKS_DEBUG
  unsigned v = 0u, z = 0u;
  if (cudaMemcpyFromSymbol(&v, g_dks_check, sizeof(v)) != cudaSuccess) return 0xffffffffu;
  cudaMemcpyToSymbol(g_dks_check, &z, sizeof(z));
  return v;
#else
  return 0u;
#endif
}

int kinetic_balance(dks_ctx* ctx, int ik, void* x, int nb, bool fp64, cudaStream_t st) {
  const KPoint& kp = ctx->k[ik];
  const size_t total = (size_t)nb * kp.npw;
  if (!total) return DKS_OK;
  const int blocks = (int)std::min<size_t>((total + 255) / 256, (size_t)ctx->num_sms * 8);
  Prof pr(P_MISC, st, 2.0 * total * 2 * (fp64 ? 16.0 : 8.0) + 24.0 * kp.npw, 16.0 * total);
  if (fp64)
    k_kinetic_balance64<<<blocks, 256, 0, st>>>((double2*)x, kp.npw, nb, kp.q, ctx->c);
  else
    k_kinetic_balance32<<<blocks, 256, 0, st>>>((float2*)x, kp.npw, nb, kp.cq32, (float)(0.5 / (ctx->c * ctx->c)));
  DKS_CUDA_TRY(cudaGetLastError());
  return DKS_OK;
}

template int apply_h<double2>(dks_ctx*, Exec&, int, const double2*, double2*, int, double, double, cudaStream_t);
template int apply_h<float2>(dks_ctx*, Exec&, int, const float2*, float2*, int, double, double, cudaStream_t);

}  // namespace dks

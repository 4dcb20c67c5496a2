// dks_rayleigh_ritz_static: the device Rayleigh-Ritz solve with its scratch space in a
// fixed, file-scope device array instead of memory allocated per call.
//
// Why: some callers cannot allocate device memory at the point where they need this
// solve -- for example a service that hands all device memory to its own arena at start-up
// and forbids later cudaMalloc/cudaFree, or a latency-critical host thread that must not
// risk the device-wide synchronisation an allocation or free can cause.  Such callers pass
// only their inputs and outputs; the scratch space (about 1.6 MB) is reserved once in every
// process that loads the library, on every device it touches, until the process exits.
//
// Contract:
//  * nz <= DKS_RR_STATIC_MAX_NZ (128); larger pencils are rejected with DKS_ERR_UNSUPPORTED
//    before anything is launched.
//  * The first call on a device looks up the device address of the array (with that device
//    current) and caches it; make that first call before any stream capture begins.
//  * All calls on a device share one array and it keeps whatever the previous call left in
//    it.  The kernel writes every scratch element before reading it, so nothing has to be
//    cleared between calls; calls whose executions overlap on the GPU (different streams
//    without ordering) race on the array and must be serialised by the caller.
//  * The array used is the current device's, so the stream must belong to the current device
//    (a stream of another device is rejected with DKS_ERR_INVALID_ARG).
//  * No cudaMalloc, cudaFree or other allocating routine is called.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "dks_internal.h"

namespace dks {

constexpr int kStaticMaxNz = DKS_RR_STATIC_MAX_NZ;
constexpr size_t kStaticElems = (size_t)6 * kStaticMaxNz * kStaticMaxNz + (size_t)16 * kStaticMaxNz + 64;

static __device__ __align__(256) double2 g_rr_static_scratch[kStaticElems];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
double2* g_static_ptr[kMaxDevices] = {nullptr};

// device address of the array for the current device (host code cannot use the symbol itself)
int static_scratch(double2** out) {
  int dev = 0;
  DKS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(DKS_ERR_UNSUPPORTED, "device index above 63");
  std::lock_guard<std::mutex> g(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_rr_static_scratch);
    if (e != cudaSuccess || !p)
      return fail(DKS_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    g_static_ptr[dev] = static_cast<double2*>(p);
  }
  *out = g_static_ptr[dev];
  return DKS_OK;
}
}  // namespace

static_assert(kStaticElems >= (size_t)6 * kStaticMaxNz * kStaticMaxNz + 16 * kStaticMaxNz + 64,
              "static scratch smaller than the Rayleigh-Ritz kernel needs");

}  // namespace dks

using namespace dks;

extern "C" int dks_rayleigh_ritz_static(const void* A, const void* S, int nz, int n, void* V, double* lam, int* info,
                                        void* stream) {
  if (!A || !S || !V || !lam || !info) return fail(DKS_ERR_INVALID_ARG, "dks_rayleigh_ritz_static: NULL pointer");
  if (nz <= 0 || n <= 0 || n > nz) return fail(DKS_ERR_INVALID_ARG, "dks_rayleigh_ritz_static: need 0 < n <= nz");
  if (nz > kStaticMaxNz)
    return fail(DKS_ERR_UNSUPPORTED, "dks_rayleigh_ritz_static: nz = " + std::to_string(nz) +
                                         " exceeds the static scratch limit " + std::to_string(kStaticMaxNz));
  if (rr_scratch_elems(nz) > kStaticElems)
    return fail(DKS_ERR_UNSUPPORTED, "dks_rayleigh_ritz_static: scratch requirement exceeds the static array");
  if (stream) {
    // the scratch array is the current device's: a stream of another device would run the
    // kernels there with this device's address
    int dev = 0, sdev = 0;
    DKS_CUDA_TRY(cudaGetDevice(&dev));
    DKS_CUDA_TRY(cudaStreamGetDevice((cudaStream_t)stream, &sdev));
    if (sdev != dev) return fail(DKS_ERR_INVALID_ARG, "dks_rayleigh_ritz_static: stream belongs to another device");
  }
  double2* scr = nullptr;
  DKS_TRY(static_scratch(&scr));
  return rayleigh_ritz((const double2*)A, (const double2*)S, nz, n, (double2*)V, lam, info, scr,
                       (cudaStream_t)stream);
}

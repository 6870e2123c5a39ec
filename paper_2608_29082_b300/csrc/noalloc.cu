// mg_smooth_noalloc: the learnable smoothing step without any allocation.
//
// Some callers cannot call cudaMalloc: a host application that owns all
// device memory (a fixed budget or its own pool) and does not let plug-ins
// allocate, or a latency-critical loop where an allocation's implicit device
// synchronisation is not acceptable.  This entry point runs nu smoothing
// steps on an operator the caller already holds in device memory (CSR) and
// keeps its only intermediate, the scaled residual delta, in the file-scope
// array below instead of in a context's workspace.
//
// The array is MG_NOALLOC_MAX_ELEMS doubles (4 MiB) and is resident on every
// GPU that loads this library until the process exits.  All calls share it
// and it keeps the last call's contents; nothing in it needs to start at zero
// (each step writes delta for every row before any row reads it).  Calls that
// overlap on the GPU (different streams, or different host threads on the
// same device) race on it.
#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

#include <cuda_runtime.h>

#include "mg.h"
#include "mg_internal.h"

namespace {

constexpr int kNoAllocThreads = 256;

static __device__ __align__(256) double g_noalloc_delta[MG_NOALLOC_MAX_ELEMS];

// Device address of g_noalloc_delta per device, looked up once per device
// with that device current.
std::mutex g_addr_mu;
double* g_addr[64] = {nullptr};

// delta = theta * (f - A u) / A_ii on CSR rows (diagonal found in the row).
__global__ void __launch_bounds__(kNoAllocThreads)
    k_noalloc_delta(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                    const double* __restrict__ val, const double* __restrict__ f,
                    const double* __restrict__ u, double* __restrict__ delta, int B, double theta) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)n * B) return;
  const int i = (int)(t / B), b = (int)(t - (size_t)i * B);
  double diag = 0.0, ax = 0.0;
  for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
    const int c = col[e];
    if (c == i)
      diag += val[e];
    else
      ax = fma(val[e], u[(size_t)c * B + b], ax);
  }
  const double r = fma(-diag, u[t], f[t]) - ax;
  delta[t] = theta * (r * (1.0 / diag));
}

// u += eta * (w1 delta_i + w2 * inv_deg_i * sum over graph neighbours of delta)
__global__ void __launch_bounds__(kNoAllocThreads)
    k_noalloc_update(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                     const double* __restrict__ val, const double* __restrict__ inv_deg,
                     const double* __restrict__ delta, double* __restrict__ u, int B, double eta,
                     double w1, double w2) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)n * B) return;
  const int i = (int)(t / B), b = (int)(t - (size_t)i * B);
  double s = 0.0;
  for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
    const int c = col[e];
    if (c != i && val[e] != 0.0) s += delta[(size_t)c * B + b];
  }
  const double phi = fma(w1, delta[t], w2 * (inv_deg[i] * s));
  u[t] = fma(eta, phi, u[t]);
}

}  // namespace

extern "C" mg_status mg_smooth_noalloc(int32_t n, const int32_t* rowptr, const int32_t* col,
                                       const double* val, const double* inv_deg, const double* f,
                                       double* u, int32_t nrhs, int32_t nu, double theta,
                                       double eta, double w1, double w2, void* stream) {
  if (n < 1 || nrhs < 1 || nu < 0 || !rowptr || !col || !val || !inv_deg || !f || !u)
    return mgi::set_global_error(MG_ERR_INVALID, "mg_smooth_noalloc: invalid arguments");
  if ((long long)n * nrhs > (long long)MG_NOALLOC_MAX_ELEMS)
    return mgi::set_global_error(
        MG_ERR_INVALID, "mg_smooth_noalloc: n * nrhs = " + std::to_string((long long)n * nrhs) +
                            " exceeds the static scratch of " +
                            std::to_string(MG_NOALLOC_MAX_ELEMS) + " doubles");
  {
    // f and u are [n][nrhs] doubles each: the byte ranges must be disjoint
    // (u is written while other threads still read f).
    const uintptr_t fb = (uintptr_t)f, ub = (uintptr_t)u;
    const uintptr_t len = (uintptr_t)n * (uintptr_t)nrhs * sizeof(double);
    if (fb < ub + len && ub < fb + len)
      return mgi::set_global_error(MG_ERR_INVALID, "mg_smooth_noalloc: f and u overlap");
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64)
    return mgi::set_global_error(MG_ERR_CUDA, "mg_smooth_noalloc: no current device");
  double* delta = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[dev]) {
      // The host-side name g_noalloc_delta is a stand-in, not a device
      // address: ask the runtime for this device's copy.
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_delta);
      if (e != cudaSuccess || !p)
        return mgi::set_global_error(
            MG_ERR_CUDA, std::string("mg_smooth_noalloc: cudaGetSymbolAddress: ") +
                             cudaGetErrorString(e));
      g_addr[dev] = (double*)p;
    }
    delta = g_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t work = (size_t)n * nrhs;
  const dim3 grid((unsigned)((work + kNoAllocThreads - 1) / kNoAllocThreads));
  for (int k = 0; k < nu; ++k) {
    k_noalloc_delta<<<grid, kNoAllocThreads, 0, s>>>(n, rowptr, col, val, f, u, delta, nrhs, theta);
    k_noalloc_update<<<grid, kNoAllocThreads, 0, s>>>(n, rowptr, col, val, inv_deg, delta, u, nrhs,
                                                      eta, w1, w2);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return mgi::set_global_error(MG_ERR_CUDA, std::string("mg_smooth_noalloc: launch: ") +
                                                  cudaGetErrorString(e));
  return MG_OK;
}

// Allocation-free periodic cubic B-spline interpolation.
//
// Who needs it: programs that may not allocate device memory while they run.
// Typical cases are applications whose device memory is owned by another
// framework's caching allocator (which may already have reserved nearly all
// of HBM, so a foreign cudaMalloc fails or fragments its pool), and
// latency-critical loops that cannot afford cudaMalloc/cudaFree, which can
// block the host and implicitly synchronise the device. Such callers can
// still pass their own input and output buffers; the only extra memory this
// path needs, the spline coefficients of the input, lives in the fixed
// array below, which every GPU that loads the library keeps until the
// process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"
#include "kernels.h"
#include "reg.h"

// Scratch for the spline coefficients of one field: REG_STATIC_MAX_POINTS
// floats (4 MiB), shared by every call in the process. In host code this
// name is only a stand-in; kernels get the address from cudaGetSymbolAddress.
static __device__ __align__(256) float g_static_coef[REG_STATIC_MAX_POINTS];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
float* g_static_ptr[kMaxDevices] = {};

bool size_ok(int n) { return n % 32 == 0 && regnk::fft_size_supported(n); }

}  // namespace

extern "C" reg_status reg_interpolate_static(int n1, int n2, const float* u, const float* disp,
                                             float* out, void* cuda_stream) {
  if (!u || !disp || !out) return REG_EINVAL;
  if (!size_ok(n1) || !size_ok(n2)) return REG_EINVAL;
  // vector loads and stores: every buffer starts on a 16-byte boundary
  if ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(disp) |
       reinterpret_cast<uintptr_t>(out)) & 15u)
    return REG_EINVAL;
  if ((long long)n1 * n2 > (long long)REG_STATIC_MAX_POINTS) return REG_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return REG_ECUDA;
  float* coef = nullptr;
  {
    // first call on this device: look up the device address of the array
    // (host code only holds a stand-in for it) with this device current
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_static_coef) != cudaSuccess || !p) return REG_ECUDA;
      g_static_ptr[dev] = static_cast<float*>(p);
    }
    coef = g_static_ptr[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // A launch error left pending by earlier, unrelated work is not this
  // call's failure: take it off the error slot here, so that only an error
  // raised by the two launches below turns into REG_ECUDA. (An error that
  // has made the context unusable fails these launches too.)
  (void)cudaGetLastError();
  // every coefficient is written by the prefilter before the gather reads it,
  // so nothing has to be cleared between calls
  regnk::launch_prefilter(n1, n2, u, nullptr, coef, 1, st);
  regnk::launch_gather(n1, n2, coef, disp, out, 1, 0, /*lagrange=*/0, st);
  return cudaGetLastError() == cudaSuccess ? REG_OK : REG_ECUDA;
}

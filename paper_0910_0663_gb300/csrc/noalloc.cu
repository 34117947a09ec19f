// vtm_residual_norm_noalloc: the FP64 residual norms of vtm_residual_norm
// without a plan and without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need a
// residual: a simulator whose memory pool already owns the whole device, a
// real-time loop that must not call cudaMalloc (which can synchronise the
// device and can fail under a fixed memory budget), or host code that only
// holds device buffers handed to it by someone else.  This entry point takes
// the matrix and the vectors from the caller and keeps its only scratch (the
// per-block partial sums, the completion counter and the two sums per column)
// in a file-scope __device__ array of fixed size that every GPU loading the
// library holds until the process exits.
#include <cmath>
#include <mutex>

#include "vtm_internal.h"

namespace {

constexpr int kMaxRhs = 64;       // columns per call
constexpr int kMaxBlocks = 1216;  // blocks of the residual kernel (8 per SM on 152 SMs)
constexpr int kCounterDoubles = 32;  // counter word, padded to 256 bytes
constexpr int kScratchDoubles = kCounterDoubles + 2 * kMaxRhs + 2 * kMaxBlocks;  // 20,736 bytes

// Shared by every call on a device; keeps the contents of the last call.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 128;
std::mutex g_mutex;
double* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).
vtm_status scratch_on_current_device(double** out) {
  int dev = 0;
  VTM_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return VTM_EINVAL;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      vtm::set_detail(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return VTM_ECUDA;
    }
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return VTM_OK;
}

// True if p is device memory of device `dev`, or managed memory (which any
// device may touch).  Memory of another device would be read over the
// interconnect at best and fault without peer access at worst.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" vtm_status vtm_residual_norm_noalloc(int64_t n, const int64_t* rowptr,
                                                const int32_t* colidx, const double* vals,
                                                const double* x, const double* b, int64_t nrhs,
                                                double* rel, void* stream) {
  if (n <= 0 || n > INT32_MAX || !rowptr || !colidx || !vals || !x || !b || !rel) {
    vtm::set_detail("vtm_residual_norm_noalloc: bad n or NULL argument");
    return VTM_EINVAL;
  }
  if (nrhs <= 0 || nrhs > kMaxRhs) {
    vtm::set_detail("vtm_residual_norm_noalloc: nrhs must be in 1.." + std::to_string(kMaxRhs) +
                    " (size of the static scratch)");
    return VTM_EINVAL;
  }
  int dev = 0;
  VTM_CUDA_TRY(cudaGetDevice(&dev));
  if (!on_device(rowptr, dev) || !on_device(colidx, dev) || !on_device(vals, dev) || !on_device(x, dev) ||
      !on_device(b, dev)) {
    vtm::set_detail("vtm_residual_norm_noalloc: matrix and vectors must be device memory of the "
                    "current device (" + std::to_string(dev) + ")");
    return VTM_EINVAL;
  }
  double* scratch = nullptr;
  VTM_TRY(scratch_on_current_device(&scratch));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned* counter = reinterpret_cast<unsigned*>(scratch);
  double* sums = scratch + kCounterDoubles;                 // (||r||^2, ||b||^2) per column
  double* partials = sums + 2 * kMaxRhs;                    // 2 * kMaxBlocks
  // the completion counter must start at zero whatever the last call left
  VTM_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned), s));
  for (int64_t c = 0; c < nrhs; ++c) {
    vtm::launch_residual(rowptr, colidx, vals, x + c * n, b + c * n, n, partials, counter,
                         sums + 2 * c, kMaxBlocks, s);
    VTM_CUDA_TRY(cudaGetLastError());
  }
  double h[2 * kMaxRhs];
  VTM_CUDA_TRY(cudaMemcpyAsync(h, sums, 2 * nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
  VTM_CUDA_TRY(cudaStreamSynchronize(s));
  for (int64_t c = 0; c < nrhs; ++c) {
    const double rr = h[2 * c], bb = h[2 * c + 1];
    rel[c] = bb > 0 ? std::sqrt(rr / bb) : std::sqrt(rr);
  }
  return VTM_OK;
}

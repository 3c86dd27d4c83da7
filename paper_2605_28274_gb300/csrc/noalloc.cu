// sylv_spmm_noalloc: the sparse block product Y = A X of sylv_apply for callers
// that must not allocate device memory.
//
// Who needs it: code that runs in a process whose device memory is owned by
// another allocator (for example a framework's caching pool that has reserved
// the device memory budget, so a raw cudaMalloc fails or fragments it), and
// latency-bound loops that cannot afford cudaMalloc/cudaFree, which can
// synchronise the whole device.  sylv_apply stages X and Y in buffers it
// allocates per call; this entry point stages them in one fixed array that is
// part of the library image instead, so a call allocates nothing.
//
// The staging array below is a file-scope __device__ array: every GPU that
// loads this library holds it (SYLV_NOALLOC_MAX_ELEMS doubles for X plus the
// same for Y, 16 MiB in total) until the process exits.  In host code the
// array's name is only a host-side stand-in; its device address is obtained
// once per device with cudaGetSymbolAddress (with that device current) and
// passed to the kernels.  That address belongs to the device's primary context: after
// cudaDeviceReset the process must not call this entry point again on that device.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/sylv.h"
#include "kernels.h"

namespace {

// X staging in [0, MAX), Y staging in [MAX, 2 MAX).  Every call overwrites the
// parts it reads before reading them, so nothing here has to start at zero.
static __device__ __align__(256) double g_noalloc_scratch[2 * SYLV_NOALLOC_MAX_ELEMS];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};


// Device address of the staging array on the current device (set up on first use).
int scratch_address(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    sylv::set_last_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return SYLV_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    sylv::set_last_error("device ordinal out of range");
    return SYLV_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_scratch_addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      sylv::set_last_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return SYLV_ECUDA;
    }
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return SYLV_OK;
}

// Every pointer must be device (or managed) memory of the current device: the staging array is
// the current device's, and a kernel given another device's or a host pointer would fault.
// cudaPointerGetAttributes allocates nothing.
int check_device_pointers(const int32_t* row_ptr, const int32_t* col_idx, const double* val, const double* X,
                          const double* Y, int64_t nnz) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    sylv::set_last_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return SYLV_ECUDA;
  }
  const void* ptrs[5] = {row_ptr, X, Y, nnz > 0 ? col_idx : nullptr, nnz > 0 ? val : nullptr};
  for (const void* p : ptrs) {
    if (p == nullptr) continue;
    cudaPointerAttributes at{};
    e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
      cudaGetLastError();  // this call's own error: cleared
      sylv::set_last_error(std::string("sylv_spmm_noalloc: cudaPointerGetAttributes: ") + cudaGetErrorString(e));
      return SYLV_EINVAL;
    }
    const bool on_device = at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
    if (!on_device || (at.type == cudaMemoryTypeDevice && at.device != dev)) {
      sylv::set_last_error("sylv_spmm_noalloc: every pointer must be device memory of the current device");
      return SYLV_EINVAL;
    }
  }
  return SYLV_OK;
}

}  // namespace

extern "C" int sylv_spmm_noalloc(int64_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx,
                                 const double* val, const double* X, double* Y, int64_t k, void* cuda_stream) {
  if (n < 1 || nnz < 0 || k < 1 || k > 8 || !row_ptr || !X || !Y || (nnz > 0 && (!col_idx || !val))) {
    sylv::set_last_error("sylv_spmm_noalloc: bad arguments (need n >= 1, 1 <= k <= 8, non-NULL device pointers)");
    return SYLV_EINVAL;
  }
  if (n > INT32_MAX - 1 || nnz > INT32_MAX) {
    sylv::set_last_error("sylv_spmm_noalloc: sizes exceed int32 indexing");
    return SYLV_EINVAL;
  }
  if (n * k > (int64_t)SYLV_NOALLOC_MAX_ELEMS) {
    sylv::set_last_error("sylv_spmm_noalloc: n * k = " + std::to_string(n * k) + " exceeds the fixed staging size " +
                    std::to_string((int64_t)SYLV_NOALLOC_MAX_ELEMS) + "; use sylv_apply");
    return SYLV_EINVAL;
  }
  // An error left pending by the caller's earlier CUDA work is reported, not cleared: after the
  // launches below, cudaGetLastError then returns this call's own launch errors only.
  cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) {
    sylv::set_last_error(std::string("sylv_spmm_noalloc: an earlier CUDA error is pending (left set): ") +
                         cudaGetErrorString(e));
    return SYLV_ECUDA;
  }
  int rc = check_device_pointers(row_ptr, col_idx, val, X, Y, nnz);
  if (rc != SYLV_OK) return rc;
  double* scratch = nullptr;
  rc = scratch_address(&scratch);
  if (rc != SYLV_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  double* xb = scratch;
  double* yb = scratch + SYLV_NOALLOC_MAX_ELEMS;
  sylv::launch_pack<double>(st, n, (int)k, X, xb);
  sylv::launch_spmm<double>(st, nullptr, n, (int)k, row_ptr, col_idx, val, xb, yb, nullptr, nullptr, 0);
  sylv::launch_unpack<double>(st, n, (int)k, 1, yb, n * k, Y);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    sylv::set_last_error(std::string("sylv_spmm_noalloc launch: ") + cudaGetErrorString(e));
    return SYLV_ECUDA;
  }
  return SYLV_OK;
}

// taser_run_host_static: taser_run_host with its workspace in a file-scope device array,
// for callers that cannot allocate device memory (see include/taser.h).
#include <cstdio>
#include <mutex>

#include "common.cuh"

namespace taser {
taser_status report(taser_status st, const char* msg);
}  // namespace taser

namespace {

// The scratch of every call on a device.  The CUDA runtime maps it when the library's
// module is loaded on that device; the library itself never allocates.
__device__ __align__(256) unsigned char g_static_scratch[TASER_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {};  // device address of g_static_scratch, per device
std::mutex g_scratch_mutex;

}  // namespace

extern "C" {

taser_status taser_run_host_static(int kind, int64_t batch, int B, int U_or_K, const void* H_or_Y, const void* y,
                                   float alpha, int t_max, int precision, int lnn_mode, int8_t* s_hat,
                                   uint32_t* flags, void* stream) {
  // Invalid shapes and empty batches: taser_run_host validates and reports them before
  // it touches any workspace.
  const size_t need = taser_host_workspace_bytes(kind, batch, B, U_or_K);
  if (batch <= 0 || need == 0) {
    return taser_run_host(kind, batch, B, U_or_K, H_or_Y, y, alpha, t_max, precision, lnn_mode, nullptr, 0, s_hat,
                          flags, stream);
  }
  if (need > TASER_STATIC_SCRATCH_BYTES) {
    char msg[256];
    snprintf(msg, sizeof(msg),
             "batch of %lld instances needs %zu bytes of scratch, the static scratch holds %zu bytes "
             "(about %lld instances of this shape): split the batch",
             (long long)batch, need, (size_t)TASER_STATIC_SCRATCH_BYTES,
             (long long)((double)TASER_STATIC_SCRATCH_BYTES / ((double)need / (double)batch)));
    return taser::report(TASER_ERR_INVALID_ARG, msg);
  }
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return taser::report(TASER_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return taser::report(TASER_ERR_UNSUPPORTED, "device ordinal beyond 63");
  void* ptr = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (g_scratch_ptr[dev] == nullptr) {
      // One-time set-up on this device (the current one): the array's device address.
      // In host code the name g_static_scratch is only a host-side stand-in.
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_static_scratch);
      if (e != cudaSuccess) return taser::report(TASER_ERR_CUDA, cudaGetErrorString(e));
      g_scratch_ptr[dev] = p;
    }
    ptr = g_scratch_ptr[dev];
  }
  return taser_run_host(kind, batch, B, U_or_K, H_or_Y, y, alpha, t_max, precision, lnn_mode, ptr,
                        TASER_STATIC_SCRATCH_BYTES, s_hat, flags, stream);
}

}  // extern "C"

// Per-stage decryption that allocates no device memory at all: its
// intermediates live in one fixed array compiled into the library.
//
// Who needs this: callers that cannot call cudaMalloc (or ask any
// allocator for memory) at decryption time -- for instance code embedded in
// a framework that owns every byte of device memory through its own
// allocator, latency-critical paths where an allocation could block on the
// device or fail under memory pressure, and services that must reserve all
// of their device memory when they load.  They still pass u, v, the keys
// and m_out; only the scratch (the w words and the RM-decoded bytes between
// the three stage kernels) comes from here.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "../../include/hqc_gb300.h"
#include "hqc_internal.h"
#include "hqc_params.cuh"

// Compiled-in scratch.  Every GPU that loads the library holds these bytes
// until the process exits, and every call on a device shares them.
static __device__ __align__(256) unsigned char g_noalloc_scratch[HQC_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_dev_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch on the current device.  In host code the
// array's name is only a host-side stand-in, so the address has to come
// from the runtime, once per device, with that device current.  The cache
// lives as long as the process: after cudaDeviceReset (which destroys the
// context that held the array) the cached address is stale.  Unsafe to call
// after cudaDeviceReset in the same process.
cudaError_t scratch_on_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_dev_ptr[dev] = p;
  }
  *out = g_dev_ptr[dev];
  return cudaSuccess;
}

// Largest count whose per-stage workspace (the same formula the
// allocating entry point checks against) fits the compiled-in array: the
// closed-form estimate, stepped down until hqc_staged_workspace_bytes
// agrees, so the limit follows any change to the workspace layout.
int64_t noalloc_max_count(int level) {
  hqc_params_t p;
  if (hqc_get_params(level, &p) != HQC_OK) return 0;
  const size_t per_ct = (size_t)p.W_v * 8 + (size_t)p.n1;
  int64_t c = (int64_t)(HQC_NOALLOC_SCRATCH_BYTES / per_ct) + 1;
  while (c > 0 && hqc_staged_workspace_bytes(level, c) > (size_t)HQC_NOALLOC_SCRATCH_BYTES) c--;
  return c;
}

// Record the message for hqc_last_error() and return the code.
int nfail(int code, const char* fmt, ...) {
  char buf[400];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  hqc::set_last_error(buf);
  return code;
}

}  // namespace

extern "C" int hqc_decrypt_batch_staged_noalloc(int level, int64_t count, const uint64_t* u, const uint64_t* v,
                                                const uint32_t* y, const hqc_keyset_t* keys, const int32_t* key_idx,
                                                uint8_t* m_out, void* stream) {
  hqc_params_t p;
  if (hqc_get_params(level, &p) != HQC_OK) return nfail(HQC_EINVAL, "level must be 1, 3 or 5 (got %d)", level);
  if (count < 0) return nfail(HQC_EINVAL, "count must be >= 0");
  if (count == 0) return HQC_OK;
  const int64_t max_count = noalloc_max_count(level);
  if (count > max_count)
    return nfail(HQC_EINVAL,
                 "count %lld exceeds the static scratch: %d bytes hold at most %lld HQC-%d ciphertexts per call",
                 (long long)count, (int)HQC_NOALLOC_SCRATCH_BYTES, (long long)max_count, level);
  void* scratch = nullptr;
  cudaError_t e = scratch_on_current_device(&scratch);
  if (e != cudaSuccess) return nfail(HQC_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
  // The existing per-stage entry point does every argument check and the
  // three launches; it is handed the static scratch as its workspace.
  const size_t ws = (size_t)HQC_NOALLOC_SCRATCH_BYTES;
  return hqc_decrypt_batch_staged(level, count, u, v, y, keys, key_idx, scratch, ws, m_out, stream);
}

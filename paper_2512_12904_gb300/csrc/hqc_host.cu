// Decryption from host buffers with copies overlapped with compute.
//
// The batch is cut into chunks; chunk i goes to one of two device slots in
// the caller's workspace.  A copy stream uploads chunk i + 1 while the
// compute stream runs the fused kernel on chunk i and copies its messages
// back, so the upload of a batch and its decryption run at the same time.
// The two internal streams are created once per device; the call is ordered
// after earlier work on the caller's stream, and the caller's stream waits
// for the last chunk.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "../../include/hqc_gb300.h"
#include "hqc_internal.h"
#include "hqc_params.cuh"

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
cudaStream_t g_copy[kMaxDevices] = {nullptr}, g_comp[kMaxDevices] = {nullptr};

int hfail(int code, const char* fmt, ...) {
  char buf[400];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  hqc::set_last_error(buf);
  return code;
}

struct SlotLayout {
  size_t u, v, k, m, total;
};

SlotLayout layout(const hqc_params_t& p, int64_t chunk) {
  SlotLayout l;
  l.u = (size_t)chunk * p.W_u_pitch * 8;
  l.v = (size_t)chunk * p.W_v * 8;
  l.k = ((size_t)chunk * 4 + 15) / 16 * 16;
  l.m = ((size_t)chunk * p.k + 15) / 16 * 16;
  l.total = l.u + l.v + l.k + l.m;
  return l;
}

}  // namespace

extern "C" size_t hqc_host_workspace_bytes(int level, int64_t chunk) {
  hqc_params_t p;
  if (hqc_get_params(level, &p) != HQC_OK || chunk <= 0) return 0;
  return 2 * layout(p, chunk).total;
}

extern "C" int hqc_decrypt_host_keyed(int level, int64_t count, const uint64_t* u_host, const uint64_t* v_host,
                                      const hqc_keyset_t* keys, const int32_t* key_idx_host, uint8_t* m_host,
                                      int64_t chunk, void* workspace, size_t workspace_bytes, void* stream) {
  hqc_params_t p;
  if (hqc_get_params(level, &p) != HQC_OK) return hfail(HQC_EINVAL, "level must be 1, 3 or 5");
  if (count < 0) return hfail(HQC_EINVAL, "count must be >= 0");
  if (count == 0) return HQC_OK;
  if (!u_host || !v_host || !keys || !key_idx_host || !m_host || !workspace)
    return hfail(HQC_EINVAL, "NULL argument");
  if (keys->level != level) return hfail(HQC_EINVAL, "keys registered for another level");
  if ((uintptr_t)workspace % 16) return hfail(HQC_EINVAL, "workspace must be 16-byte aligned");
  cudaError_t e = cudaSuccess;
  if (chunk <= 0) {
    // whole waves of the persistent grid, about eight chunks per batch, as
    // many as the workspace holds
    int64_t wave = 0;
    if ((e = hqc::fused_wave(level, true, hqc::level_cfg(level), &wave)) != cudaSuccess || wave <= 0)
      return hfail(HQC_ECUDA, "launch shape query: %s", cudaGetErrorString(e));
    const int64_t waves = (count + 8 * wave - 1) / (8 * wave);
    chunk = waves * wave;
    while (chunk > wave && 2 * layout(p, chunk).total > workspace_bytes) chunk -= wave;
    while (chunk > 1 && 2 * layout(p, chunk).total > workspace_bytes) chunk /= 2;
  }
  const SlotLayout L = layout(p, chunk);
  if (workspace_bytes < 2 * L.total)
    return hfail(HQC_ENOMEM, "workspace has %zu bytes, needs %zu", workspace_bytes, 2 * L.total);
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev >= kMaxDevices) return hfail(HQC_ECUDA, "cudaGetDevice");
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_copy[dev]) {
      if ((e = cudaStreamCreateWithFlags(&g_copy[dev], cudaStreamNonBlocking)) != cudaSuccess ||
          (e = cudaStreamCreateWithFlags(&g_comp[dev], cudaStreamNonBlocking)) != cudaSuccess)
        return hfail(HQC_ECUDA, "stream creation: %s", cudaGetErrorString(e));
    }
  }
  cudaStream_t cs = g_copy[dev], ks = g_comp[dev], us = (cudaStream_t)stream;
  cudaEvent_t start, copied[2], done[2];
  cudaEventCreateWithFlags(&start, cudaEventDisableTiming);
  for (int s = 0; s < 2; s++) {
    cudaEventCreateWithFlags(&copied[s], cudaEventDisableTiming);
    cudaEventCreateWithFlags(&done[s], cudaEventDisableTiming);
  }
  auto finish = [&](int rc) {
    cudaEventDestroy(start);
    for (int s = 0; s < 2; s++) {
      cudaEventDestroy(copied[s]);
      cudaEventDestroy(done[s]);
    }
    return rc;
  };
  // order after the caller's earlier work
  e = cudaEventRecord(start, us);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, start, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ks, start, 0);
  char* base = static_cast<char*>(workspace);
  const int64_t nchunks = (count + chunk - 1) / chunk;
  for (int64_t c = 0; c < nchunks && e == cudaSuccess; c++) {
    const int s = (int)(c & 1);
    const int64_t first = c * chunk, n = (count - first) < chunk ? (count - first) : chunk;
    uint64_t* du = reinterpret_cast<uint64_t*>(base + s * L.total);
    uint64_t* dv = reinterpret_cast<uint64_t*>(base + s * L.total + L.u);
    int32_t* dk = reinterpret_cast<int32_t*>(base + s * L.total + L.u + L.v);
    uint8_t* dm = reinterpret_cast<uint8_t*>(base + s * L.total + L.u + L.v + L.k);
    // the slot is free once the chunk that last used it was decrypted and copied out
    if (c >= 2) e = cudaStreamWaitEvent(cs, done[s], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(du, u_host + first * p.W_u_pitch, (size_t)n * p.W_u_pitch * 8, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dv, v_host + first * p.W_v, (size_t)n * p.W_v * 8, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dk, key_idx_host + first, (size_t)n * 4, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaEventRecord(copied[s], cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ks, copied[s], 0);
    if (e == cudaSuccess) {
      hqc::DecArgs a;
      a.count = n;
      a.u = du;
      a.v = dv;
      a.y = keys->d_table;
      a.key_idx = dk;
      a.nkeys = keys->nkeys;
      a.m = dm;
      e = hqc::launch_fused(level, true, a, ks, hqc::level_cfg(level));
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(m_host + first * p.k, dm, (size_t)n * p.k, cudaMemcpyDeviceToHost, ks);
    if (e == cudaSuccess) e = cudaEventRecord(done[s], ks);
  }
  // the caller's stream continues after the last chunk
  if (e == cudaSuccess) e = cudaStreamWaitEvent(us, done[(nchunks - 1) & 1], 0);
  if (e == cudaSuccess && nchunks > 1) e = cudaStreamWaitEvent(us, done[(nchunks - 2) & 1], 0);
  if (e != cudaSuccess) return finish(hfail(HQC_ECUDA, "pipelined decrypt: %s", cudaGetErrorString(e)));
  return finish(HQC_OK);
}

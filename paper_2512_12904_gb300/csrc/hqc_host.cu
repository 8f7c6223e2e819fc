// Decryption and decapsulation from host buffers with copies overlapped
// with compute.
//
// The batch is cut into chunks; chunk i goes to one of two device slots in
// the caller's workspace.  A copy stream uploads chunk i + 1 while the
// compute stream runs the kernels on chunk i and copies its results back,
// so the upload of a batch and its processing run at the same time.  The
// two internal streams are created once per device; the call is ordered
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

size_t r16(size_t b) { return (b + 15) / 16 * 16; }

// Device slot of one chunk: inputs, outputs and (for decapsulation) the
// KEM workspace of a chunk.
struct SlotLayout {
  size_t u, v, k, salt, out, ok, kem, total;
};

SlotLayout layout(const hqc_params_t& p, int64_t chunk, bool kem) {
  SlotLayout l;
  l.u = r16((size_t)chunk * p.W_u_pitch * 8);
  l.v = r16((size_t)chunk * p.W_v * 8);
  l.k = r16((size_t)chunk * 4);
  l.salt = kem ? r16((size_t)chunk * 16) : 0;
  l.out = kem ? r16((size_t)chunk * 32) : r16((size_t)chunk * p.k);
  l.ok = kem ? r16((size_t)chunk * 4) : 0;
  l.kem = kem ? hqc_kem_workspace_bytes(p.level, chunk) : 0;
  l.total = l.u + l.v + l.k + l.salt + l.out + l.ok + l.kem;
  return l;
}

struct Slot {
  uint64_t *u, *v;
  int32_t* k;
  uint8_t *salt, *out;
  uint32_t* ok;
  void* kem;
};

Slot slot_at(void* base, const SlotLayout& L, int s) {
  char* b = static_cast<char*>(base) + (size_t)s * L.total;
  Slot x;
  x.u = reinterpret_cast<uint64_t*>(b);
  b += L.u;
  x.v = reinterpret_cast<uint64_t*>(b);
  b += L.v;
  x.k = reinterpret_cast<int32_t*>(b);
  b += L.k;
  x.salt = reinterpret_cast<uint8_t*>(b);
  b += L.salt;
  x.out = reinterpret_cast<uint8_t*>(b);
  b += L.out;
  x.ok = reinterpret_cast<uint32_t*>(b);
  b += L.ok;
  x.kem = b;
  return x;
}

// Chunk size: `chunk` if positive, else whole waves of the persistent
// decryption grid, as large as the workspace holds: about eight chunks per
// batch for decryption, two for decapsulation (its one-thread-per-item
// SHAKE kernels need tens of thousands of items to fill the GPU).
int pick_chunk(const hqc_params_t& p, int64_t count, int64_t chunk, size_t workspace_bytes, bool kem,
               int64_t* out) {
  if (chunk <= 0) {
    int64_t wave = 0;
    cudaError_t e = hqc::fused_wave(p.level, true, hqc::level_cfg(p.level), &wave);
    if (e != cudaSuccess || wave <= 0) return hfail(HQC_ECUDA, "launch shape query: %s", cudaGetErrorString(e));
    const int64_t parts = kem ? 2 : 8;
    const int64_t waves = (count + parts * wave - 1) / (parts * wave);
    chunk = waves * wave;
    while (chunk > wave && 2 * layout(p, chunk, kem).total > workspace_bytes) chunk -= wave;
    while (chunk > 1 && 2 * layout(p, chunk, kem).total > workspace_bytes) chunk /= 2;
  }
  if (2 * layout(p, chunk, kem).total > workspace_bytes)
    return hfail(HQC_ENOMEM, "workspace has %zu bytes, needs %zu", workspace_bytes, 2 * layout(p, chunk, kem).total);
  *out = chunk;
  return HQC_OK;
}

// The double-buffered pipeline.  upload(first, n, slot, copy_stream),
// compute(first, n, slot, compute_stream) and download(first, n, slot,
// compute_stream) enqueue one chunk's work and return a CUDA status.
template <class Up, class Comp, class Down>
int run_pipeline(int64_t count, int64_t chunk, void* workspace, const SlotLayout& L, void* stream, Up upload,
                 Comp compute, Down download) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
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
  // order after the caller's earlier work
  e = cudaEventRecord(start, us);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, start, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ks, start, 0);
  const int64_t nchunks = (count + chunk - 1) / chunk;
  for (int64_t c = 0; c < nchunks && e == cudaSuccess; c++) {
    const int s = (int)(c & 1);
    const int64_t first = c * chunk, n = (count - first) < chunk ? (count - first) : chunk;
    const Slot slot = slot_at(workspace, L, s);
    // the slot is free once the chunk that last used it was processed and copied out
    if (c >= 2) e = cudaStreamWaitEvent(cs, done[s], 0);
    if (e == cudaSuccess) e = upload(first, n, slot, cs);
    if (e == cudaSuccess) e = cudaEventRecord(copied[s], cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ks, copied[s], 0);
    if (e == cudaSuccess) e = compute(first, n, slot, ks);
    if (e == cudaSuccess) e = download(first, n, slot, ks);
    if (e == cudaSuccess) e = cudaEventRecord(done[s], ks);
  }
  // the caller's stream continues after the last chunk
  if (e == cudaSuccess) e = cudaStreamWaitEvent(us, done[(nchunks - 1) & 1], 0);
  if (e == cudaSuccess && nchunks > 1) e = cudaStreamWaitEvent(us, done[(nchunks - 2) & 1], 0);
  cudaEventDestroy(start);
  for (int s = 0; s < 2; s++) {
    cudaEventDestroy(copied[s]);
    cudaEventDestroy(done[s]);
  }
  if (e != cudaSuccess) return hfail(HQC_ECUDA, "pipelined batch: %s", cudaGetErrorString(e));
  return HQC_OK;
}

cudaError_t h2d(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
}

}  // namespace

extern "C" size_t hqc_host_workspace_bytes(int level, int64_t chunk) {
  hqc_params_t p;
  if (hqc_get_params(level, &p) != HQC_OK || chunk <= 0) return 0;
  return 2 * layout(p, chunk, false).total;
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
  int rc = pick_chunk(p, count, chunk, workspace_bytes, false, &chunk);
  if (rc != HQC_OK) return rc;
  const SlotLayout L = layout(p, chunk, false);
  const hqc::LaunchCfg cfg = hqc::level_cfg(level);
  auto up = [&](int64_t first, int64_t n, const Slot& s, cudaStream_t st) {
    cudaError_t e = h2d(s.u, u_host + first * p.W_u_pitch, (size_t)n * p.W_u_pitch * 8, st);
    if (e == cudaSuccess) e = h2d(s.v, v_host + first * p.W_v, (size_t)n * p.W_v * 8, st);
    if (e == cudaSuccess) e = h2d(s.k, key_idx_host + first, (size_t)n * 4, st);
    return e;
  };
  auto comp = [&](int64_t, int64_t n, const Slot& s, cudaStream_t st) {
    hqc::DecArgs a;
    a.count = n;
    a.u = s.u;
    a.v = s.v;
    a.y = keys->d_table;
    a.key_idx = s.k;
    a.nkeys = keys->nkeys;
    a.m = s.out;
    return hqc::launch_fused(level, true, a, st, cfg);
  };
  auto down = [&](int64_t first, int64_t n, const Slot& s, cudaStream_t st) {
    return cudaMemcpyAsync(m_host + first * p.k, s.out, (size_t)n * p.k, cudaMemcpyDeviceToHost, st);
  };
  return run_pipeline(count, chunk, workspace, L, stream, up, comp, down);
}

extern "C" size_t hqc_kem_host_workspace_bytes(int level, int64_t chunk) {
  hqc_params_t p;
  if (hqc_get_params(level, &p) != HQC_OK || chunk <= 0) return 0;
  return 2 * layout(p, chunk, true).total;
}

extern "C" int hqc_kem_decaps_host(int level, int64_t count, const hqc_keyset_t* keys, const uint64_t* h,
                                   const uint64_t* s, const uint8_t* sigma, const int32_t* key_idx_host,
                                   const uint64_t* u_host, const uint64_t* v_host, const uint8_t* salt_host,
                                   uint8_t* K_host, uint32_t* ok_host, int64_t chunk, void* workspace,
                                   size_t workspace_bytes, void* stream) {
  hqc_params_t p;
  if (hqc_get_params(level, &p) != HQC_OK) return hfail(HQC_EINVAL, "level must be 1, 3 or 5");
  if (count < 0) return hfail(HQC_EINVAL, "count must be >= 0");
  if (count == 0) return HQC_OK;
  if (!keys || !h || !s || !sigma || !key_idx_host || !u_host || !v_host || !salt_host || !K_host || !workspace)
    return hfail(HQC_EINVAL, "NULL argument");
  if (keys->level != level) return hfail(HQC_EINVAL, "keys registered for another level");
  if ((uintptr_t)workspace % 16) return hfail(HQC_EINVAL, "workspace must be 16-byte aligned");
  const int rc0 = pick_chunk(p, count, chunk, workspace_bytes, true, &chunk);
  if (rc0 != HQC_OK) return rc0;
  const SlotLayout L = layout(p, chunk, true);
  auto up = [&](int64_t first, int64_t n, const Slot& sl, cudaStream_t st) {
    cudaError_t e = h2d(sl.u, u_host + first * p.W_u_pitch, (size_t)n * p.W_u_pitch * 8, st);
    if (e == cudaSuccess) e = h2d(sl.v, v_host + first * p.W_v, (size_t)n * p.W_v * 8, st);
    if (e == cudaSuccess) e = h2d(sl.k, key_idx_host + first, (size_t)n * 4, st);
    if (e == cudaSuccess) e = h2d(sl.salt, salt_host + first * 16, (size_t)n * 16, st);
    return e;
  };
  int rc_kem = HQC_OK;
  char kem_err[400] = "";
  auto comp = [&](int64_t, int64_t n, const Slot& sl, cudaStream_t st) {
    rc_kem = hqc_kem_decaps(level, n, keys, h, s, sigma, sl.k, sl.u, sl.v, sl.salt, sl.out, sl.ok, sl.kem, L.kem,
                            st);
    if (rc_kem != HQC_OK) snprintf(kem_err, sizeof kem_err, "%s", hqc_last_error());
    return rc_kem == HQC_OK ? cudaSuccess : cudaErrorLaunchFailure;
  };
  auto down = [&](int64_t first, int64_t n, const Slot& sl, cudaStream_t st) {
    cudaError_t e = cudaMemcpyAsync(K_host + first * 32, sl.out, (size_t)n * 32, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && ok_host)
      e = cudaMemcpyAsync(ok_host + first, sl.ok, (size_t)n * 4, cudaMemcpyDeviceToHost, st);
    return e;
  };
  const int rc = run_pipeline(count, chunk, workspace, L, stream, up, comp, down);
  if (rc_kem != HQC_OK) {
    hqc::set_last_error(kem_err);
    return rc_kem;
  }
  return rc;
}

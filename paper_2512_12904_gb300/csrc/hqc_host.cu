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
#include <cstdint>
#include <mutex>
#include <vector>

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
// Chunk schedule: `sizes` (each at most the slot's capacity) covering the
// batch in order.
std::vector<int64_t> uniform_chunks(int64_t count, int64_t chunk) {
  std::vector<int64_t> v;
  for (int64_t f = 0; f < count; f += chunk) v.push_back(count - f < chunk ? count - f : chunk);
  return v;
}

// Full chunks, then the remainder split so that the last chunk is about a
// quarter chunk: the pipeline's tail (the last chunk's kernels and copy
// back, which nothing overlaps) stays short.
std::vector<int64_t> tapered_chunks(int64_t count, int64_t chunk) {
  std::vector<int64_t> v;
  const int64_t q = chunk / 4 > 0 ? chunk / 4 : 1;
  int64_t left = count;
  while (left > chunk + q) {
    v.push_back(chunk);
    left -= chunk;
  }
  if (left > q) {
    v.push_back(left - q);
    v.push_back(q);
  } else if (left > 0) {
    v.push_back(left);
  }
  return v;
}

template <class Up, class Comp, class Down>
int run_pipeline(const std::vector<int64_t>& sizes, void* workspace, const SlotLayout& L, void* stream, Up upload,
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
  const int64_t nchunks = (int64_t)sizes.size();
  int64_t first = 0;
  for (int64_t c = 0; c < nchunks && e == cudaSuccess; first += sizes[(size_t)c], c++) {
    const int s = (int)(c & 1);
    const int64_t n = sizes[(size_t)c];
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
  const bool tapered = chunk <= 0;
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
    // the m rows come back from this slot: the ones the kernel skips (key
    // index outside [0, nkeys)) come back as zeros, not as an older chunk's
    cudaError_t e = cudaMemsetAsync(s.out, 0, (size_t)n * p.k, st);
    if (e != cudaSuccess) return e;
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
  return run_pipeline(tapered ? tapered_chunks(count, chunk) : uniform_chunks(count, chunk), workspace, L, stream, up,
                      comp, down);
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
    // K and ok come back from this slot: items skipped for a bad key index
    // come back as zero K rows with ok = 0
    cudaError_t e = cudaMemsetAsync(sl.out, 0, (size_t)n * 32, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sl.ok, 0, (size_t)n * 4, st);
    if (e != cudaSuccess) return e;
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
  const int rc = run_pipeline(uniform_chunks(count, chunk), workspace, L, stream, up, comp, down);
  if (rc_kem != HQC_OK) {
    hqc::set_last_error(kem_err);
    return rc_kem;
  }
  return rc;
}

// ---------------------------------------------------------------------------
// Mixed-level batches from host buffers.  Each chunk's item records and the
// arena range its rows span go up on the copy stream; on the compute stream
// a one-block kernel groups the chunk's records by level, then one
// persistent kernel per level decrypts its items, and the chunk's m range
// comes back.  The device slot holds the arena range at the same offsets as
// the host arena minus the chunk's first row, so the records need no
// rewriting: the kernels get an arena pointer moved back by that amount.
// ---------------------------------------------------------------------------
namespace {

constexpr int kGroupThreads = 1024;

__global__ void __launch_bounds__(kGroupThreads) k_group_items(const hqc::MixedItem* __restrict__ in, int64_t n,
                                                              int64_t s0, int64_t s1, int64_t s2,
                                                              hqc::MixedItem* __restrict__ out) {
  __shared__ unsigned int cnt[3];
  if (threadIdx.x < 3) cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t start[3] = {s0, s1, s2};
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const hqc::MixedItem it = in[i];
    const int li = it.level == 1 ? 0 : it.level == 3 ? 1 : it.level == 5 ? 2 : -1;
    if (li < 0) continue;
    const unsigned int pos = atomicAdd(&cnt[li], 1u);
    out[start[li] + pos] = it;
  }
}

struct MixedChunk {
  int64_t first, n, base, words, mbase, mbytes, cnt[3];
};

// Scan the items once: order checks, per-chunk ranges and level counts.
int mixed_chunks(int64_t count, const hqc_item_t* items, int64_t arena_words, int64_t m_bytes, int64_t chunk,
                 std::vector<MixedChunk>* out) {
  hqc_params_t prm[3];
  for (int li = 0; li < 3; li++) hqc_get_params(li == 0 ? 1 : li == 1 ? 3 : 5, &prm[li]);
  out->clear();
  for (int64_t first = 0; first < count; first += chunk) {
    MixedChunk c{};
    c.first = first;
    c.n = count - first < chunk ? count - first : chunk;
    c.base = items[first].u_off & ~(int64_t)1;
    c.mbase = items[first].m_off;
    int64_t end = c.base, mend = c.mbase;
    for (int64_t i = first; i < first + c.n; i++) {
      const hqc_item_t& it = items[i];
      if (i > 0 && (it.u_off < items[i - 1].u_off || it.m_off < items[i - 1].m_off))
        return hfail(HQC_EINVAL, "item %lld: items must be in arena order (u_off and m_off non-decreasing)",
                     (long long)i);
      const int li = hqc::level_index(it.level);
      if (li < 0) continue;  // skipped by the kernels, as in hqc_decrypt_mixed
      if (it.u_off < c.base || it.v_off < c.base || it.m_off < c.mbase)
        return hfail(HQC_EINVAL, "item %lld: rows before the item's own chunk", (long long)i);
      c.cnt[li]++;
      const int64_t e1 = it.u_off + prm[li].W_u_pitch, e2 = it.v_off + prm[li].W_v, e3 = it.m_off + prm[li].k;
      end = e1 > end ? e1 : end;
      end = e2 > end ? e2 : end;
      mend = e3 > mend ? e3 : mend;
    }
    if (end > arena_words || mend > m_bytes) return hfail(HQC_EINVAL, "items reach past the arena or m");
    c.words = end - c.base;
    c.mbytes = mend - c.mbase;
    out->push_back(c);
  }
  return HQC_OK;
}

struct MixedSlot {
  size_t words, items, grouped, m, total;
};

MixedSlot mixed_slot(int64_t chunk, int64_t max_words, int64_t max_m) {
  MixedSlot s;
  s.words = r16((size_t)max_words * 8);
  s.items = r16((size_t)chunk * sizeof(hqc::MixedItem));
  s.grouped = s.items;
  s.m = r16((size_t)max_m);
  s.total = s.words + s.items + s.grouped + s.m;
  return s;
}

int64_t default_mixed_chunk(int64_t count) {
  // about four chunks, each at least one HQC-1 wave of the persistent grid
  int64_t wave = 0;
  if (hqc::fused_wave(1, true, hqc::level_cfg(1), &wave) != cudaSuccess || wave <= 0) wave = 8192;
  int64_t c = (count + 3) / 4;
  return c < wave ? (count < wave ? count : wave) : c;
}

}  // namespace

extern "C" size_t hqc_mixed_host_workspace_bytes(int64_t count, const hqc_item_t* items_host, int64_t chunk) {
  if (count <= 0 || !items_host) return 0;
  if (chunk <= 0) chunk = default_mixed_chunk(count);
  std::vector<MixedChunk> cs;
  if (mixed_chunks(count, items_host, INT64_MAX / 4, INT64_MAX / 4, chunk, &cs) != HQC_OK) return 0;
  int64_t mw = 0, mm = 0;
  for (const auto& c : cs) {
    mw = c.words > mw ? c.words : mw;
    mm = c.mbytes > mm ? c.mbytes : mm;
  }
  return 2 * mixed_slot(chunk, mw, mm).total;
}

extern "C" int hqc_decrypt_mixed_host(int64_t count, const hqc_item_t* items_host, const uint64_t* arena_host,
                                      int64_t arena_words, const hqc_keyset_t* const keys[3], uint8_t* m_host,
                                      int64_t m_bytes, int64_t chunk, void* workspace, size_t workspace_bytes,
                                      void* stream) {
  if (count < 0) return hfail(HQC_EINVAL, "count must be >= 0");
  if (count == 0) return HQC_OK;
  if (!items_host || !arena_host || !keys || !m_host || !workspace) return hfail(HQC_EINVAL, "NULL argument");
  if ((uintptr_t)workspace % 16) return hfail(HQC_EINVAL, "workspace must be 16-byte aligned");
  for (int li = 0; li < 3; li++)
    if (keys[li] && keys[li]->level != (li == 0 ? 1 : li == 1 ? 3 : 5))
      return hfail(HQC_EINVAL, "keys[%d] registered for another level", li);
  if (chunk <= 0) chunk = default_mixed_chunk(count);
  std::vector<MixedChunk> cs;
  int rc = mixed_chunks(count, items_host, arena_words, m_bytes, chunk, &cs);
  if (rc != HQC_OK) return rc;
  int64_t mw = 0, mm = 0;
  for (const auto& c : cs) {
    mw = c.words > mw ? c.words : mw;
    mm = c.mbytes > mm ? c.mbytes : mm;
  }
  const MixedSlot M = mixed_slot(chunk, mw, mm);
  if (2 * M.total > workspace_bytes)
    return hfail(HQC_ENOMEM, "workspace has %zu bytes, needs %zu", workspace_bytes, 2 * M.total);
  // the generic driver's slot layout carries only sizes here
  SlotLayout L{};
  L.total = M.total;
  auto parts = [&](const Slot& s, uint64_t** w, hqc::MixedItem** raw, hqc::MixedItem** grouped, uint8_t** m) {
    char* b = reinterpret_cast<char*>(s.u);  // slot base
    *w = reinterpret_cast<uint64_t*>(b);
    *raw = reinterpret_cast<hqc::MixedItem*>(b + M.words);
    *grouped = reinterpret_cast<hqc::MixedItem*>(b + M.words + M.items);
    *m = reinterpret_cast<uint8_t*>(b + M.words + M.items + M.grouped);
  };
  auto chunk_of = [&](int64_t first) -> const MixedChunk& { return cs[(size_t)(first / chunk)]; };
  auto up = [&](int64_t first, int64_t, const Slot& s, cudaStream_t st) {
    const MixedChunk& c = chunk_of(first);
    uint64_t* w;
    hqc::MixedItem *raw, *grouped;
    uint8_t* m;
    parts(s, &w, &raw, &grouped, &m);
    cudaError_t e = h2d(w, arena_host + c.base, (size_t)c.words * 8, st);
    if (e == cudaSuccess) e = h2d(raw, items_host + c.first, (size_t)c.n * sizeof(hqc::MixedItem), st);
    return e;
  };
  auto comp = [&](int64_t first, int64_t, const Slot& s, cudaStream_t st) {
    const MixedChunk& c = chunk_of(first);
    uint64_t* w;
    hqc::MixedItem *raw, *grouped;
    uint8_t* m;
    parts(s, &w, &raw, &grouped, &m);
    const int64_t s1 = c.cnt[0], s2 = c.cnt[0] + c.cnt[1];
    // m bytes no valid item writes come back as zero
    cudaError_t e = cudaMemsetAsync(m, 0, (size_t)c.mbytes, st);
    if (e != cudaSuccess) return e;
    k_group_items<<<1, kGroupThreads, 0, st>>>(raw, c.n, 0, s1, s2, grouped);
    e = cudaGetLastError();
    const int64_t start[3] = {0, s1, s2};
    for (int li = 0; li < 3 && e == cudaSuccess; li++) {
      if (c.cnt[li] == 0 || !keys[li]) continue;
      hqc::MixedArgs a;
      a.count = c.cnt[li];
      a.items = grouped + start[li];
      a.arena = w - c.base;  // record offsets are absolute in the host arena
      a.arena_words = c.base + c.words;
      for (int k = 0; k < 3; k++) {
        a.keys[k] = keys[k] ? keys[k]->d_table : nullptr;
        a.nkeys[k] = keys[k] ? keys[k]->nkeys : 0;
      }
      a.m = m - c.mbase;
      a.m_bytes = c.mbase + c.mbytes;
      e = hqc::launch_items(li == 0 ? 1 : li == 1 ? 3 : 5, a, 0, st, hqc::LaunchCfg{});
    }
    return e;
  };
  auto down = [&](int64_t first, int64_t, const Slot& s, cudaStream_t st) {
    const MixedChunk& c = chunk_of(first);
    uint64_t* w;
    hqc::MixedItem *raw, *grouped;
    uint8_t* m;
    parts(s, &w, &raw, &grouped, &m);
    return cudaMemcpyAsync(m_host + c.mbase, m, (size_t)c.mbytes, cudaMemcpyDeviceToHost, st);
  };
  return run_pipeline(uniform_chunks(count, chunk), workspace, L, stream, up, comp, down);
}

// C ABI of the library (include/hqc_gb300.h): argument checks, keysets,
// launch configuration; every data-path step runs in the kernels of
// hqc_decrypt.cu / hqc_encrypt.cu.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/hqc_gb300.h"
#include "hqc_internal.h"
#include "hqc_params.cuh"

namespace {

thread_local std::string g_err;
hqc::LaunchCfg g_cfg[4];  // 0 mixed, 1..3 levels 1/3/5

int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(HQC_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

template <int L>
void fill(hqc_params_t* p) {
  using LV = hqc::Level<L>;
  p->level = L;
  p->n = LV::n;
  p->n1 = LV::n1;
  p->k = LV::k;
  p->delta = LV::delta;
  p->n2 = LV::n2;
  p->mult = LV::mult;
  p->w = LV::w;
  p->wr = LV::wr;
  p->we = LV::we;
  p->W_u = LV::W_u;
  p->W_u_pitch = LV::W_u_pitch;
  p->W_v = LV::W_v;
}

bool params_of(int level, hqc_params_t* p) {
  switch (level) {
    case 1: fill<1>(p); return true;
    case 3: fill<3>(p); return true;
    case 5: fill<5>(p); return true;
  }
  return false;
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

int check_common(int level, int64_t count, const uint64_t* u, const uint64_t* v, const uint8_t* m_out,
                 hqc_params_t* p) {
  g_err.clear();
  if (!params_of(level, p)) return fail(HQC_EINVAL, "level must be 1, 3 or 5 (got %d)", level);
  if (count < 0) return fail(HQC_EINVAL, "count must be >= 0");
  if (count > ((int64_t)1 << 40)) return fail(HQC_EINVAL, "count too large");
  if (count == 0) return HQC_OK;
  if (!u || !v || !m_out) return fail(HQC_EINVAL, "u, v and m_out must be non-NULL");
  if (!aligned(u, 16) || !aligned(v, 16)) return fail(HQC_EINVAL, "u and v must be 16-byte aligned");
  return HQC_OK;
}

int launch_result(cudaError_t e, const char* what) { return e == cudaSuccess ? HQC_OK : cuda_fail(e, what); }

// Adds to *out the number of key_idx entries outside [0, nkeys): one
// warp-wide sum per warp, one atomic per warp that found any.
constexpr int COUNT_THREADS = 256;
__global__ void __launch_bounds__(COUNT_THREADS) k_count_bad_key_idx(int64_t count, const int32_t* __restrict__ key_idx,
                                                                     int64_t nkeys, uint32_t* __restrict__ out) {
  uint32_t bad = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    bad += (uint32_t)__ldg(key_idx + i) >= (uint64_t)nkeys ? 1u : 0u;
  bad = __reduce_add_sync(0xFFFFFFFFu, bad);
  if ((threadIdx.x & 31) == 0 && bad) atomicAdd(out, bad);
}

}  // namespace

void hqc::set_last_error(const char* msg) { g_err = msg; }

namespace hqc {
LaunchCfg level_cfg(int level) { return level_index(level) < 0 ? LaunchCfg{} : g_cfg[level_index(level) + 1]; }
}  // namespace hqc

extern "C" {

int hqc_get_params(int level, hqc_params_t* out) {
  g_err.clear();
  if (!out) return fail(HQC_EINVAL, "out is NULL");
  if (!params_of(level, out)) return fail(HQC_EINVAL, "level must be 1, 3 or 5 (got %d)", level);
  return HQC_OK;
}

const char* hqc_last_error(void) { return g_err.c_str(); }

int hqc_decrypt_batch(int level, int64_t count, const uint64_t* u, const uint64_t* v, const uint32_t* y,
                      uint8_t* m_out, void* stream) {
  hqc_params_t p{};
  int rc = check_common(level, count, u, v, m_out, &p);
  if (rc != HQC_OK || count == 0) return rc;
  if (!y || !aligned(y, 4)) return fail(HQC_EINVAL, "y must be a non-NULL 4-byte aligned device pointer");
  hqc::DecArgs a;
  a.count = count;
  a.u = u;
  a.v = v;
  a.y = y;
  a.m = m_out;
  return launch_result(hqc::launch_fused(level, false, a, (cudaStream_t)stream, g_cfg[hqc::level_index(level) + 1]),
                       "fused decrypt launch");
}

int hqc_keys_register(int level, int64_t nkeys, const uint32_t* y_host, hqc_keyset_t** out) {
  g_err.clear();
  hqc_params_t p{};
  if (!out) return fail(HQC_EINVAL, "out is NULL");
  *out = nullptr;
  if (!params_of(level, &p)) return fail(HQC_EINVAL, "level must be 1, 3 or 5 (got %d)", level);
  if (nkeys <= 0 || nkeys > (1 << 30)) return fail(HQC_EINVAL, "nkeys must be in [1, 2^30]");
  if (!y_host) return fail(HQC_EINVAL, "y_host is NULL");
  for (int64_t i = 0; i < nkeys; i++) {
    const uint32_t* row = y_host + i * p.w;
    for (int a = 0; a < p.w; a++) {
      if (row[a] >= (uint32_t)p.n)
        return fail(HQC_EINVAL, "key %lld entry %d = %u is >= n = %d", (long long)i, a, row[a], p.n);
      for (int b = 0; b < a; b++)
        if (row[a] == row[b]) return fail(HQC_EINVAL, "key %lld repeats position %u", (long long)i, row[a]);
    }
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  const size_t bytes = (size_t)nkeys * p.w * sizeof(uint32_t);
  uint32_t* d = nullptr;
  e = cudaMalloc(&d, bytes);
  if (e != cudaSuccess) return fail(HQC_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  e = cudaMemcpy(d, y_host, bytes, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(d);
    return cuda_fail(e, "copying keys");
  }
  hqc_keyset_t* ks = new hqc_keyset_t{level, nkeys, dev, d};
  *out = ks;
  return HQC_OK;
}

int hqc_keys_free(hqc_keyset_t* keys) {
  g_err.clear();
  if (!keys) return HQC_OK;
  cudaError_t e = cudaFree(keys->d_table);
  delete keys;
  return e == cudaSuccess ? HQC_OK : cuda_fail(e, "cudaFree keys");
}

int hqc_keys_info(const hqc_keyset_t* keys, int* level, int64_t* nkeys, const uint32_t** device_table) {
  g_err.clear();
  if (!keys) return fail(HQC_EINVAL, "keys is NULL");
  if (level) *level = keys->level;
  if (nkeys) *nkeys = keys->nkeys;
  if (device_table) *device_table = keys->d_table;
  return HQC_OK;
}

int hqc_decrypt_batch_keyed(int level, int64_t count, const uint64_t* u, const uint64_t* v, const hqc_keyset_t* keys,
                            const int32_t* key_idx, uint8_t* m_out, void* stream) {
  hqc_params_t p{};
  int rc = check_common(level, count, u, v, m_out, &p);
  if (rc != HQC_OK || count == 0) return rc;
  if (!keys || keys->level != level) return fail(HQC_EINVAL, "keys missing or registered for another level");
  if (!key_idx || !aligned(key_idx, 4)) return fail(HQC_EINVAL, "key_idx must be a non-NULL aligned device pointer");
  hqc::DecArgs a;
  a.count = count;
  a.u = u;
  a.v = v;
  a.y = keys->d_table;
  a.key_idx = key_idx;
  a.nkeys = keys->nkeys;
  a.m = m_out;
  return launch_result(hqc::launch_fused(level, true, a, (cudaStream_t)stream, g_cfg[hqc::level_index(level) + 1]),
                       "fused keyed decrypt launch");
}

int hqc_count_bad_key_idx(int64_t count, const int32_t* key_idx, int64_t nkeys, uint32_t* out, void* stream) {
  g_err.clear();
  if (count < 0 || count > (int64_t)0xFFFFFFFFu) return fail(HQC_EINVAL, "count must be in [0, 2^32)");
  if (nkeys < 0) return fail(HQC_EINVAL, "nkeys must be >= 0");
  if (!out || !aligned(out, 4)) return fail(HQC_EINVAL, "out must be a non-NULL 4-byte aligned device pointer");
  if (count > 0 && (!key_idx || !aligned(key_idx, 4)))
    return fail(HQC_EINVAL, "key_idx must be a non-NULL 4-byte aligned device pointer");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return cuda_fail(e, "zeroing the count");
  if (count == 0) return HQC_OK;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (count + COUNT_THREADS - 1) / COUNT_THREADS;
  const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * 8;
  const unsigned grid = (unsigned)(want < cap ? want : cap);
  k_count_bad_key_idx<<<grid, COUNT_THREADS, 0, st>>>(count, key_idx, nkeys, out);
  return launch_result(cudaGetLastError(), "count launch");
}

int hqc_rm_decode_batch(int level, int64_t count, const uint64_t* w, uint8_t* r_out, int use_tensor_cores,
                        void* stream) {
  g_err.clear();
  hqc_params_t p{};
  if (!params_of(level, &p)) return fail(HQC_EINVAL, "level must be 1, 3 or 5");
  if (count < 0) return fail(HQC_EINVAL, "count must be >= 0");
  if (count == 0) return HQC_OK;
  if (!w || !aligned(w, 16)) return fail(HQC_EINVAL, "w must be a non-NULL 16-byte aligned device pointer");
  if (!r_out) return fail(HQC_EINVAL, "r_out must be a non-NULL device pointer");
  return launch_result(hqc::launch_rm_decode(level, count, w, r_out, use_tensor_cores != 0, (cudaStream_t)stream),
                       "RM decode launch");
}

int hqc_rm_tc_timeouts(int* out) {
  g_err.clear();
  if (!out) return fail(HQC_EINVAL, "out must be a non-NULL host pointer");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "synchronising the device");
  e = hqc::rm_tc_take_timeouts(out);
  if (e != cudaSuccess) return cuda_fail(e, "reading the timeout counter");
  return HQC_OK;
}

size_t hqc_staged_workspace_bytes(int level, int64_t count) {
  hqc_params_t p{};
  if (!params_of(level, &p) || count <= 0) return 0;
  const size_t w = (size_t)count * p.W_v * 8;
  const size_t r = ((size_t)count * p.n1 + 15) / 16 * 16;
  return w + r;
}

int hqc_decrypt_batch_staged(int level, int64_t count, const uint64_t* u, const uint64_t* v, const uint32_t* y,
                             const hqc_keyset_t* keys, const int32_t* key_idx, void* workspace,
                             size_t workspace_bytes, uint8_t* m_out, void* stream) {
  hqc_params_t p{};
  int rc = check_common(level, count, u, v, m_out, &p);
  if (rc != HQC_OK || count == 0) return rc;
  const bool keyed = keys != nullptr;
  if (keyed) {
    if (keys->level != level) return fail(HQC_EINVAL, "keys registered for another level");
    if (!key_idx || !aligned(key_idx, 4)) return fail(HQC_EINVAL, "key_idx must be a non-NULL aligned device pointer");
  } else if (!y || !aligned(y, 4)) {
    return fail(HQC_EINVAL, "give y, or keys and key_idx");
  }
  const size_t need = hqc_staged_workspace_bytes(level, count);
  if (!workspace || !aligned(workspace, 16)) return fail(HQC_EINVAL, "workspace must be a 16-byte aligned device pointer");
  if (workspace_bytes < need) return fail(HQC_ENOMEM, "workspace has %zu bytes, needs %zu", workspace_bytes, need);
  hqc::DecArgs a;
  a.count = count;
  a.u = u;
  a.v = v;
  a.y = keyed ? keys->d_table : y;
  a.key_idx = key_idx;
  a.nkeys = keyed ? keys->nkeys : 0;
  a.m = m_out;
  uint64_t* w = static_cast<uint64_t*>(workspace);
  uint8_t* r = reinterpret_cast<uint8_t*>(w + (size_t)count * p.W_v);
  return launch_result(hqc::launch_staged(level, keyed, a, w, r, (cudaStream_t)stream), "staged decrypt launch");
}

int hqc_decrypt_debug(int level, int64_t count, const uint64_t* u, const uint64_t* v, const uint32_t* y,
                      const hqc_debug_dump_t* dump, uint8_t* m_out, void* stream) {
  hqc_params_t p{};
  int rc = check_common(level, count, u, v, m_out, &p);
  if (rc != HQC_OK || count == 0) return rc;
  if (!y || !dump) return fail(HQC_EINVAL, "y and dump must be non-NULL");
  if (!dump->t || !dump->w || !dump->r || !dump->S || !dump->lam || !dump->L || !dump->errmask || !dump->errval ||
      !dump->cw || !dump->flag)
    return fail(HQC_EINVAL, "every dump pointer must be non-NULL");
  if (!aligned(dump->w, 16)) return fail(HQC_EINVAL, "dump->w must be 16-byte aligned");
  hqc::DecArgs a;
  a.count = count;
  a.u = u;
  a.v = v;
  a.y = y;
  a.m = m_out;
  hqc::DebugArgs d{dump->t, dump->w, dump->r, dump->S, dump->lam, dump->L, dump->errmask, dump->errval, dump->cw, dump->flag};
  return launch_result(hqc::launch_debug(level, a, d, (cudaStream_t)stream), "debug decrypt launch");
}

int hqc_decrypt_debug_team(int level, int form, int64_t count, const uint64_t* u, const uint64_t* v, const uint32_t* y,
                           const hqc_debug_dump_t* dump, uint8_t* m_out, void* stream) {
  hqc_params_t p{};
  int rc = check_common(level, count, u, v, m_out, &p);
  if (rc != HQC_OK) return rc;
  if (form < 0 || form > 2)
    return fail(HQC_EINVAL, "form must be 0 (four-warp team), 1 (cluster) or 2 (throughput kernels)");
  if (count == 0) return HQC_OK;
  if (!y || !dump) return fail(HQC_EINVAL, "y and dump must be non-NULL");
  if (!dump->r || !dump->S || !dump->lam) return fail(HQC_EINVAL, "dump->r, dump->S and dump->lam must be non-NULL");
  hqc::DecArgs a;
  a.count = count;
  a.u = u;
  a.v = v;
  a.y = y;
  a.m = m_out;
  hqc::DebugArgs d{nullptr, nullptr, dump->r, dump->S, dump->lam, nullptr, nullptr, nullptr, nullptr, nullptr};
  return launch_result(hqc::launch_debug_team(level, form, a, d, (cudaStream_t)stream), "debug team launch");
}

size_t hqc_mixed_workspace_bytes(void) { return 256; }

int hqc_decrypt_mixed(int64_t count, const hqc_item_t* items, const uint64_t* arena, int64_t arena_words,
                      const hqc_keyset_t* const keys[3], uint8_t* m_arena, int64_t m_bytes, void* workspace,
                      size_t workspace_bytes, void* stream) {
  g_err.clear();
  static_assert(sizeof(hqc_item_t) == sizeof(hqc::MixedItem), "item layout");
  if (count < 0) return fail(HQC_EINVAL, "count must be >= 0");
  if (count == 0) return HQC_OK;
  if (count > ((int64_t)1 << 31)) return fail(HQC_EINVAL, "count must be <= 2^31");
  if (!items || !arena || !m_arena || !keys) return fail(HQC_EINVAL, "items, arena, m_arena and keys must be non-NULL");
  if (!aligned(items, 8) || !aligned(arena, 16)) return fail(HQC_EINVAL, "items 8-byte and arena 16-byte aligned");
  if (arena_words < 0 || m_bytes < 0) return fail(HQC_EINVAL, "negative arena size");
  if (!workspace || !aligned(workspace, 16) || workspace_bytes < hqc_mixed_workspace_bytes())
    return fail(HQC_ENOMEM, "workspace must be >= %zu bytes, 16-byte aligned", hqc_mixed_workspace_bytes());
  hqc::MixedArgs a;
  a.count = count;
  a.items = reinterpret_cast<const hqc::MixedItem*>(items);
  a.arena = arena;
  a.arena_words = arena_words;
  const int lv[3] = {1, 3, 5};
  for (int i = 0; i < 3; i++) {
    if (keys[i]) {
      if (keys[i]->level != lv[i]) return fail(HQC_EINVAL, "keys[%d] is not a level-%d keyset", i, lv[i]);
      a.keys[i] = keys[i]->d_table;
      a.nkeys[i] = keys[i]->nkeys;
    }
  }
  a.m = m_arena;
  a.m_bytes = m_bytes;
  // a small batch with the default shape: one team of warps per item
  if (count <= hqc::MIXED_LATENCY_MAX && g_cfg[0].warps_per_cta == 0 && g_cfg[0].ctas_per_sm == 0)
    return launch_result(hqc::launch_mixed_latency(a, (cudaStream_t)stream), "mixed decrypt launch");
  a.counter = static_cast<uint32_t*>(workspace);
  cudaError_t e = cudaMemsetAsync(workspace, 0, sizeof(uint32_t), (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "zeroing the work counter");
  return launch_result(hqc::launch_mixed(a, (cudaStream_t)stream, g_cfg[0]), "mixed decrypt launch");
}

int hqc_set_launch_config(int level, const hqc_launch_cfg_t* cfg) {
  g_err.clear();
  const int idx = level == 0 ? 0 : hqc::level_index(level) + 1;
  if (level != 0 && idx == 0) return fail(HQC_EINVAL, "level must be 0, 1, 3 or 5");
  if (!cfg) {
    g_cfg[idx] = hqc::LaunchCfg{};
    return HQC_OK;
  }
  if (cfg->warps_per_cta < 0 || cfg->warps_per_cta > 32 || cfg->ctas_per_sm < 0 || cfg->ctas_per_sm > 32)
    return fail(HQC_EINVAL, "warps_per_cta in [0, 32], ctas_per_sm in [0, 32]");
  g_cfg[idx].warps_per_cta = cfg->warps_per_cta;
  g_cfg[idx].ctas_per_sm = cfg->ctas_per_sm;
  return HQC_OK;
}

int hqc_get_launch_shape(int level, int keyed, int32_t* warps, int32_t* ctas_per_sm, int32_t* grid) {
  g_err.clear();
  if (hqc::level_index(level) < 0) return fail(HQC_EINVAL, "level must be 1, 3 or 5");
  int w = 0, c = 0, g = 0;
  cudaError_t e = hqc::fused_occupancy(level, keyed != 0, g_cfg[hqc::level_index(level) + 1], &w, &c, &g);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
  if (warps) *warps = w;
  if (ctas_per_sm) *ctas_per_sm = c;
  if (grid) *grid = g;
  return HQC_OK;
}

int hqc_keygen_batch(int level, int64_t nkeys, const uint64_t* h, const uint32_t* x, const uint32_t* y,
                     uint64_t* s_out, void* stream) {
  g_err.clear();
  hqc_params_t p{};
  if (!params_of(level, &p)) return fail(HQC_EINVAL, "level must be 1, 3 or 5");
  if (nkeys < 0) return fail(HQC_EINVAL, "nkeys must be >= 0");
  if (nkeys == 0) return HQC_OK;
  if (!h || !x || !y || !s_out) return fail(HQC_EINVAL, "NULL pointer");
  if (!aligned(h, 16) || !aligned(s_out, 16)) return fail(HQC_EINVAL, "h and s_out must be 16-byte aligned");
  return launch_result(hqc::launch_keygen(level, nkeys, h, x, y, s_out, (cudaStream_t)stream), "keygen launch");
}

int hqc_encrypt_batch(int level, int64_t count, const uint64_t* h, const uint64_t* s, int64_t nkeys,
                      const int32_t* key_idx, const uint8_t* m, const uint32_t* r1, const uint32_t* r2,
                      const uint32_t* e, uint64_t* u_out, uint64_t* v_out, void* stream) {
  g_err.clear();
  hqc_params_t p{};
  if (!params_of(level, &p)) return fail(HQC_EINVAL, "level must be 1, 3 or 5");
  if (count < 0 || nkeys < 0) return fail(HQC_EINVAL, "count and nkeys must be >= 0");
  if (count == 0) return HQC_OK;
  if (nkeys == 0) return fail(HQC_EINVAL, "nkeys must be >= 1");
  if (!h || !s || !key_idx || !m || !r1 || !r2 || !e || !u_out || !v_out) return fail(HQC_EINVAL, "NULL pointer");
  if (!aligned(h, 16) || !aligned(s, 16) || !aligned(u_out, 16) || !aligned(v_out, 16))
    return fail(HQC_EINVAL, "h, s, u_out and v_out must be 16-byte aligned");
  return launch_result(hqc::launch_encrypt(level, count, h, s, nkeys, key_idx, m, r1, r2, e, u_out, v_out,
                                           (cudaStream_t)stream),
                       "encrypt launch");
}

}  // extern "C"

// Plans: a fixed batch (pointers and count) captured once in a CUDA graph
// and replayed with one cudaGraphLaunch, with the kernel variant and the
// launch shape chosen by an autotuner that times the candidates on the
// caller's own data and keeps every measurement (hqc_plan_describe).
//
//  * keyed plan  -- one level: every kernel variant (the library's default
//    choice; solo warps taking G = 1, 2 or 4 ciphertexts per turn; two-warp
//    teams sharing one operand) at every launch shape (warps per block x
//    blocks per SM).
//  * mixed plan  -- a shuffled HQC-1/3/5 item list.  Four forms compete:
//      (1) the single mixed persistent kernel (dynamic work counter), at
//          every launch shape;
//      (2) the list partitioned by level once at plan creation, one
//          persistent kernel per level side by side as parallel branches of
//          the graph, each on its own share of the SMs;
//      (3) the same per-level kernels one after another, each on the whole
//          GPU;
//      (4) one launch whose blocks take a level by block range, each level
//          with its own warp count and shared-memory layout.
//    Forms 2-4 use, per level, the kernel variant that ran that level
//    fastest alone; the SM shares of forms 2 and 4 start proportional to
//    the levels' solo times and are then refined by measurement.  Forms 2-4
//    let every level run at its own occupancy (HQC-1 fits 32 warps per SM,
//    HQC-5 13 solo warps or 12 teams) instead of all items at HQC-5's.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/hqc_gb300.h"
#include "hqc_internal.h"
#include "hqc_params.cuh"

// One measurement of the tuner: a form, its kernel variant(s), a launch
// shape or per-level block counts, and the mean time of one batch.
struct PlanCand {
  int kind;
  int levels;      // bit i set: level i's items took part (all present ones, except in per-level solo runs)
  int variant[3];  // keyed: variant[0]; mixed forms 2-4: per level 1, 3, 5
  int warps, ctas;
  int grid[3];
  float ms;
};

struct hqc_plan_s {
  int kind = 0;  // 0 keyed, 1 mixed single kernel, 2 mixed level-partitioned, 3 mixed per-level sequential,
                 // 4 mixed one launch by block ranges
  int level = 0;
  int variant = hqc::VAR_DEFAULT;       // keyed: kernel variant
  int lvariant[3] = {hqc::VAR_DEFAULT, hqc::VAR_DEFAULT, hqc::VAR_DEFAULT};  // forms 2, 3: per level
  hqc::DecArgs dec;
  hqc::MixedArgs mixed;                 // the caller's list (single kernel form)
  hqc::MixedArgs part[3];               // per-level lists (partitioned forms)
  hqc::MixedItem* d_items = nullptr;    // plan-owned, partitioned copy
  uint32_t* d_counter = nullptr;        // plan-owned work counter
  hqc::LaunchCfg cfg;
  int grid[3] = {0, 0, 0};              // forms 2, 4: blocks per level
  float tuned_ms = 0.f;
  std::vector<PlanCand> cands;          // every candidate the tuner timed
  cudaStream_t side[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t fork = nullptr, join[3] = {nullptr, nullptr, nullptr};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

int pfail(int code, const char* fmt, ...) {
  char buf[400];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  hqc::set_last_error(buf);
  return code;
}

int pcuda(cudaError_t e, const char* what) {
  return pfail(HQC_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

const int kLevels[3] = {1, 3, 5};

// Enqueue the plan's work once on `st` (also used inside graph capture).
cudaError_t enqueue(hqc_plan_s* p, cudaStream_t st) {
  if (p->kind == 0) return hqc::launch_fused_variant(p->level, p->variant, p->dec, st, p->cfg);
  if (p->kind == 1) {
    cudaError_t e = cudaMemsetAsync(p->d_counter, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    return hqc::launch_mixed(p->mixed, st, p->cfg);
  }
  if (p->kind == 4) return hqc::launch_mixed_ranges(p->part, p->grid, st);
  if (p->kind == 3) {
    for (int li = 2; li >= 0; li--) {
      if (p->part[li].count == 0) continue;
      cudaError_t e = hqc::launch_items_variant(kLevels[li], p->lvariant[li], p->part[li], 0, st, hqc::LaunchCfg{});
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  // partitioned: fork onto side streams, one kernel per level, join back
  cudaError_t e = cudaEventRecord(p->fork, st);
  if (e != cudaSuccess) return e;
  for (int li = 2; li >= 0; li--) {
    if (p->part[li].count == 0) continue;
    if ((e = cudaStreamWaitEvent(p->side[li], p->fork, 0)) != cudaSuccess) return e;
    if ((e = hqc::launch_items_variant(kLevels[li], p->lvariant[li], p->part[li], p->grid[li], p->side[li],
                                       hqc::LaunchCfg{})) != cudaSuccess)
      return e;
    if ((e = cudaEventRecord(p->join[li], p->side[li])) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(st, p->join[li], 0)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Mean time of `reps` back-to-back enqueues on `st` (after one warm-up).
cudaError_t time_enqueue(hqc_plan_s* p, cudaStream_t st, int reps, float* ms) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaError_t e = enqueue(p, st);
  if (e == cudaSuccess) e = cudaEventRecord(a, st);
  for (int i = 0; i < reps && e == cudaSuccess; i++) e = enqueue(p, st);
  if (e == cudaSuccess) e = cudaEventRecord(b, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *ms = t / reps;
  return e;
}

// Time the plan's current configuration and record it; a configuration
// that cannot launch (shape does not fit) is skipped.  Returns the time or
// a huge value.
float measure(hqc_plan_s* p, cudaStream_t st, int reps) {
  float ms = 0.f;
  if (time_enqueue(p, st, reps, &ms) != cudaSuccess) {
    cudaGetLastError();
    return 1e30f;
  }
  PlanCand c;
  c.kind = p->kind;
  c.levels = 0;
  if (p->kind == 0 || p->kind == 1) {
    c.levels = 7;
  } else {
    for (int i = 0; i < 3; i++) c.levels |= p->part[i].count > 0 ? 1 << i : 0;
  }
  if (p->kind == 0) {
    c.variant[0] = p->variant;
    c.variant[1] = c.variant[2] = -1;
  } else {
    for (int i = 0; i < 3; i++) c.variant[i] = p->lvariant[i];
  }
  c.warps = p->cfg.warps_per_cta;
  c.ctas = p->cfg.ctas_per_sm;
  for (int i = 0; i < 3; i++) c.grid[i] = p->grid[i];
  c.ms = ms;
  p->cands.push_back(c);
  return ms;
}

int capture(hqc_plan_s* p) {
  cudaStream_t cs;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return pcuda(e, "capture stream");
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    cudaError_t e2 = enqueue(p, cs);
    e = cudaStreamEndCapture(cs, &p->graph);
    if (e2 != cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
  cudaStreamDestroy(cs);
  return e == cudaSuccess ? HQC_OK : pcuda(e, "graph capture");
}

void release(hqc_plan_s* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  for (int i = 0; i < 3; i++) {
    if (p->side[i]) cudaStreamDestroy(p->side[i]);
    if (p->join[i]) cudaEventDestroy(p->join[i]);
  }
  if (p->fork) cudaEventDestroy(p->fork);
  cudaFree(p->d_items);
  cudaFree(p->d_counter);
  delete p;
}

// Candidate launch shapes for a single persistent kernel.
std::vector<hqc::LaunchCfg> shape_candidates(int max_warps) {
  std::vector<hqc::LaunchCfg> c;
  for (int w : {4, 8, 12, 16, 18, 20, 22, 24, 26, 27, 28, 30, 32})
    if (w <= max_warps)
      for (int k : {1, 2}) c.push_back(hqc::LaunchCfg{w, k});
  c.push_back(hqc::LaunchCfg{});  // library default
  return c;
}

// Blocks per level for the forms that share the GPU between the levels
// (2: parallel graph branches, 4: one launch by block ranges): shares of
// `total` blocks proportional to the levels' solo times, then a few moves
// of blocks between levels; leaves the best split in p->grid and returns
// its time.
float tune_shares(hqc_plan_s* p, cudaStream_t st, int total, const float solo[3]) {
  const float tot = solo[0] + solo[1] + solo[2];
  if (tot <= 0.f) return 1e30f;
  int base[3], used = 0;
  for (int i = 0; i < 3; i++) {
    base[i] = p->part[i].count > 0 ? std::max(1, (int)(total * solo[i] / tot + 0.5f)) : 0;
    used += base[i];
  }
  const int big = (int)(std::max_element(base, base + 3) - base);
  base[big] += total - used;
  const int deltas[][3] = {{0, 0, 0}, {4, -2, -2}, {-4, 2, 2}, {-2, 4, -2}, {2, -4, 2}, {-2, -2, 4},
                           {2, 2, -4}, {8, -4, -4}, {-8, 4, 4}};
  float best = 1e30f;
  int gbest[3] = {base[0], base[1], base[2]};
  for (const auto& d : deltas) {
    bool ok = true;
    for (int i = 0; i < 3; i++) {
      p->grid[i] = p->part[i].count > 0 ? base[i] + d[i] : 0;
      if (p->part[i].count > 0 && p->grid[i] < 1) ok = false;
    }
    if (!ok) continue;
    const float ms = measure(p, st, 3);
    if (ms < best) {
      best = ms;
      for (int i = 0; i < 3; i++) gbest[i] = p->grid[i];
    }
  }
  for (int i = 0; i < 3; i++) p->grid[i] = gbest[i];
  return best;
}

const char* form_name(int kind) {
  switch (kind) {
    case 0: return "keyed";
    case 1: return "mixed-single-kernel";
    case 2: return "mixed-level-partitioned";
    case 3: return "mixed-per-level-sequential";
    case 4: return "mixed-one-launch-block-ranges";
  }
  return "?";
}

}  // namespace

extern "C" {

// mode 0: the library's default kernel and shape; 1: tune; 2: the given
// variant and shape
static int keyed_plan(int level, int64_t count, const uint64_t* u, const uint64_t* v, const hqc_keyset_t* keys,
                      const int32_t* key_idx, uint8_t* m_out, int mode, int fixed_variant,
                      const hqc_launch_cfg_t* fixed_cfg, void* stream, hqc_plan_t** out) {
  if (!out) return pfail(HQC_EINVAL, "out is NULL");
  *out = nullptr;
  hqc_params_t prm;
  if (hqc_get_params(level, &prm) != HQC_OK) return HQC_EINVAL;
  if (count <= 0) return pfail(HQC_EINVAL, "count must be >= 1");
  if (!u || !v || !m_out || !keys || !key_idx) return pfail(HQC_EINVAL, "NULL argument");
  if (((uintptr_t)u | (uintptr_t)v) % 16) return pfail(HQC_EINVAL, "u and v must be 16-byte aligned");
  if (keys->level != level) return pfail(HQC_EINVAL, "keys registered for another level");
  cudaStream_t st = (cudaStream_t)stream;
  hqc_plan_s* p = new hqc_plan_s;
  p->kind = 0;
  p->level = level;
  p->dec.count = count;
  p->dec.u = u;
  p->dec.v = v;
  p->dec.y = keys->d_table;
  p->dec.key_idx = key_idx;
  p->dec.nkeys = keys->nkeys;
  p->dec.m = m_out;
  p->cfg = hqc::level_cfg(level);
  if (mode == 2) {
    p->variant = fixed_variant;
    p->cfg = fixed_cfg ? hqc::LaunchCfg{fixed_cfg->warps_per_cta, fixed_cfg->ctas_per_sm} : hqc::LaunchCfg{};
  }
  if (mode == 1) {
    // every kernel variant (the library's default choice, solo warps with
    // G = 1, 2, 4 ciphertexts per turn, two-warp teams) at every shape
    float best = 1e30f;
    int bestv = hqc::VAR_DEFAULT;
    hqc::LaunchCfg bestc;
    for (int var = 0; var < hqc::VAR_COUNT; var++) {
      if (!hqc::variant_exists(level, var)) continue;
      for (const hqc::LaunchCfg& c : shape_candidates(32)) {
        p->variant = var;
        p->cfg = c;
        const float ms = measure(p, st, 3);
        if (ms < best) {
          best = ms;
          bestv = var;
          bestc = c;
        }
      }
    }
    p->variant = bestv;
    p->cfg = bestc;
    p->tuned_ms = best < 1e30f ? best : 0.f;
  }
  int rc = capture(p);
  if (rc != HQC_OK) {
    release(p);
    return rc;
  }
  *out = p;
  return HQC_OK;
}

int hqc_plan_create_keyed(int level, int64_t count, const uint64_t* u, const uint64_t* v, const hqc_keyset_t* keys,
                          const int32_t* key_idx, uint8_t* m_out, int autotune, void* stream, hqc_plan_t** out) {
  return keyed_plan(level, count, u, v, keys, key_idx, m_out, autotune ? 1 : 0, 0, nullptr, stream, out);
}

int hqc_plan_create_keyed_fixed(int level, int64_t count, const uint64_t* u, const uint64_t* v,
                                const hqc_keyset_t* keys, const int32_t* key_idx, uint8_t* m_out, int variant,
                                const hqc_launch_cfg_t* cfg, void* stream, hqc_plan_t** out) {
  if (out) *out = nullptr;
  if (variant < 0 || variant >= hqc::VAR_COUNT || !hqc::variant_exists(level, variant))
    return pfail(HQC_EINVAL, "variant %d does not exist at level %d", variant, level);
  if (cfg && (cfg->warps_per_cta < 0 || cfg->warps_per_cta > 32 || cfg->ctas_per_sm < 0 || cfg->ctas_per_sm > 32))
    return pfail(HQC_EINVAL, "warps_per_cta in [0, 32], ctas_per_sm in [0, 32]");
  return keyed_plan(level, count, u, v, keys, key_idx, m_out, 2, variant, cfg, stream, out);
}

// mode 0: the single mixed kernel at the default shape; 1: tune; 2: the
// given form, shape, per-level variants and blocks
static int mixed_plan(int64_t count, const hqc_item_t* items, const uint64_t* arena, int64_t arena_words,
                      const hqc_keyset_t* const keys[3], uint8_t* m_arena, int64_t m_bytes, int mode, int fixed_form,
                      const hqc_launch_cfg_t* fixed_cfg, const int32_t* fixed_variants, const int32_t* fixed_grids,
                      void* stream, hqc_plan_t** out) {
  if (!out) return pfail(HQC_EINVAL, "out is NULL");
  *out = nullptr;
  if (count <= 0 || count > ((int64_t)1 << 31)) return pfail(HQC_EINVAL, "count must be in [1, 2^31]");
  if (!items || !arena || !m_arena || !keys) return pfail(HQC_EINVAL, "NULL argument");
  if ((uintptr_t)items % 8 || (uintptr_t)arena % 16) return pfail(HQC_EINVAL, "items 8-byte, arena 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  hqc_plan_s* p = new hqc_plan_s;
  p->kind = 1;
  hqc::MixedArgs& a = p->mixed;
  a.count = count;
  a.items = reinterpret_cast<const hqc::MixedItem*>(items);
  a.arena = arena;
  a.arena_words = arena_words;
  for (int i = 0; i < 3; i++) {
    if (keys[i]) {
      if (keys[i]->level != kLevels[i]) {
        release(p);
        return pfail(HQC_EINVAL, "keys[%d] is not a level-%d keyset", i, kLevels[i]);
      }
      a.keys[i] = keys[i]->d_table;
      a.nkeys[i] = keys[i]->nkeys;
    }
  }
  a.m = m_arena;
  a.m_bytes = m_bytes;
  cudaError_t e = cudaMalloc(&p->d_counter, 256);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_items, (size_t)count * sizeof(hqc::MixedItem));
  if (e != cudaSuccess) {
    release(p);
    return pfail(HQC_ENOMEM, "plan buffers: %s", cudaGetErrorString(e));
  }
  a.counter = p->d_counter;
  // partition the item list by level once (host round trip at creation)
  std::vector<hqc::MixedItem> h((size_t)count), sorted;
  sorted.reserve((size_t)count);
  e = cudaMemcpy(h.data(), items, h.size() * sizeof(hqc::MixedItem), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    release(p);
    return pcuda(e, "reading the item list");
  }
  int64_t start[3] = {0, 0, 0}, n[3] = {0, 0, 0};
  for (int i = 0; i < 3; i++) {
    start[i] = (int64_t)sorted.size();
    for (const auto& it : h)
      if (it.level == kLevels[i]) sorted.push_back(it);
    n[i] = (int64_t)sorted.size() - start[i];
  }
  if (!sorted.empty()) {
    e = cudaMemcpy(p->d_items, sorted.data(), sorted.size() * sizeof(hqc::MixedItem), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      release(p);
      return pcuda(e, "writing the partitioned list");
    }
  }
  for (int i = 0; i < 3; i++) {
    p->part[i] = a;
    p->part[i].items = p->d_items + start[i];
    p->part[i].count = n[i];
    p->part[i].counter = nullptr;
    if ((e = cudaStreamCreateWithFlags(&p->side[i], cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&p->join[i], cudaEventDisableTiming)) != cudaSuccess) {
      release(p);
      return pcuda(e, "plan streams");
    }
  }
  if ((e = cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming)) != cudaSuccess) {
    release(p);
    return pcuda(e, "plan events");
  }
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);

  p->kind = 1;
  p->cfg = hqc::LaunchCfg{};
  float best = 0.f;
  if (mode == 2) {
    p->kind = fixed_form;
    if (fixed_cfg) p->cfg = hqc::LaunchCfg{fixed_cfg->warps_per_cta, fixed_cfg->ctas_per_sm};
    for (int i = 0; i < 3; i++) {
      p->lvariant[i] = fixed_variants ? fixed_variants[i] : hqc::VAR_DEFAULT;
      p->grid[i] = fixed_grids ? fixed_grids[i] : 0;
      if (p->lvariant[i] < 0 || p->lvariant[i] >= hqc::VAR_COUNT || !hqc::variant_exists(kLevels[i], p->lvariant[i])) {
        release(p);
        return pfail(HQC_EINVAL, "variant %d does not exist at level %d", p->lvariant[i], kLevels[i]);
      }
      if ((fixed_form == 2 || fixed_form == 4) && p->part[i].count > 0 && p->grid[i] < 1) {
        release(p);
        return pfail(HQC_EINVAL, "forms 2 and 4 need at least one block for every level present");
      }
    }
  }
  if (mode == 1) {
    // form 1: the single mixed kernel at every shape
    float b1 = 1e30f;
    hqc::LaunchCfg bc;
    int mw = 0, mc = 0, mg = 0;
    hqc::mixed_occupancy(hqc::LaunchCfg{}, &mw, &mc, &mg);
    for (const hqc::LaunchCfg& c : shape_candidates(mw)) {
      p->cfg = c;
      const float ms = measure(p, st, 3);
      if (ms < b1) {
        b1 = ms;
        bc = c;
      }
    }
    p->cfg = bc;
    best = b1;
    int kind = 1;
    // each level alone on the whole GPU, every kernel variant: the fastest
    // variant per level, and the levels' solo times for the SM shares
    float solo[3] = {0.f, 0.f, 0.f};
    hqc::MixedArgs keep[3] = {p->part[0], p->part[1], p->part[2]};
    p->kind = 3;
    for (int i = 0; i < 3; i++) {
      if (keep[i].count == 0) continue;
      for (int j = 0; j < 3; j++) p->part[j].count = j == i ? keep[j].count : 0;
      float bs = 1e30f;
      int bv = hqc::VAR_DEFAULT;
      for (int var = 0; var < hqc::VAR_COUNT; var++) {
        if (!hqc::variant_exists(kLevels[i], var)) continue;
        p->lvariant[i] = var;
        const float ms = measure(p, st, 2);
        if (ms < bs) {
          bs = ms;
          bv = var;
        }
      }
      p->lvariant[i] = bv;
      solo[i] = bs < 1e30f ? bs : 0.f;
    }
    for (int j = 0; j < 3; j++) p->part[j] = keep[j];
    // form 3: the levels one after another, each on the whole GPU
    const float b3 = measure(p, st, 3);
    if (b3 < best) {
      best = b3;
      kind = 3;
    }
    // form 2: the levels side by side as graph branches on shares of the SMs
    p->kind = 2;
    const float b2 = tune_shares(p, st, sms, solo);
    const int g2[3] = {p->grid[0], p->grid[1], p->grid[2]};
    if (b2 < best) {
      best = b2;
      kind = 2;
    }
    // form 4: one launch, blocks taking a level by block range
    p->kind = 4;
    const float b4 = tune_shares(p, st, sms, solo);
    if (b4 < best) {
      best = b4;
      kind = 4;
    }
    p->kind = kind;
    if (kind == 2)
      for (int i = 0; i < 3; i++) p->grid[i] = g2[i];
    if (kind != 2 && kind != 4)
      for (int i = 0; i < 3; i++) p->grid[i] = 0;
  }
  p->tuned_ms = best;
  int rc = capture(p);
  if (rc != HQC_OK) {
    release(p);
    return rc;
  }
  *out = p;
  return HQC_OK;
}

int hqc_plan_create_mixed(int64_t count, const hqc_item_t* items, const uint64_t* arena, int64_t arena_words,
                          const hqc_keyset_t* const keys[3], uint8_t* m_arena, int64_t m_bytes, int autotune,
                          void* stream, hqc_plan_t** out) {
  return mixed_plan(count, items, arena, arena_words, keys, m_arena, m_bytes, autotune ? 1 : 0, 1, nullptr, nullptr,
                    nullptr, stream, out);
}

int hqc_plan_create_mixed_fixed(int64_t count, const hqc_item_t* items, const uint64_t* arena, int64_t arena_words,
                                const hqc_keyset_t* const keys[3], uint8_t* m_arena, int64_t m_bytes, int form,
                                const hqc_launch_cfg_t* cfg, const int32_t* variants3, const int32_t* grids3,
                                void* stream, hqc_plan_t** out) {
  if (out) *out = nullptr;
  if (form < 1 || form > 4) return pfail(HQC_EINVAL, "form must be 1, 2, 3 or 4");
  if (cfg && (cfg->warps_per_cta < 0 || cfg->warps_per_cta > 32 || cfg->ctas_per_sm < 0 || cfg->ctas_per_sm > 32))
    return pfail(HQC_EINVAL, "warps_per_cta in [0, 32], ctas_per_sm in [0, 32]");
  return mixed_plan(count, items, arena, arena_words, keys, m_arena, m_bytes, 2, form, cfg, variants3, grids3, stream,
                    out);
}

int hqc_plan_launch(hqc_plan_t* plan, void* stream) {
  if (!plan || !plan->exec) return pfail(HQC_EINVAL, "plan is NULL or not instantiated");
  cudaError_t e = cudaGraphLaunch(plan->exec, (cudaStream_t)stream);
  return e == cudaSuccess ? HQC_OK : pcuda(e, "cudaGraphLaunch");
}

int hqc_plan_info(const hqc_plan_t* plan, int32_t* form, hqc_launch_cfg_t* cfg, int32_t* grids3, float* tuned_ms) {
  if (!plan) return pfail(HQC_EINVAL, "plan is NULL");
  if (form) *form = plan->kind;
  if (cfg) {
    cfg->warps_per_cta = plan->cfg.warps_per_cta;
    cfg->ctas_per_sm = plan->cfg.ctas_per_sm;
  }
  if (grids3)
    for (int i = 0; i < 3; i++) grids3[i] = plan->grid[i];
  if (tuned_ms) *tuned_ms = plan->tuned_ms;
  return HQC_OK;
}

int hqc_plan_describe(const hqc_plan_t* plan, char* buf, size_t cap) {
  if (!plan || !buf || cap == 0) return pfail(HQC_EINVAL, "plan and buf must be non-NULL, cap > 0");
  std::string o;
  char t[256];
  auto vname = [](int v) { return v < 0 ? "-" : hqc::variant_name(v); };
  snprintf(t, sizeof t, "{\"form\": \"%s\", ", form_name(plan->kind));
  o += t;
  if (plan->kind == 0) {
    snprintf(t, sizeof t, "\"variant\": \"%s\", ", vname(plan->variant));
    o += t;
  } else {
    snprintf(t, sizeof t, "\"level_variants\": [\"%s\", \"%s\", \"%s\"], ", vname(plan->lvariant[0]),
             vname(plan->lvariant[1]), vname(plan->lvariant[2]));
    o += t;
  }
  snprintf(t, sizeof t, "\"warps_per_cta\": %d, \"ctas_per_sm\": %d, \"grids\": [%d, %d, %d], \"tuned_ms\": %.5f, ",
           plan->cfg.warps_per_cta, plan->cfg.ctas_per_sm, plan->grid[0], plan->grid[1], plan->grid[2],
           plan->tuned_ms);
  o += t;
  // the levels the whole batch holds (candidates with fewer were per-level
  // solo runs that chose each level's variant)
  int whole = 7;
  if (plan->kind != 0) {
    whole = 0;
    for (int i = 0; i < 3; i++) whole |= plan->part[i].count > 0 ? 1 << i : 0;
    if (plan->kind == 1 && whole == 0) whole = 7;
  }
  std::vector<PlanCand> c = plan->cands;
  for (auto& x : c)
    if (x.kind == 0 || x.kind == 1) x.levels = whole;
  std::sort(c.begin(), c.end(), [](const PlanCand& x, const PlanCand& y) { return x.ms < y.ms; });
  o += "\"candidates\": [";
  for (size_t i = 0; i < c.size(); i++) {
    snprintf(t, sizeof t,
             "%s{\"form\": \"%s\", \"whole_batch\": %s, \"levels\": [%s%s%s], \"variants\": [\"%s\", \"%s\", "
             "\"%s\"], \"warps\": %d, \"ctas\": %d, \"grids\": [%d, %d, %d], \"ms\": %.5f}",
             i ? ", " : "", form_name(c[i].kind), c[i].levels == whole ? "true" : "false",
             c[i].levels & 1 ? "1" : "", c[i].levels & 2 ? ((c[i].levels & 1) ? ", 3" : "3") : "",
             c[i].levels & 4 ? ((c[i].levels & 3) ? ", 5" : "5") : "", vname(c[i].variant[0]),
             vname(c[i].variant[1]), vname(c[i].variant[2]), c[i].warps, c[i].ctas, c[i].grid[0], c[i].grid[1],
             c[i].grid[2], c[i].ms);
    o += t;
  }
  o += "]}";
  if (o.size() + 1 > cap) return pfail(HQC_ENOMEM, "description needs %zu bytes", o.size() + 1);
  memcpy(buf, o.c_str(), o.size() + 1);
  return HQC_OK;
}

int hqc_plan_destroy(hqc_plan_t* plan) {
  release(plan);
  return HQC_OK;
}

}  // extern "C"

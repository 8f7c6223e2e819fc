// Plans: a fixed batch (pointers and count) captured once in a CUDA graph
// and replayed with one cudaGraphLaunch, with the launch shape chosen by a
// small autotuner that times candidate shapes on the caller's own data.
//
//  * keyed plan  -- one level, the fused persistent kernel;
//  * mixed plan  -- a shuffled HQC-1/3/5 item list.  Two forms compete:
//      (a) the single mixed persistent kernel (dynamic work counter), and
//      (b) the item list partitioned by level once at plan creation, one
//          persistent kernel per level running side by side as parallel
//          branches of the graph, each on its own share of the SMs (shares
//          proportional to measured per-level time, then refined).
//      (c) the same per-level kernels one after another, each on the whole
//          GPU.
//    (b) and (c) let every level run at its own occupancy (HQC-1 fits 32
//    warps per SM, HQC-5 13) instead of all items at HQC-5's.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/hqc_gb300.h"
#include "hqc_internal.h"
#include "hqc_params.cuh"

struct hqc_plan_s {
  int kind = 0;  // 0 keyed, 1 mixed single kernel, 2 mixed level-partitioned, 3 mixed per-level sequential
  int level = 0;
  hqc::DecArgs dec;
  hqc::MixedArgs mixed;                 // the caller's list (single kernel form)
  hqc::MixedArgs part[3];               // per-level lists (partitioned form)
  hqc::MixedItem* d_items = nullptr;    // plan-owned, partitioned copy
  uint32_t* d_counter = nullptr;        // plan-owned work counter
  hqc::LaunchCfg cfg;
  int grid[3] = {0, 0, 0};              // partitioned: blocks per level
  float tuned_ms = 0.f;
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

// Enqueue the plan's work once on `st` (also used inside graph capture).
cudaError_t enqueue(hqc_plan_s* p, cudaStream_t st) {
  if (p->kind == 0) return hqc::launch_fused(p->level, true, p->dec, st, p->cfg);
  if (p->kind == 1) {
    cudaError_t e = cudaMemsetAsync(p->d_counter, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    return hqc::launch_mixed(p->mixed, st, p->cfg);
  }
  if (p->kind == 3) {
    const int lv3[3] = {5, 3, 1};
    for (int i = 0; i < 3; i++) {
      const int li = hqc::level_index(lv3[i]);
      if (p->part[li].count == 0) continue;
      cudaError_t e = hqc::launch_items(lv3[i], p->part[li], 0, st, hqc::LaunchCfg{});
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  // partitioned: fork onto side streams, one kernel per level, join back
  cudaError_t e = cudaEventRecord(p->fork, st);
  if (e != cudaSuccess) return e;
  const int lv[3] = {5, 3, 1};
  for (int i = 0; i < 3; i++) {
    const int li = hqc::level_index(lv[i]);
    if (p->part[li].count == 0) continue;
    if ((e = cudaStreamWaitEvent(p->side[li], p->fork, 0)) != cudaSuccess) return e;
    if ((e = hqc::launch_items(lv[i], p->part[li], p->grid[li], p->side[li], hqc::LaunchCfg{})) != cudaSuccess)
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
  for (int w : {4, 8, 12, 16, 20, 24, 32})
    if (w <= max_warps)
      for (int k : {1, 2, 4}) c.push_back(hqc::LaunchCfg{w, k});
  c.push_back(hqc::LaunchCfg{});  // library default
  return c;
}

}  // namespace

extern "C" {

int hqc_plan_create_keyed(int level, int64_t count, const uint64_t* u, const uint64_t* v, const hqc_keyset_t* keys,
                          const int32_t* key_idx, uint8_t* m_out, int autotune, void* stream, hqc_plan_t** out) {
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
  if (autotune) {
    float best = 1e30f;
    hqc::LaunchCfg bestc;
    int mw = 0, mc = 0, mg = 0;
    hqc::fused_occupancy(level, true, hqc::LaunchCfg{}, &mw, &mc, &mg);
    for (const hqc::LaunchCfg& c : shape_candidates(32)) {
      p->cfg = c;
      float ms = 0.f;
      if (time_enqueue(p, st, 3, &ms) != cudaSuccess) {
        cudaGetLastError();  // shape does not fit: skip it
        continue;
      }
      if (ms < best) {
        best = ms;
        bestc = c;
      }
    }
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

int hqc_plan_create_mixed(int64_t count, const hqc_item_t* items, const uint64_t* arena, int64_t arena_words,
                          const hqc_keyset_t* const keys[3], uint8_t* m_arena, int64_t m_bytes, int autotune,
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
  const int lv[3] = {1, 3, 5};
  for (int i = 0; i < 3; i++) {
    if (keys[i]) {
      if (keys[i]->level != lv[i]) {
        release(p);
        return pfail(HQC_EINVAL, "keys[%d] is not a level-%d keyset", i, lv[i]);
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
      if (it.level == lv[i]) sorted.push_back(it);
    n[i] = (int64_t)sorted.size() - start[i];
  }
  e = cudaMemcpy(p->d_items, sorted.data(), sorted.size() * sizeof(hqc::MixedItem), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    release(p);
    return pcuda(e, "writing the partitioned list");
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

  // (a) single mixed kernel, default shape; (b) partitioned, shares from
  // per-level solo times
  float best = 0.f;
  p->kind = 1;
  p->cfg = hqc::LaunchCfg{};
  if (autotune) {
    float bms = 1e30f;
    hqc::LaunchCfg bc;
    int mw = 0, mc = 0, mg = 0;
    hqc::mixed_occupancy(hqc::LaunchCfg{}, &mw, &mc, &mg);
    for (const hqc::LaunchCfg& c : shape_candidates(mw)) {
      p->cfg = c;
      float ms = 0.f;
      if (time_enqueue(p, st, 3, &ms) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      if (ms < bms) {
        bms = ms;
        bc = c;
      }
    }
    p->cfg = bc;
    best = bms;
    // per-level solo times on the whole GPU
    float solo[3] = {0.f, 0.f, 0.f};
    p->kind = 2;
    for (int i = 0; i < 3; i++) {
      int g = 0;
      hqc::items_occupancy(lv[i], hqc::LaunchCfg{}, nullptr, nullptr, &g);
      for (int j = 0; j < 3; j++) p->grid[j] = 0;
      hqc::MixedArgs keep[3] = {p->part[0], p->part[1], p->part[2]};
      for (int j = 0; j < 3; j++)
        if (j != i) p->part[j].count = 0;
      p->grid[i] = g;
      float ms = 0.f;
      if (p->part[i].count > 0 && time_enqueue(p, st, 2, &ms) == cudaSuccess) solo[i] = ms;
      for (int j = 0; j < 3; j++) p->part[j] = keep[j];
    }
    float tot = solo[0] + solo[1] + solo[2];
    if (tot > 0.f) {
      // SM shares proportional to solo time, then a few refinements
      int base[3];
      int used = 0;
      for (int i = 0; i < 3; i++) {
        base[i] = p->part[i].count > 0 ? std::max(1, (int)(sms * solo[i] / tot + 0.5f)) : 0;
        used += base[i];
      }
      int big = (int)(std::max_element(base, base + 3) - base);
      base[big] += sms - used;
      const int deltas[][3] = {{0, 0, 0}, {4, -2, -2}, {-4, 2, 2}, {-2, 4, -2}, {2, -4, 2}, {-2, -2, 4},
                               {2, 2, -4}, {8, -4, -4}, {-8, 4, 4}};
      float pbest = 1e30f;
      int gbest[3] = {base[0], base[1], base[2]};
      for (const auto& d : deltas) {
        bool ok = true;
        for (int i = 0; i < 3; i++) {
          p->grid[i] = base[i] + d[i];
          if (p->part[i].count > 0 && p->grid[i] < 1) ok = false;
          if (p->part[i].count == 0) p->grid[i] = 0;
        }
        if (!ok) continue;
        float ms = 0.f;
        if (time_enqueue(p, st, 3, &ms) != cudaSuccess) {
          cudaGetLastError();
          continue;
        }
        if (ms < pbest) {
          pbest = ms;
          for (int i = 0; i < 3; i++) gbest[i] = p->grid[i];
        }
      }
      for (int i = 0; i < 3; i++) p->grid[i] = gbest[i];
      int kind = 1;
      if (pbest < best) {
        best = pbest;
        kind = 2;
      }
      // (c) sequential per-level kernels on the whole GPU
      p->kind = 3;
      float sms3 = 0.f;
      if (time_enqueue(p, st, 3, &sms3) == cudaSuccess && sms3 < best) {
        best = sms3;
        kind = 3;
      }
      cudaGetLastError();
      p->kind = kind;
    } else {
      p->kind = 1;
    }
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

int hqc_plan_destroy(hqc_plan_t* plan) {
  release(plan);
  return HQC_OK;
}

}  // extern "C"

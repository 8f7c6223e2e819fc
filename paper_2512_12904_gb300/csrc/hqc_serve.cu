// Continuous-batching decryption service loop (host C++).
//
// Requests arrive open-loop at given times.  Their ciphertext rows sit in a
// pinned host ring in arrival order, the way a receive path would leave
// them.  One dispatcher thread:
//   * admits arrived requests into a batch for any free stream, while the
//     batch fits that stream's share of the device-memory budget and
//     max_batch; arrivals beyond max_queue waiting requests are rejected;
//   * per batch: the item list grouped by level, then either (in-place
//     mode) the kernels read the batch's ring range straight from host
//     memory and write m into mapped pinned memory -- one launch (small
//     batch) or one persistent kernel per level, then an event; or (copy
//     mode) one H2D copy of the contiguous ring range, the kernels, one D2H
//     copy of the m bytes, an event;
//   * polls the events; a completed batch frees its memory and stamps every
//     request's completion time.
// So requests that arrive while batches run on the GPU are admitted as soon
// as a stream and its memory free up, and up to `streams` batches overlap
// on the device.  Keys stay resident (registered keysets).
//
// Why in-place reads: measured on GB300, DMA copies from pinned host memory
// run at ~192 GB/s but collapse to ~8 GB/s for tens of milliseconds about
// twice a second, while loads that the SMs issue to the same host memory
// over the C2C link hold ~182 GB/s throughout.  A batch whose upload falls
// into such a window waits milliseconds, and at high load the backlog it
// leaves sets the tail latency.  Reading the ring from the kernels keeps
// the copy engines off the request path altogether.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <thread>
#include <vector>

#include "../../include/hqc_gb300.h"
#include "hqc_internal.h"
#include "hqc_params.cuh"

namespace {

int sfail(int code, const char* fmt, ...) {
  char buf[400];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  hqc::set_last_error(buf);
  return code;
}

struct Slot {
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  uint64_t* d_words = nullptr;       // ring bytes of the batch (copy mode)
  uint8_t* d_m = nullptr;            // m bytes of the batch (copy mode)
  hqc::MixedItem* d_items = nullptr; // grouped by level (copy mode)
  hqc::MixedItem* h_items = nullptr; // pinned, mapped
  uint8_t* h_m = nullptr;            // pinned, mapped
  const hqc::MixedItem* k_items = nullptr;  // what the kernels read: d_items, or h_items' device address
  uint8_t* k_m = nullptr;                   // what the kernels write: d_m, or h_m's device address
  int64_t words_cap = 0, m_cap = 0;
  bool busy = false;
  int64_t t_launch = 0;              // host time the batch was issued
  int64_t first = 0, last = 0;       // requests [first, last)
  bool dense = false;                // every request in [first, last) runs: m is one contiguous range
  int64_t m_first = 0, m_bytes = 0;  // that range of the ring's m layout
};

// Batches of at most this many requests run as one mixed-kernel launch
// (lowest latency); larger ones as one persistent kernel per level.
constexpr int64_t kSmallBatch = hqc::MIXED_LATENCY_MAX;

inline int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

}  // namespace

extern "C" int hqc_serve_run(const hqc_serve_cfg_t* cfg, const hqc_keyset_t* const keys[3],
                             const hqc_serve_ring_t* ring, int64_t count, const int64_t* arrival_ns,
                             int32_t* status, int64_t* latency_ns, uint8_t* m_out, hqc_serve_stats_t* stats) {
  if (!cfg || !keys || !ring || !arrival_ns || !status || !latency_ns) return sfail(HQC_EINVAL, "NULL argument");
  if (cfg->streams < 1 || cfg->streams > 16 || cfg->max_batch < 1 || cfg->budget_bytes <= 0 || cfg->max_queue < 1 ||
      cfg->stall_ms < 0)
    return sfail(HQC_EINVAL, "streams in [1, 16], max_batch >= 1, budget_bytes > 0, max_queue >= 1, stall_ms >= 0");
  const int64_t stall_ns = (int64_t)(cfg->stall_ms ? cfg->stall_ms : 10000) * 1000000;
  if (ring->period < 1 || !ring->level || !ring->key || !ring->word_off || !ring->words || !ring->m_off)
    return sfail(HQC_EINVAL, "ring is incomplete");
  if (count < 0) return sfail(HQC_EINVAL, "count must be >= 0");
  if (cfg->transfer < 0 || cfg->transfer > 2) return sfail(HQC_EINVAL, "transfer must be 0, 1 or 2");
  const int lv[3] = {1, 3, 5};
  hqc_params_t prm[3];
  for (int i = 0; i < 3; i++) hqc_get_params(lv[i], &prm[i]);
  for (int i = 0; i < 3; i++)
    if (keys[i] && keys[i]->level != lv[i]) return sfail(HQC_EINVAL, "keys[%d] is not a level-%d keyset", i, lv[i]);
  // every ring entry's rows lie inside [0, word_off[period]) and its m bytes
  // inside [0, m_off[period]): in in-place mode the kernels read the ring
  // at these offsets, so they are checked once here
  if (ring->word_off[0] != 0 || ring->m_off[0] != 0) return sfail(HQC_EINVAL, "ring offsets must start at 0");
  bool even = ((uintptr_t)ring->words % 16) == 0;  // every row 16-byte aligned in host memory
  for (int64_t j = 0; j < ring->period; j++) {
    if (ring->word_off[j + 1] < ring->word_off[j] || ring->m_off[j + 1] < ring->m_off[j])
      return sfail(HQC_EINVAL, "ring offsets must be non-decreasing (entry %lld)", (long long)j);
    even = even && (ring->word_off[j] & 1) == 0;
  }
  // In-place reads need a device address for the caller's ring -- the mapped
  // address of pinned memory, or the host address itself on a device that
  // reads pageable host memory through the host's page tables -- and rows
  // on 16-byte boundaries (the kernels load u with 16-byte vectors).
  const uint64_t* ring_dev = nullptr;
  if (cfg->transfer == 2 && !even)
    return sfail(HQC_EINVAL, "transfer 2 needs a 16-byte aligned ring with even word offsets");
  if (cfg->transfer != 1 && even) {
    void* p = nullptr;
    if (cudaHostGetDevicePointer(&p, const_cast<uint64_t*>(ring->words), 0) == cudaSuccess) {
      ring_dev = static_cast<const uint64_t*>(p);
    } else {
      cudaGetLastError();
      int dev = 0, pageable = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccessUsesHostPageTables, dev);
      if (pageable) ring_dev = ring->words;
    }
    if (!ring_dev && cfg->transfer == 2)
      return sfail(HQC_EINVAL, "transfer 2: the device cannot read the ring in place (not mapped, no host page tables)");
  }
  const bool in_place = ring_dev != nullptr;

  // per-slot device memory: an even split of the budget between words,
  // m bytes and item records in proportion to the largest request
  const int S = cfg->streams;
  const int64_t per_slot = cfg->budget_bytes / S;
  const int64_t unit = (int64_t)prm[2].W_u_pitch * 8 + (int64_t)prm[2].W_v * 8 + 32 + (int64_t)sizeof(hqc::MixedItem);
  const int64_t max_items = std::max<int64_t>(1, std::min<int64_t>(cfg->max_batch, per_slot / unit));
  std::vector<Slot> slots(S);
  cudaError_t e = cudaSuccess;
  auto cleanup = [&]() {
    for (auto& s : slots) {
      if (s.st) cudaStreamSynchronize(s.st);
      if (s.ev) cudaEventDestroy(s.ev);
      if (s.st) cudaStreamDestroy(s.st);
      cudaFree(s.d_words);
      cudaFree(s.d_m);
      cudaFree(s.d_items);
      cudaFreeHost(s.h_items);
      cudaFreeHost(s.h_m);
    }
  };
  for (auto& s : slots) {
    s.m_cap = max_items * 32;
    const int64_t item_bytes = max_items * (int64_t)sizeof(hqc::MixedItem);
    s.words_cap = (per_slot - s.m_cap - item_bytes) / 8;
    s.words_cap -= s.words_cap & 1;
    if (s.words_cap < 2) {
      cleanup();
      return sfail(HQC_ENOMEM, "budget too small for one request per stream");
    }
    if ((e = cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaHostAlloc(&s.h_items, item_bytes, cudaHostAllocMapped)) != cudaSuccess ||
        (e = cudaHostAlloc(&s.h_m, s.m_cap, cudaHostAllocMapped)) != cudaSuccess) {
      cleanup();
      return sfail(HQC_ENOMEM, "serving buffers: %s", cudaGetErrorString(e));
    }
    if (in_place) {
      void *pi = nullptr, *pm = nullptr;
      if ((e = cudaHostGetDevicePointer(&pi, s.h_items, 0)) != cudaSuccess ||
          (e = cudaHostGetDevicePointer(&pm, s.h_m, 0)) != cudaSuccess) {
        cleanup();
        return sfail(HQC_ECUDA, "mapping the serving buffers: %s", cudaGetErrorString(e));
      }
      s.k_items = static_cast<const hqc::MixedItem*>(pi);
      s.k_m = static_cast<uint8_t*>(pm);
    } else {
      if ((e = cudaMalloc(&s.d_words, s.words_cap * 8)) != cudaSuccess ||
          (e = cudaMalloc(&s.d_m, s.m_cap)) != cudaSuccess || (e = cudaMalloc(&s.d_items, item_bytes)) != cudaSuccess) {
        cleanup();
        return sfail(HQC_ENOMEM, "serving buffers: %s", cudaGetErrorString(e));
      }
      s.k_items = s.d_items;
      s.k_m = s.d_m;
    }
  }
  hqc::LaunchCfg lcfg;
  lcfg.warps_per_cta = cfg->warps_per_cta;

  // request i uses ring slot i % period
  auto rslot = [&](int64_t i) { return i % ring->period; };
  auto req_words = [&](int64_t j) { return ring->word_off[j + 1] - ring->word_off[j]; };
  auto req_m = [&](int64_t j) { return ring->m_off[j + 1] - ring->m_off[j]; };
  auto valid_req = [&](int64_t j) {
    const int li = hqc::level_index(ring->level[j]);
    if (li < 0 || !keys[li]) return false;
    if ((uint32_t)ring->key[j] >= (uint64_t)keys[li]->nkeys) return false;
    return req_words(j) == (int64_t)prm[li].W_u_pitch + prm[li].W_v && req_m(j) == prm[li].k;
  };

  int64_t arrived = 0, head = 0, done = 0, rej_queue = 0, rej_invalid = 0, rej_size = 0, batches = 0, batch_items = 0;
  // Touch every per-request output before the clock starts: on a fresh
  // (lazily mapped) array of 10^7 requests these 120 MB of first writes
  // fault in pages for tens of milliseconds, and every request arriving
  // meanwhile would wait for them.
  for (int64_t i = 0; i < count; i++) status[i] = -1, latency_ns[i] = -1;
  const int64_t t0 = now_ns();
  int64_t t_last = t0;

  std::vector<hqc::MixedItem> lists[3];
  auto fill_stats = [&]() {
    if (!stats) return;
    stats->completed = done;
    stats->rejected_queue = rej_queue;
    stats->rejected_invalid = rej_invalid;
    stats->rejected_size = rej_size;
    stats->batches = batches;
    stats->mean_batch = batches ? (double)batch_items / (double)batches : 0.0;
    stats->wall_ns = t_last - t0;
    stats->items_per_slot = max_items;
    stats->in_place = in_place ? 1 : 0;
  };
  // a batch past its limit: wait a bounded time for everything in flight,
  // free the buffers if it all finished, and report the stall
  auto stalled = [&](const Slot& late) {
    const int64_t n_late = late.last - late.first;
    const int64_t until = now_ns() + stall_ns + 1000000000;
    bool drained = true;
    for (auto& s : slots) {
      if (!s.busy) continue;
      cudaError_t q;
      while ((q = cudaEventQuery(s.ev)) == cudaErrorNotReady && now_ns() < until) std::this_thread::yield();
      if (q == cudaErrorNotReady) drained = false;
    }
    if (drained) cleanup();
    fill_stats();
    return sfail(HQC_ETIMEOUT, "a batch of %lld requests did not complete within %lld ms%s", (long long)n_late,
                 (long long)(stall_ns / 1000000), drained ? "" : "; its buffers are still held");
  };
  while (done + rej_queue + rej_invalid + rej_size < count) {
    const int64_t now = now_ns() - t0;
    // arrivals; invalid requests are answered at once, overflow is rejected
    while (arrived < count && arrival_ns[arrived] <= now) {
      const int64_t j = rslot(arrived);
      if (!valid_req(j)) {
        status[arrived] = HQC_STATUS_INVALID;
        rej_invalid++;
      } else if (arrived - head >= cfg->max_queue) {
        status[arrived] = HQC_STATUS_REJECTED;
        rej_queue++;
      } else {
        status[arrived] = HQC_STATUS_QUEUED;
      }
      arrived++;
    }
    // completions
    for (auto& s : slots) {
      if (!s.busy) continue;
      e = cudaEventQuery(s.ev);
      if (e == cudaErrorNotReady) {
        if (now_ns() - s.t_launch > stall_ns) return stalled(s);
        continue;
      }
      if (e != cudaSuccess) {
        cleanup();
        return sfail(HQC_ECUDA, "batch failed: %s", cudaGetErrorString(e));
      }
      const int64_t tc = now_ns();
      t_last = tc;
      if (s.dense) {
        // the batch's m bytes are one range of the ring's m layout
        if (m_out) std::memcpy(m_out + s.m_first, s.h_m, (size_t)s.m_bytes);
        const int64_t lat0 = tc - t0;
        for (int64_t i = s.first; i < s.last; i++) {
          latency_ns[i] = lat0 - arrival_ns[i];
          status[i] = HQC_STATUS_DONE;
        }
        done += s.last - s.first;
      } else {
        int64_t mpos = 0;
        for (int64_t i = s.first; i < s.last; i++) {
          if (status[i] != HQC_STATUS_RUNNING) continue;
          const int64_t j = rslot(i);
          const int64_t mb = req_m(j);
          if (m_out) std::memcpy(m_out + ring->m_off[j], s.h_m + mpos, (size_t)mb);
          mpos += mb;
          latency_ns[i] = tc - t0 - arrival_ns[i];
          status[i] = HQC_STATUS_DONE;
          done++;
        }
      }
      s.busy = false;
    }
    // admissions: head .. arrived, skipping requests already answered
    while (head < arrived && status[head] != HQC_STATUS_QUEUED) head++;
    for (auto& s : slots) {
      if (s.busy || head >= arrived) continue;
      // contiguous run of requests from head that fits this slot; the copy
      // range starts at the first admitted request (base)
      int64_t i = head, words = 0, mbytes = 0, n = 0, base = -1, prev = -1;
      bool dense = true;  // no request skipped between the first admitted and the last
      int64_t j_next = rslot(head);
      for (auto& l : lists) l.clear();
      while (i < arrived && n < max_items) {
        const int64_t j = j_next;
        j_next = j + 1 == ring->period ? 0 : j + 1;
        if (status[i] != HQC_STATUS_QUEUED) {
          if (n > 0) dense = false;
          i++;
          continue;
        }
        if (n > 0 && j <= prev) break;  // the ring wrapped: next batch
        const int64_t b = base >= 0 ? base : j;
        const int64_t span = ring->word_off[j + 1] - ring->word_off[b];  // ring words up to this request
        const int64_t mb = req_m(j);
        if (span > s.words_cap || mbytes + mb > s.m_cap) {
          if (n == 0) {  // a single request larger than the slot
            status[i] = HQC_STATUS_TOO_LARGE;
            rej_size++;
            i++;
            continue;
          }
          break;
        }
        base = b;
        const int li = hqc::level_index(ring->level[j]);
        hqc::MixedItem it;
        it.level = ring->level[j];
        it.key = ring->key[j];
        it.u_off = ring->word_off[j] - ring->word_off[base];
        it.v_off = it.u_off + prm[li].W_u_pitch;
        it.m_off = mbytes;
        lists[li].push_back(it);
        status[i] = HQC_STATUS_RUNNING;
        words = span;
        prev = j;
        mbytes += mb;
        n++;
        i++;
      }
      if (n == 0) {
        head = i;
        continue;
      }
      s.first = head;
      s.last = i;
      // requests before the first admitted one (already answered) are not
      // part of the range; trailing skipped ones would have cleared dense
      while (s.first < i && status[s.first] != HQC_STATUS_RUNNING) s.first++;
      s.dense = dense;
      s.m_first = ring->m_off[rslot(s.first)];
      s.m_bytes = mbytes;
      head = i;
      // the m bytes of the batch are laid out in admission order; the item
      // lists are grouped by level
      int64_t nitems = 0, start[3];
      for (int li = 0; li < 3; li++) {
        start[li] = nitems;
        std::memcpy(s.h_items + nitems, lists[li].data(), lists[li].size() * sizeof(hqc::MixedItem));
        nitems += (int64_t)lists[li].size();
      }
      const int64_t wbytes = words * 8;  // up to the last admitted request (<= words_cap)
      const uint64_t* arena = s.d_words;
      e = cudaSuccess;  // (e may still hold another slot's not-ready poll)
      if (in_place) {
        arena = ring_dev + ring->word_off[base];
      } else {
        e = cudaMemcpyAsync(s.d_words, ring->words + ring->word_off[base], (size_t)wbytes, cudaMemcpyHostToDevice,
                            s.st);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(s.d_items, s.h_items, (size_t)nitems * sizeof(hqc::MixedItem), cudaMemcpyHostToDevice,
                              s.st);
      }
      if (nitems <= kSmallBatch && e == cudaSuccess) {
        // a small batch: one launch of the latency form of the mixed kernel
        // (a team of warps per item), so its items spread over every SM and
        // the slowest one's chain is split over its team
        hqc::MixedArgs a;
        a.count = nitems;
        a.items = s.k_items;
        a.arena = arena;
        a.arena_words = wbytes / 8;
        for (int k = 0; k < 3; k++) {
          a.keys[k] = keys[k] ? keys[k]->d_table : nullptr;
          a.nkeys[k] = keys[k] ? keys[k]->nkeys : 0;
        }
        a.m = s.k_m;
        a.m_bytes = mbytes;
        e = hqc::launch_mixed_latency(a, s.st);
        for (auto& l : lists) l.clear();
      }
      for (int li = 0; li < 3 && e == cudaSuccess; li++) {
        if (lists[li].empty()) continue;
        hqc::MixedArgs a;
        a.count = (int64_t)lists[li].size();
        a.items = s.k_items + start[li];
        a.arena = arena;
        a.arena_words = wbytes / 8;
        for (int k = 0; k < 3; k++) {
          a.keys[k] = keys[k] ? keys[k]->d_table : nullptr;
          a.nkeys[k] = keys[k] ? keys[k]->nkeys : 0;
        }
        a.m = s.k_m;
        a.m_bytes = mbytes;
        e = hqc::launch_items(lv[li], a, 0, s.st, lcfg);
      }
      if (e == cudaSuccess && !in_place)
        e = cudaMemcpyAsync(s.h_m, s.d_m, (size_t)mbytes, cudaMemcpyDeviceToHost, s.st);
      if (e == cudaSuccess) e = cudaEventRecord(s.ev, s.st);
      if (e != cudaSuccess) {
        cleanup();
        return sfail(HQC_ECUDA, "batch launch: %s", cudaGetErrorString(e));
      }
      s.busy = true;
      s.t_launch = now_ns();
      batches++;
      batch_items += n;
    }
  }
  cleanup();
  fill_stats();
  return HQC_OK;
}

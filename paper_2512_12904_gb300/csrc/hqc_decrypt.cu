// The default decryption kernels and their launchers: the fused
// persistent kernels, the latency forms, the mixed-level kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <type_traits>

#include "hqc_kernels.cuh"

namespace hqc {

int level_index(int level) { return level == 1 ? 0 : level == 3 ? 1 : level == 5 ? 2 : -1; }

// Fused persistent kernel over a mixed-level item list (see mixed_item).
__global__ void __launch_bounds__(MIXED_MAX_THREADS, 1) k_decrypt_mixed(MixedArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  gf_tables_init(smem, threadIdx.x, blockDim.x);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const GF gf(smem, lane);
  uint32_t* ws = reinterpret_cast<uint32_t*>(smem + GF_TABLE_BYTES) + warp * MIXED_WARP_WORDS;
  const int64_t stride = (int64_t)gridDim.x * nw;
  int64_t it = (int64_t)blockIdx.x * nw + warp;
  if (a.counter) {
    uint32_t c = 0;
    if (lane == 0) c = atomicAdd(a.counter, 1u);
    it = (int64_t)__shfl_sync(FULL_MASK, c, 0);
  }
  while (it < a.count) {
    const MixedItem item = a.items[it];
    if (item.level == 1) mixed_item<Level<1>>(gf, ws, lane, a, item);
    else if (item.level == 3) mixed_item<Level<3>>(gf, ws, lane, a, item);
    else if (item.level == 5) mixed_item<Level<5>>(gf, ws, lane, a, item);
    if (a.counter) {
      uint32_t c = 0;
      if (lane == 0) c = atomicAdd(a.counter, 1u);
      it = (int64_t)__shfl_sync(FULL_MASK, c, 0);
    } else {
      it += stride;
    }
  }
}

// Largest batch that runs the latency form (one four-warp team per
// ciphertext) under the default launch shape.
template <int LEVEL> struct FusedLatencyMax { static constexpr int64_t count = 512; };

template <int LEVEL, bool KEYED>
static cudaError_t launch_latency(const DecArgs& a, cudaStream_t st) {
  constexpr int T = LAT_TEAM;
  constexpr size_t sm = GF_TABLE_BYTES + (size_t)Team<Level<LEVEL>, T, 1>::WORDS * 4;
  static_assert(sm <= 48 * 1024, "fits the default dynamic shared memory limit");
  const int64_t grid = a.count < MAX_LATENCY_GRID ? a.count : MAX_LATENCY_GRID;
  k_decrypt_latency<LEVEL, KEYED, T><<<(unsigned)grid, 32 * T, sm, st>>>(a);
  return cudaGetLastError();
}

// The cluster latency form (C blocks on C SMs per ciphertext) for batches
// of at most max_count: a lone ciphertext finishes sooner when its product
// and RM blocks are spread over four SMs' shared-memory bandwidth.
template <int LEVEL> struct ClusterLatency {
  static constexpr int C = 4;
  static constexpr int64_t max_count = 8;
};

template <int LEVEL, bool KEYED>
static cudaError_t launch_latency_cluster(const DecArgs& a, cudaStream_t st) {
  constexpr int C = ClusterLatency<LEVEL>::C, T = LAT_TEAM;
  constexpr size_t sm = GF_TABLE_BYTES + (size_t)ClusterShare<Level<LEVEL>, C, T>::WORDS * 4;
  // above the default 48 KB: raise the kernel's limit once per device
  static std::atomic<uint64_t> attr_done{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = 1ull << (dev & 63);
  if (!(attr_done.load() & bit)) {
    e = cudaFuncSetAttribute(k_decrypt_latency_cluster<LEVEL, KEYED, C, T>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    attr_done.fetch_or(bit);
  }
  const int64_t clusters = std::min<int64_t>(a.count, MAX_LATENCY_GRID / C);
  k_decrypt_latency_cluster<LEVEL, KEYED, C, T><<<(unsigned)(clusters * C), 32 * T, sm, st>>>(a);
  return cudaGetLastError();
}

template <int LEVEL, bool KEYED>
static cudaError_t team_level(const DecArgs& a, cudaStream_t st, const LaunchCfg& cfg, bool launch, int* warps,
                              int* ctas, int* grid) {
  int nw = 0, c = 0, g = 0;
  size_t sm = 0;
  cudaError_t e = shape_for(k_decrypt_team<LEVEL, KEYED>, TeamBound<LEVEL>::threads,
                            (size_t)Team<Level<LEVEL>>::WORDS * 2, cfg, &nw, &c, &g, &sm, true);
  if (e != cudaSuccess) return e;
  if (warps) *warps = nw;
  if (ctas) *ctas = c;
  if (grid) *grid = g;
  if (!launch || a.count == 0) return cudaSuccess;
  // less than one wave: fewer warps per block so the batch spreads over
  // every SM instead of filling a few
  if (cfg.warps_per_cta == 0 && a.count < (int64_t)g * nw) {
    const int64_t sms = g / c;
    const int want = std::max(2, ((int)((a.count + sms - 1) / sms) + 1) & ~1);
    if (want < nw) {
      LaunchCfg sc;
      sc.warps_per_cta = want;
      sc.ctas_per_sm = cfg.ctas_per_sm;
      e = shape_for(k_decrypt_team<LEVEL, KEYED>, TeamBound<LEVEL>::threads, (size_t)Team<Level<LEVEL>>::WORDS * 2,
                    sc, &nw, &c, &g, &sm, true);
      if (e != cudaSuccess) return e;
    }
  }
  const int64_t need = (a.count + nw - 1) / nw;  // nw / 2 teams, two ciphertexts each
  if (need < g) g = (int)need;
  k_decrypt_team<LEVEL, KEYED><<<g, nw * 32, sm, st>>>(a);
  return cudaGetLastError();
}

template <int LEVEL, bool KEYED>
static cudaError_t fused_level(const DecArgs& a, cudaStream_t st, const LaunchCfg& cfg, bool launch, int* warps,
                               int* ctas, int* grid) {
  // a small batch with the default shape: a team of warps per ciphertext
  if (launch && a.count > 0 && cfg.warps_per_cta == 0 && cfg.ctas_per_sm == 0 &&
      a.count <= FusedLatencyMax<LEVEL>::count)
    return a.count <= ClusterLatency<LEVEL>::max_count ? launch_latency_cluster<LEVEL, KEYED>(a, st)
                                                       : launch_latency<LEVEL, KEYED>(a, st);
  if (UseTeam<LEVEL>::value) return team_level<LEVEL, KEYED>(a, st, cfg, launch, warps, ctas, grid);
  int nw = 0, c = 0, g = 0;
  size_t sm = 0;
  cudaError_t e = shape_for(k_decrypt_fused<LEVEL, KEYED>, FusedBound<LEVEL>::threads,
                            (size_t)fused_words<LEVEL>() * 4, cfg, &nw, &c, &g, &sm, false, fused_fixed_bytes<LEVEL>());
  if (e != cudaSuccess) return e;
  if (warps) *warps = nw;
  if (ctas) *ctas = c;
  if (grid) *grid = g;
  if (!launch || a.count == 0) return cudaSuccess;
  constexpr int G = FusedGroup<LEVEL>::G;
  // at most one group per warp even when spread over every SM: one
  // ciphertext per warp (G = 1) halves each warp's serial chain
  if (G > 1 && cfg.warps_per_cta == 0 && a.count <= (int64_t)(g / c) * nw) {
    const int64_t sms = g / c;
    LaunchCfg sc;
    sc.warps_per_cta = (int)((a.count + sms - 1) / sms);
    e = shape_for(k_decrypt_fused<LEVEL, KEYED, 1>, FusedBound<LEVEL>::threads,
                  (size_t)fused_warp_words<Level<LEVEL>, 1>() * 4, sc, &nw, &c, &g, &sm, false,
                  fused_fixed_bytes<LEVEL>());
    if (e != cudaSuccess) return e;
    const int64_t need1 = (a.count + nw - 1) / nw;
    if (need1 < g) g = (int)need1;
    k_decrypt_fused<LEVEL, KEYED, 1><<<g, nw * 32, sm, st>>>(a);
    return cudaGetLastError();
  }
  // less than one wave: fewer warps per block so the batch spreads over
  // every SM instead of filling a few
  if (cfg.warps_per_cta == 0 && a.count < (int64_t)g * nw * G) {
    const int64_t sms = g / c;
    const int want = std::max(1, (int)((a.count + sms * G - 1) / (sms * G)));
    if (want < nw) {
      LaunchCfg sc;
      sc.warps_per_cta = want;
      sc.ctas_per_sm = cfg.ctas_per_sm;
      e = shape_for(k_decrypt_fused<LEVEL, KEYED>, FusedBound<LEVEL>::threads, (size_t)fused_words<LEVEL>() * 4, sc,
                    &nw, &c, &g, &sm, false, fused_fixed_bytes<LEVEL>());
      if (e != cudaSuccess) return e;
    }
  }
  const int64_t need = (a.count + (int64_t)nw * G - 1) / ((int64_t)nw * G);
  if (need < g) g = (int)need;
  k_decrypt_fused<LEVEL, KEYED><<<g, nw * 32, sm, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_fused(int level, bool keyed, const DecArgs& a, cudaStream_t st, const LaunchCfg& cfg) {
  switch (level) {
    case 1: return keyed ? fused_level<1, true>(a, st, cfg, true, 0, 0, 0) : fused_level<1, false>(a, st, cfg, true, 0, 0, 0);
    case 3: return keyed ? fused_level<3, true>(a, st, cfg, true, 0, 0, 0) : fused_level<3, false>(a, st, cfg, true, 0, 0, 0);
    case 5: return keyed ? fused_level<5, true>(a, st, cfg, true, 0, 0, 0) : fused_level<5, false>(a, st, cfg, true, 0, 0, 0);
  }
  return cudaErrorInvalidValue;
}

cudaError_t fused_wave(int level, bool keyed, const LaunchCfg& cfg, int64_t* items) {
  int w = 0, c = 0, g = 0;
  cudaError_t e = fused_occupancy(level, keyed, cfg, &w, &c, &g);
  if (e != cudaSuccess) return e;
  // ciphertexts per two warps: one for a team, 2G for single-warp groups
  auto per2 = [](auto lv) {
    constexpr int L = decltype(lv)::value;
    return UseTeam<L>::value ? 1 : 2 * FusedGroup<L>::G;
  };
  const int64_t per_two = level == 1   ? per2(std::integral_constant<int, 1>{})
                          : level == 3 ? per2(std::integral_constant<int, 3>{})
                                       : per2(std::integral_constant<int, 5>{});
  *items = (int64_t)g * w * per_two / 2;
  return cudaSuccess;
}

cudaError_t fused_occupancy(int level, bool keyed, const LaunchCfg& cfg, int* warps, int* ctas, int* grid) {
  DecArgs none;
  switch (level) {
    case 1: return keyed ? fused_level<1, true>(none, 0, cfg, false, warps, ctas, grid) : fused_level<1, false>(none, 0, cfg, false, warps, ctas, grid);
    case 3: return keyed ? fused_level<3, true>(none, 0, cfg, false, warps, ctas, grid) : fused_level<3, false>(none, 0, cfg, false, warps, ctas, grid);
    case 5: return keyed ? fused_level<5, true>(none, 0, cfg, false, warps, ctas, grid) : fused_level<5, false>(none, 0, cfg, false, warps, ctas, grid);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_mixed(const MixedArgs& a, cudaStream_t st, const LaunchCfg& cfg) {
  int nw = 0, c = 0, g = 0;
  size_t sm = 0;
  cudaError_t e = shape_for(k_decrypt_mixed, MIXED_MAX_THREADS, (size_t)MIXED_WARP_WORDS * 4, cfg, &nw, &c, &g, &sm);
  if (e != cudaSuccess) return e;
  if (a.count == 0) return cudaSuccess;
  const int64_t need = (a.count + nw - 1) / nw;
  if (need < g) g = (int)need;
  k_decrypt_mixed<<<g, nw * 32, sm, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_mixed_latency(const MixedArgs& a, cudaStream_t st) {
  if (a.count == 0) return cudaSuccess;
  if (a.count > MIXED_LATENCY_MAX) return cudaErrorInvalidValue;
  constexpr int T = LAT_TEAM;
  constexpr size_t sm = GF_TABLE_BYTES + (size_t)lat_team_words<T>() * 4;
  static_assert(sm <= 48 * 1024, "fits the default dynamic shared memory limit");
  k_decrypt_mixed_team<T><<<(unsigned)a.count, 32 * T, sm, st>>>(a);
  return cudaGetLastError();
}

template <int LEVEL>
static cudaError_t items_team_level(const MixedArgs& a, int grid, cudaStream_t st, const LaunchCfg& cfg, bool launch,
                                    int* warps, int* ctas, int* full_grid) {
  int nw = 0, c = 0, g = 0;
  size_t sm = 0;
  LaunchCfg tc = cfg;  // teams need an even warp count
  if (tc.warps_per_cta > 0) tc.warps_per_cta = std::max(2, tc.warps_per_cta & ~1);
  cudaError_t e = shape_for(k_decrypt_items_team<LEVEL>, TeamBound<LEVEL>::threads,
                            (size_t)Team<Level<LEVEL>>::WORDS * 2, tc, &nw, &c, &g, &sm, true);
  if (e != cudaSuccess) return e;
  if (warps) *warps = nw;
  if (ctas) *ctas = c;
  if (full_grid) *full_grid = g;
  if (!launch || a.count == 0) return cudaSuccess;
  // a full grid for less than one wave: fewer warps per block so the items
  // spread over every SM
  if (grid <= 0 && tc.warps_per_cta == 0 && a.count < (int64_t)g * nw) {
    const int64_t sms = g / c;
    const int small = std::max(2, ((int)((a.count + sms - 1) / sms) + 1) & ~1);
    if (small < nw) {
      LaunchCfg sc;
      sc.warps_per_cta = small;
      e = shape_for(k_decrypt_items_team<LEVEL>, TeamBound<LEVEL>::threads, (size_t)Team<Level<LEVEL>>::WORDS * 2,
                    sc, &nw, &c, &g, &sm, true);
      if (e != cudaSuccess) return e;
    }
  }
  if (grid <= 0 || grid > g) grid = g;
  const int64_t need = (a.count + nw - 1) / nw;
  if (need < grid) grid = (int)need;
  k_decrypt_items_team<LEVEL><<<grid, nw * 32, sm, st>>>(a);
  return cudaGetLastError();
}

template <int LEVEL>
static cudaError_t items_level(const MixedArgs& a, int grid, cudaStream_t st, const LaunchCfg& cfg, bool launch,
                               int* warps, int* ctas, int* full_grid) {
  if (UseTeam<LEVEL>::value) return items_team_level<LEVEL>(a, grid, st, cfg, launch, warps, ctas, full_grid);
  int nw = 0, c = 0, g = 0;
  size_t sm = 0;
  cudaError_t e = shape_for(k_decrypt_items<LEVEL>, FusedBound<LEVEL>::threads, (size_t)fused_words<LEVEL>() * 4,
                            cfg, &nw, &c, &g, &sm, false, fused_fixed_bytes<LEVEL>());
  if (e != cudaSuccess) return e;
  if (warps) *warps = nw;
  if (ctas) *ctas = c;
  if (full_grid) *full_grid = g;
  if (!launch || a.count == 0) return cudaSuccess;
  constexpr int G = FusedGroup<LEVEL>::G;
  // a full grid for less than one wave: fewer warps per block so the items
  // spread over every SM
  if (grid <= 0 && cfg.warps_per_cta == 0 && a.count < (int64_t)g * nw * G) {
    const int64_t sms = g / c;
    const int small = std::max(1, (int)((a.count + sms * G - 1) / (sms * G)));
    if (small < nw) {
      LaunchCfg sc;
      sc.warps_per_cta = small;
      e = shape_for(k_decrypt_items<LEVEL>, FusedBound<LEVEL>::threads, (size_t)fused_words<LEVEL>() * 4, sc, &nw, &c,
                    &g, &sm, false, fused_fixed_bytes<LEVEL>());
      if (e != cudaSuccess) return e;
    }
  }
  if (grid <= 0 || grid > g) grid = g;
  const int64_t need = (a.count + (int64_t)nw * G - 1) / ((int64_t)nw * G);
  if (need < grid) grid = (int)need;
  k_decrypt_items<LEVEL><<<grid, nw * 32, sm, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_items(int level, const MixedArgs& a, int grid, cudaStream_t st, const LaunchCfg& cfg) {
  switch (level) {
    case 1: return items_level<1>(a, grid, st, cfg, true, 0, 0, 0);
    case 3: return items_level<3>(a, grid, st, cfg, true, 0, 0, 0);
    case 5: return items_level<5>(a, grid, st, cfg, true, 0, 0, 0);
  }
  return cudaErrorInvalidValue;
}

cudaError_t items_occupancy(int level, const LaunchCfg& cfg, int* warps, int* ctas, int* grid) {
  MixedArgs none;
  switch (level) {
    case 1: return items_level<1>(none, 0, 0, cfg, false, warps, ctas, grid);
    case 3: return items_level<3>(none, 0, 0, cfg, false, warps, ctas, grid);
    case 5: return items_level<5>(none, 0, 0, cfg, false, warps, ctas, grid);
  }
  return cudaErrorInvalidValue;
}

cudaError_t mixed_occupancy(const LaunchCfg& cfg, int* warps, int* ctas, int* grid) {
  int nw = 0, c = 0, g = 0;
  size_t sm = 0;
  cudaError_t e = shape_for(k_decrypt_mixed, MIXED_MAX_THREADS, (size_t)MIXED_WARP_WORDS * 4, cfg, &nw, &c, &g, &sm);
  if (warps) *warps = nw;
  if (ctas) *ctas = c;
  if (grid) *grid = g;
  return e;
}

}  // namespace hqc

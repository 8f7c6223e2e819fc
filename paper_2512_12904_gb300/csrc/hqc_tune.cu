// Kernel variants that the plans' autotuner times on the caller's data
// (hqc_plan.cu), beside the library's default kernels:
//   * solo warps taking G = 1, 2 or 4 ciphertexts per turn (their RS stages
//     side by side on 32 / G lanes each), for the keyed batch and for one
//     level of a partitioned mixed list;
//   * two-warp teams sharing one doubled operand, at every level;
//   * one launch for a whole partitioned mixed list whose blocks take a
//     level by block range (k_decrypt_mixed_ranges), each level with its
//     own warp count and shared-memory layout inside a common block size.
// All of them compute exactly what the default kernels compute; only the
// mapping of ciphertexts to warps and the launch shape differ.
#include <cuda_runtime.h>

#include <algorithm>

#include "hqc_kernels.cuh"

namespace hqc {

namespace {

// Solo-warp keyed kernel with G ciphertexts per turn, no sub-wave or
// small-batch adjustments: the tuner explores the shapes itself.
template <int LEVEL, int G>
cudaError_t solo_keyed(const DecArgs& a, cudaStream_t st, const LaunchCfg& cfg, bool launch, int* w, int* c, int* g) {
  int nw = 0, cc = 0, gg = 0;
  size_t sm = 0;
  cudaError_t e = shape_for(k_decrypt_fused<LEVEL, true, G>, FusedBound<LEVEL>::threads,
                            (size_t)fused_warp_words<Level<LEVEL>, G>() * 4, cfg, &nw, &cc, &gg, &sm, false,
                            fused_fixed_bytes<LEVEL>());
  if (e != cudaSuccess) return e;
  if (w) *w = nw;
  if (c) *c = cc;
  if (g) *g = gg;
  if (!launch || a.count == 0) return cudaSuccess;
  const int64_t need = (a.count + (int64_t)nw * G - 1) / ((int64_t)nw * G);
  k_decrypt_fused<LEVEL, true, G><<<(unsigned)std::min<int64_t>(need, gg), nw * 32, sm, st>>>(a);
  return cudaGetLastError();
}

template <int LEVEL>
cudaError_t team_keyed(const DecArgs& a, cudaStream_t st, const LaunchCfg& cfg, bool launch, int* w, int* c, int* g) {
  int nw = 0, cc = 0, gg = 0;
  size_t sm = 0;
  LaunchCfg tc = cfg;  // teams need an even warp count
  if (tc.warps_per_cta > 0) tc.warps_per_cta = std::max(2, tc.warps_per_cta & ~1);
  cudaError_t e = shape_for(k_decrypt_team<LEVEL, true>, TeamBound<LEVEL>::threads,
                            (size_t)Team<Level<LEVEL>>::WORDS * 2, tc, &nw, &cc, &gg, &sm, true);
  if (e != cudaSuccess) return e;
  if (w) *w = nw;
  if (c) *c = cc;
  if (g) *g = gg;
  if (!launch || a.count == 0) return cudaSuccess;
  const int64_t need = (a.count + nw - 1) / nw;  // nw / 2 teams, two ciphertexts each
  k_decrypt_team<LEVEL, true><<<(unsigned)std::min<int64_t>(need, gg), nw * 32, sm, st>>>(a);
  return cudaGetLastError();
}

// One level of a partitioned mixed list; grid <= 0 = a full persistent grid.
template <int LEVEL, int G>
cudaError_t solo_items(const MixedArgs& a, int grid, cudaStream_t st, const LaunchCfg& cfg, bool launch, int* w,
                       int* c, int* g) {
  int nw = 0, cc = 0, gg = 0;
  size_t sm = 0;
  cudaError_t e = shape_for(k_decrypt_items<LEVEL, G>, FusedBound<LEVEL>::threads,
                            (size_t)fused_warp_words<Level<LEVEL>, G>() * 4, cfg, &nw, &cc, &gg, &sm, false,
                            fused_fixed_bytes<LEVEL>());
  if (e != cudaSuccess) return e;
  if (w) *w = nw;
  if (c) *c = cc;
  if (g) *g = gg;
  if (!launch || a.count == 0) return cudaSuccess;
  if (grid <= 0 || grid > gg) grid = gg;
  const int64_t need = (a.count + (int64_t)nw * G - 1) / ((int64_t)nw * G);
  k_decrypt_items<LEVEL, G><<<(unsigned)std::min<int64_t>(need, grid), nw * 32, sm, st>>>(a);
  return cudaGetLastError();
}

template <int LEVEL>
cudaError_t team_items(const MixedArgs& a, int grid, cudaStream_t st, const LaunchCfg& cfg, bool launch, int* w,
                       int* c, int* g) {
  int nw = 0, cc = 0, gg = 0;
  size_t sm = 0;
  LaunchCfg tc = cfg;
  if (tc.warps_per_cta > 0) tc.warps_per_cta = std::max(2, tc.warps_per_cta & ~1);
  cudaError_t e = shape_for(k_decrypt_items_team<LEVEL>, TeamBound<LEVEL>::threads,
                            (size_t)Team<Level<LEVEL>>::WORDS * 2, tc, &nw, &cc, &gg, &sm, true);
  if (e != cudaSuccess) return e;
  if (w) *w = nw;
  if (c) *c = cc;
  if (g) *g = gg;
  if (!launch || a.count == 0) return cudaSuccess;
  if (grid <= 0 || grid > gg) grid = gg;
  const int64_t need = (a.count + nw - 1) / nw;
  k_decrypt_items_team<LEVEL><<<(unsigned)std::min<int64_t>(need, grid), nw * 32, sm, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

bool variant_exists(int level, int variant) {
  switch (variant) {
    case VAR_DEFAULT: return level_index(level) >= 0;
    case VAR_SOLO1:
    case VAR_SOLO2:
    case VAR_TEAM: return level_index(level) >= 0;
    case VAR_SOLO4: return level == 1 || level == 3;
  }
  return false;
}

const char* variant_name(int variant) {
  switch (variant) {
    case VAR_DEFAULT: return "default";
    case VAR_SOLO1: return "solo-G1";
    case VAR_SOLO2: return "solo-G2";
    case VAR_SOLO4: return "solo-G4";
    case VAR_TEAM: return "team2";
  }
  return "?";
}

template <int LEVEL>
static cudaError_t keyed_variant(int variant, const DecArgs& a, cudaStream_t st, const LaunchCfg& cfg, bool launch,
                                 int* w, int* c, int* g) {
  switch (variant) {
    case VAR_SOLO1: return solo_keyed<LEVEL, 1>(a, st, cfg, launch, w, c, g);
    case VAR_SOLO2: return solo_keyed<LEVEL, 2>(a, st, cfg, launch, w, c, g);
    case VAR_SOLO4:
      if constexpr (LEVEL != 5) return solo_keyed<LEVEL, 4>(a, st, cfg, launch, w, c, g);
      break;
    case VAR_TEAM: return team_keyed<LEVEL>(a, st, cfg, launch, w, c, g);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_fused_variant(int level, int variant, const DecArgs& a, cudaStream_t st, const LaunchCfg& cfg) {
  if (variant == VAR_DEFAULT) return launch_fused(level, true, a, st, cfg);
  switch (level) {
    case 1: return keyed_variant<1>(variant, a, st, cfg, true, 0, 0, 0);
    case 3: return keyed_variant<3>(variant, a, st, cfg, true, 0, 0, 0);
    case 5: return keyed_variant<5>(variant, a, st, cfg, true, 0, 0, 0);
  }
  return cudaErrorInvalidValue;
}

template <int LEVEL>
static cudaError_t items_variant(int variant, const MixedArgs& a, int grid, cudaStream_t st, const LaunchCfg& cfg,
                                 bool launch, int* w, int* c, int* g) {
  switch (variant) {
    case VAR_SOLO1: return solo_items<LEVEL, 1>(a, grid, st, cfg, launch, w, c, g);
    case VAR_SOLO2: return solo_items<LEVEL, 2>(a, grid, st, cfg, launch, w, c, g);
    case VAR_SOLO4:
      if constexpr (LEVEL != 5) return solo_items<LEVEL, 4>(a, grid, st, cfg, launch, w, c, g);
      break;
    case VAR_TEAM: return team_items<LEVEL>(a, grid, st, cfg, launch, w, c, g);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_items_variant(int level, int variant, const MixedArgs& a, int grid, cudaStream_t st,
                                 const LaunchCfg& cfg) {
  if (variant == VAR_DEFAULT) return launch_items(level, a, grid, st, cfg);
  switch (level) {
    case 1: return items_variant<1>(variant, a, grid, st, cfg, true, 0, 0, 0);
    case 3: return items_variant<3>(variant, a, grid, st, cfg, true, 0, 0, 0);
    case 5: return items_variant<5>(variant, a, grid, st, cfg, true, 0, 0, 0);
  }
  return cudaErrorInvalidValue;
}

cudaError_t items_variant_occupancy(int level, int variant, const LaunchCfg& cfg, int* warps, int* ctas, int* grid) {
  if (variant == VAR_DEFAULT) return items_occupancy(level, cfg, warps, ctas, grid);
  MixedArgs none;
  switch (level) {
    case 1: return items_variant<1>(variant, none, 0, 0, cfg, false, warps, ctas, grid);
    case 3: return items_variant<3>(variant, none, 0, 0, cfg, false, warps, ctas, grid);
    case 5: return items_variant<5>(variant, none, 0, 0, cfg, false, warps, ctas, grid);
  }
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// One launch over a level-partitioned mixed list: blocks [0, grid[0]) take
// the HQC-1 items, the next grid[1] blocks the HQC-3 items and the last
// grid[2] the HQC-5 items.  A block runs warps[level] of its RANGE_THREADS
// / 32 warps (the others leave at once) with that level's shared-memory
// layout: solo warps with two ciphertexts per turn (HQC-1) or one (HQC-3),
// two-warp teams (HQC-5).  The block size and the register budget are the
// launch's, common to all three levels.
// ---------------------------------------------------------------------------
namespace {

struct RangeArgs {
  MixedArgs part[3];
  int32_t grid[3];
  int32_t warps[3];
};

constexpr int RANGE_THREADS = 768;
constexpr size_t RANGE_PER_WARP[3] = {(size_t)fused_warp_words<Level<1>, 2>() * 4,
                                      (size_t)fused_warp_words<Level<3>, 1>() * 4,
                                      (size_t)Team<Level<5>>::WORDS * 2};

__global__ void __launch_bounds__(RANGE_THREADS, 1) k_decrypt_mixed_ranges(RangeArgs r) {
  extern __shared__ __align__(16) uint8_t smem[];
  gf_tables_init(smem, threadIdx.x, blockDim.x);
  __syncthreads();
  const int64_t b = blockIdx.x;
  const int warp = threadIdx.x >> 5;
  if (b < r.grid[0]) {
    if (warp < r.warps[0]) items_solo<1, 2>(r.part[0], smem, b, r.grid[0], warp, r.warps[0]);
  } else if (b < (int64_t)r.grid[0] + r.grid[1]) {
    if (warp < r.warps[1]) items_solo<3, 1>(r.part[1], smem, b - r.grid[0], r.grid[1], warp, r.warps[1]);
  } else {
    if (warp < r.warps[2]) items_team<5>(r.part[2], smem, b - r.grid[0] - r.grid[1], r.grid[2], warp, r.warps[2]);
  }
}

}  // namespace

cudaError_t launch_mixed_ranges(const MixedArgs part[3], const int grid[3], cudaStream_t st) {
  int sms = 0, optin = 0;
  device_props(&sms, &optin);
  RangeArgs r;
  size_t smem = GF_TABLE_BYTES;
  int64_t total = 0;
  for (int li = 0; li < 3; li++) {
    r.part[li] = part[li];
    int nw = (int)std::min<size_t>(RANGE_THREADS / 32, (size_t)(optin - GF_TABLE_BYTES) / RANGE_PER_WARP[li]);
    if (li == 2) nw = std::min(nw & ~1, 30);  // teams: an even count, 15 named barriers
    if (nw < (li == 2 ? 2 : 1)) return cudaErrorInvalidConfiguration;
    r.warps[li] = nw;
    r.grid[li] = part[li].count > 0 ? std::max(0, grid[li]) : 0;
    if (part[li].count > 0 && r.grid[li] == 0) return cudaErrorInvalidValue;
    if (r.grid[li] > 0) smem = std::max(smem, GF_TABLE_BYTES + (size_t)nw * RANGE_PER_WARP[li]);
    total += r.grid[li];
  }
  if (total == 0) return cudaSuccess;
  if (total > 65535) return cudaErrorInvalidValue;
  {
    std::lock_guard<std::mutex> lock(g_shape_mu);
    static size_t attr = 0;
    if (smem > attr) {
      cudaError_t e = cudaFuncSetAttribute(k_decrypt_mixed_ranges, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
      if (e != cudaSuccess) return e;
      attr = smem;
    }
  }
  k_decrypt_mixed_ranges<<<(unsigned)total, RANGE_THREADS, smem, st>>>(r);
  return cudaGetLastError();
}

}  // namespace hqc

// Decryption kernel templates for sm_103a, shared by the translation
// units that instantiate them (the default kernels, the per-stage form,
// the autotuner's variants), and the launch-shape helper they all use.
//   * k_decrypt_fused  -- persistent kernel, G ciphertexts per warp per
//     turn, S1-S9 fused with every intermediate in shared memory/registers;
//   * k_decrypt_team   -- the same with two-warp teams sharing one operand;
//   * k_decrypt_latency / k_decrypt_mixed_team -- a four-warp team per
//     ciphertext (small batches);
//   * k_decrypt_items  -- persistent kernels over one level of a mixed list;
//   * k_stage_*        -- the plain one-kernel-per-stage form (product, RM,
//     RS) with intermediates in global memory, also used by the debug path
//     that dumps every intermediate.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>

#include "hqc_device.cuh"
#include "hqc_internal.h"

namespace hqc {


// Largest block of the persistent kernels per level.  Shared memory caps
// the warps per SM at about 40 / 20 / 13 for HQC-1 / 3 / 5; the bound lets
// the compiler spend the rest of the register file on each warp.
template <int LEVEL> struct FusedBound;
template <> struct FusedBound<1> { static constexpr int threads = 1024; };
template <> struct FusedBound<3> { static constexpr int threads = 640; };
template <> struct FusedBound<5> { static constexpr int threads = 416; };
constexpr int MIXED_MAX_THREADS = 416;

// Ciphertexts a warp takes per turn: their Reed-Solomon stages run side by
// side on 32 / G lanes each.  Measured on GB300 (G = 1, 2, 4): two per turn
// pays for HQC-1 (+6 %), one is best for HQC-3 and HQC-5.
template <int LEVEL> struct FusedGroup { static constexpr int G = 1; };
template <> struct FusedGroup<1> { static constexpr int G = 2; };

template <int LEVEL>
__host__ __device__ constexpr int fused_words() { return fused_warp_words<Level<LEVEL>, FusedGroup<LEVEL>::G>(); }

// Levels whose fused kernels compute the syndromes by Horner's rule on the
// block's syndrome table (rs_syndromes_horner): 16 KB more shared memory
// per block.  HQC-1 has the room (its warps are capped by the 1,024-thread
// block, not by shared memory); HQC-3 would lose two of its 20 warps, and
// HQC-5's 58 syndromes need two table columns per lane.
template <int LEVEL> struct FusedSyn { static constexpr bool on = LEVEL == 1; };

// Shared bytes of a fused block before the warps' slices.
template <int LEVEL>
__host__ __device__ constexpr int fused_fixed_bytes() {
  return GF_TABLE_BYTES + (FusedSyn<LEVEL>::on ? SYN_TABLE_BYTES : 0);
}

// ---------------------------------------------------------------------------
// Fused persistent kernel, one level.  Warp w takes groups of G consecutive
// ciphertexts w, w + (all warps), ...
// ---------------------------------------------------------------------------
template <int LEVEL, bool KEYED, int G = FusedGroup<LEVEL>::G>
__global__ void __launch_bounds__(FusedBound<LEVEL>::threads, 1) k_decrypt_fused(DecArgs a) {
  using LV = Level<LEVEL>;
  constexpr bool SYN = FusedSyn<LEVEL>::on;
  extern __shared__ __align__(16) uint8_t smem[];
  gf_tables_init(smem, threadIdx.x, blockDim.x);
  if constexpr (SYN) syn_table_init(smem + GF_TABLE_BYTES, threadIdx.x, blockDim.x);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const GF gf(smem, lane);
  uint32_t* ws = reinterpret_cast<uint32_t*>(smem + fused_fixed_bytes<LEVEL>()) + warp * fused_warp_words<LV, G>();
  const int64_t ngroups = (a.count + G - 1) / G;
  for (int64_t q = (int64_t)blockIdx.x * nw + warp; q < ngroups; q += (int64_t)gridDim.x * nw) {
    auto rows = [&](int g, const uint64_t*& u, const uint64_t*& v, const uint32_t*& y, uint8_t*& m) {
      const int64_t it0 = q * G + g;
      bool ok = it0 < a.count;
      const int64_t it = ok ? it0 : q * G;
      if (KEYED) {
        // an index outside [0, nkeys) skips the item: m stays untouched
        const uint32_t ki = (uint32_t)__ldg(a.key_idx + it);
        const bool kok = ki < (uint64_t)a.nkeys;
        y = a.y + (kok ? (int64_t)ki : 0) * LV::w;
        ok = ok && kok;
      } else {
        y = a.y + it * LV::w;
      }
      u = a.u + it * LV::W_u_pitch;
      v = a.v + it * LV::W_v;
      m = a.m + it * LV::k;
      return ok;
    };
    decrypt_group<LV, G, !KEYED, SYN>(gf, ws, lane, rows, smem + GF_TABLE_BYTES);
  }
}

// ---------------------------------------------------------------------------
// Fused persistent kernel with two-warp teams (HQC-3 and HQC-5): team t of
// the grid takes pairs of consecutive ciphertexts t, t + (all teams), ...
// At most 15 teams per block (named barriers 1..15).
// ---------------------------------------------------------------------------
template <int LEVEL> struct TeamBound;
template <> struct TeamBound<1> { static constexpr int threads = 960; };
template <> struct TeamBound<3> { static constexpr int threads = 960; };
template <> struct TeamBound<5> { static constexpr int threads = 768; };
// Levels that use the team kernels.  Measured on GB300: HQC-5 gains 26 %
// (24 warps per SM instead of 13); HQC-3 loses 17 % (its half strips waste
// 8.6 % of the product and 20 solo warps already hide enough latency).
template <int LEVEL> struct UseTeam { static constexpr bool value = LEVEL == 5; };

template <int LEVEL, bool KEYED>
__global__ void __launch_bounds__(TeamBound<LEVEL>::threads, 1) k_decrypt_team(DecArgs a) {
  using LV = Level<LEVEL>;
  extern __shared__ __align__(16) uint8_t smem[];
  gf_tables_init(smem, threadIdx.x, blockDim.x);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int team = warp >> 1, wt = warp & 1, nteams = blockDim.x >> 6;
  const GF gf(smem, lane);
  uint32_t* ws = reinterpret_cast<uint32_t*>(smem + GF_TABLE_BYTES) + team * Team<LV>::WORDS;
  const TeamSync sync{(uint32_t)(1 + team)};
  const int64_t ngroups = (a.count + 1) / 2;
  for (int64_t q = (int64_t)blockIdx.x * nteams + team; q < ngroups; q += (int64_t)gridDim.x * nteams) {
    auto rows = [&](int g, const uint64_t*& u, const uint64_t*& v, const uint32_t*& y, uint8_t*& m) {
      const int64_t it0 = 2 * q + g;
      bool ok = it0 < a.count;
      const int64_t it = ok ? it0 : 2 * q;
      if (KEYED) {
        // an index outside [0, nkeys) skips the item: m stays untouched
        const uint32_t ki = (uint32_t)__ldg(a.key_idx + it);
        const bool kok = ki < (uint64_t)a.nkeys;
        y = a.y + (kok ? (int64_t)ki : 0) * LV::w;
        ok = ok && kok;
      } else {
        y = a.y + it * LV::w;
      }
      u = a.u + it * LV::W_u_pitch;
      v = a.v + it * LV::W_v;
      m = a.m + it * LV::k;
      return ok;
    };
    decrypt_team<LV, !KEYED>(gf, ws, wt, lane, sync, rows);
  }
}

// ---------------------------------------------------------------------------
// Fused persistent kernel over a mixed-level item list.  Each warp claims
// the next item from a.counter (or walks a static stride when no counter is
// given); shared memory per warp is sized for HQC-5.  Items whose level,
// key or offsets fall outside the given arrays are skipped.
// ---------------------------------------------------------------------------
constexpr int MIXED_WARP_WORDS =
    cmax(fused_warp_words<Level<1>, 1>(), cmax(fused_warp_words<Level<3>, 1>(), fused_warp_words<Level<5>, 1>()));

template <class LV>
__device__ __forceinline__ void mixed_item(const GF& gf, uint32_t* ws, int lane, const MixedArgs& a,
                                           const MixedItem& it) {
  const int li = LV::level == 1 ? 0 : LV::level == 3 ? 1 : 2;
  const bool ok = (uint32_t)it.key < (uint64_t)a.nkeys[li] && it.u_off >= 0 && (it.u_off & 1) == 0 &&
                  it.u_off + LV::W_u_pitch <= a.arena_words && it.v_off >= 0 &&
                  it.v_off + LV::W_v <= a.arena_words && it.m_off >= 0 && it.m_off + LV::k <= a.m_bytes;
  if (!ok) return;
  decrypt_one<LV, false>(gf, ws, lane, a.arena + it.u_off, a.arena + it.v_off, a.keys[li] + (int64_t)it.key * LV::w,
                         a.m + it.m_off);
}


// ---------------------------------------------------------------------------
// Latency form of the mixed kernel: a team of LAT_TEAM warps decodes one
// item of any level at a time, splitting the product strips and the RM
// blocks over the team; the first warp runs the Reed-Solomon stage.  One
// team per block, so a small batch spreads over every SM.  In a batch that
// fits one wave the slowest item sets the time, and its chain is shorter.
// ---------------------------------------------------------------------------
constexpr int LAT_TEAM = 4;
constexpr int64_t MAX_LATENCY_GRID = 65535;
template <int T>
__host__ __device__ constexpr int lat_team_words() {
  return cmax(Team<Level<1>, T, 1>::WORDS, cmax(Team<Level<3>, T, 1>::WORDS, Team<Level<5>, T, 1>::WORDS));
}

template <class LV, int T>
__device__ __forceinline__ void mixed_item_team(const GF& gf, uint32_t* ws, int wt, int lane, const TeamSync& sync,
                                                const MixedArgs& a, const MixedItem& it) {
  const int li = LV::level == 1 ? 0 : LV::level == 3 ? 1 : 2;
  const bool ok = (uint32_t)it.key < (uint64_t)a.nkeys[li] && it.u_off >= 0 && (it.u_off & 1) == 0 &&
                  it.u_off + LV::W_u_pitch <= a.arena_words && it.v_off >= 0 &&
                  it.v_off + LV::W_v <= a.arena_words && it.m_off >= 0 && it.m_off + LV::k <= a.m_bytes;
  if (!ok) return;  // the same item for the whole team: all its warps leave together
  auto rows = [&](int g, const uint64_t*& u, const uint64_t*& v, const uint32_t*& y, uint8_t*& m) {
    u = a.arena + it.u_off;
    v = a.arena + it.v_off;
    y = a.keys[li] + (int64_t)it.key * LV::w;
    m = a.m + it.m_off;
    return g == 0;
  };
  decrypt_team<LV, false, T, 1>(gf, ws, wt, lane, sync, rows);
}

template <int T>
__global__ void __launch_bounds__(32 * T, 4) k_decrypt_mixed_team(MixedArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  gf_tables_init(smem, threadIdx.x, blockDim.x);
  __syncthreads();
  const int lane = threadIdx.x & 31, wt = threadIdx.x >> 5;
  const GF gf(smem, lane);
  uint32_t* ws = reinterpret_cast<uint32_t*>(smem + GF_TABLE_BYTES);
  const TeamSync sync{1u, 32u * T};
  for (int64_t it = blockIdx.x; it < a.count; it += gridDim.x) {
    const MixedItem item = a.items[it];
    if (item.level == 1) mixed_item_team<Level<1>, T>(gf, ws, wt, lane, sync, a, item);
    else if (item.level == 3) mixed_item_team<Level<3>, T>(gf, ws, wt, lane, sync, a, item);
    else if (item.level == 5) mixed_item_team<Level<5>, T>(gf, ws, wt, lane, sync, a, item);
  }
}

// The same latency form for a batch of one level (literal or keyed
// supports): block b decodes ciphertexts b, b + grid, ... with its team.
// after(it, ws) runs once per item, after its decryption, on the whole
// block: the kernel passes a no-op; the debug path reads the team's RM
// bytes and RS intermediates back from shared memory there.
template <int LEVEL, bool KEYED, int T, class After>
__device__ __forceinline__ void latency_items(const DecArgs& a, uint8_t* smem, const After& after) {
  using LV = Level<LEVEL>;
  gf_tables_init(smem, threadIdx.x, blockDim.x);
  __syncthreads();
  const int lane = threadIdx.x & 31, wt = threadIdx.x >> 5;
  const GF gf(smem, lane);
  uint32_t* ws = reinterpret_cast<uint32_t*>(smem + GF_TABLE_BYTES);
  const TeamSync sync{1u, 32u * T};
  for (int64_t it = blockIdx.x; it < a.count; it += gridDim.x) {
    auto rows = [&](int g, const uint64_t*& u, const uint64_t*& v, const uint32_t*& y, uint8_t*& m) {
      bool ok = g == 0;
      if (KEYED) {
        // an index outside [0, nkeys) skips the item: m stays untouched
        const uint32_t ki = (uint32_t)__ldg(a.key_idx + it);
        const bool kok = ki < (uint64_t)a.nkeys;
        y = a.y + (kok ? (int64_t)ki : 0) * LV::w;
        ok = ok && kok;
      } else {
        y = a.y + it * LV::w;
      }
      u = a.u + it * LV::W_u_pitch;
      v = a.v + it * LV::W_v;
      m = a.m + it * LV::k;
      return ok;
    };
    decrypt_team<LV, !KEYED, T, 1>(gf, ws, wt, lane, sync, rows);
    after(it, ws);
  }
}

template <int LEVEL, bool KEYED, int T>
__global__ void __launch_bounds__(32 * T, 4) k_decrypt_latency(DecArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  latency_items<LEVEL, KEYED, T>(a, smem, [](int64_t, uint32_t*) {});
}

// ---------------------------------------------------------------------------
// Cluster latency form: the C blocks of a thread-block cluster decode ONE
// ciphertext together.  With four warps on one SM, the product of one
// HQC-5 ciphertext needs 131 x 16 x 4 shared-memory wavefronts, about 4 us
// of that SM's shared-memory bandwidth alone; split over C SMs it takes a
// C-th of that.  Block c of the cluster owns RM blocks [b0(c), b0(c + 1)):
// it builds the whole doubled operand, computes the product words of those
// blocks (strips of WPT words over its 32 T lanes, starting at its first
// word), XORs v, decodes its RM blocks in one pass of lane pairs, and
// stores the bytes into block 0's shared memory (distributed shared
// memory).  After a cluster barrier, block 0's team runs the RS stage.
// Only block 0 fills the GF tables.  Every block of a cluster takes the
// same items in the same order and meets the same two barriers per item
// (hardware barriers, no spin): A (block 0 has finished reading the
// previous item's bytes, and every block is running before the first
// remote store) and B (every byte is in block 0's memory).
// ---------------------------------------------------------------------------
template <class LV, int C, int T>
struct ClusterShare {
  static constexpr int NW = LV::n2 / 32;     // words per RM block
  static constexpr int MAXB = cdiv(LV::n1, C);  // most RM blocks per block
  static constexpr int WPT = odd_at_least(cdiv(MAXB * NW, 32 * T));
  __host__ __device__ static constexpr int b0(int c) { return c * LV::n1 / C; }
  // product reads reach word w0 + WPT + (n >> 5) for the last strip
  static constexpr int U2W =
      round_up(cmax(cdiv(2 * LV::n, 32), b0(C - 1) * NW + 32 * T * WPT + (LV::n >> 5) + 1), 4);
  static constexpr int RB = cdiv(LV::n1, 4) * 4;
  static constexpr int WORDS = round_up(U2W + LV::WP + RB / 4, 4);
  static_assert(LV::n2 % 32 == 0 && MAXB <= 16 * T, "one pass of lane pairs covers a block's RM share");
  static_assert(rs_team_scratch<T>() <= U2W && U2W % 4 == 0 && LV::WP % 4 == 0, "RS scratch fits; alignment");
};

__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }
// one byte into the same shared-memory offset of block `rank` of the cluster
__device__ __forceinline__ void st_cluster_u8(const uint8_t* local, uint32_t rank, uint32_t v) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(local);
  uint32_t ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
  asm volatile("st.shared::cluster.u8 [%0], %1;" ::"r"(ra), "r"(v) : "memory");
}

// after(it, ws, rbuf) runs on block 0 once per item, after RS, as in
// latency_items.
template <int LEVEL, bool KEYED, int C, int T, class After>
__device__ __forceinline__ void cluster_items(const DecArgs& a, uint8_t* smem, const After& after) {
  using LV = Level<LEVEL>;
  using CS = ClusterShare<LV, C, T>;
  const uint32_t rank = cluster_ctarank();
  if (rank == 0) gf_tables_init(smem, threadIdx.x, blockDim.x);
  __syncthreads();
  const int tid = threadIdx.x, lane = tid & 31, wt = tid >> 5;
  const GF gf(smem, lane);
  uint32_t* ws = reinterpret_cast<uint32_t*>(smem + GF_TABLE_BYTES);
  uint32_t* u2 = ws;
  uint32_t* sup = ws + CS::U2W;
  uint8_t* rbuf = reinterpret_cast<uint8_t*>(sup + LV::WP);
  const TeamSync sync{1u, 32u * T};
  const int b0 = CS::b0((int)rank), b1 = CS::b0((int)rank + 1);
  const int w_lo = b0 * CS::NW, w_hi = b1 * CS::NW;
  const int w0 = w_lo + tid * CS::WPT;
  const int64_t nclusters = gridDim.x / C;
  for (int64_t it = blockIdx.x / C; it < a.count; it += nclusters) {
    cluster_arrive();  // A
    bool ok = true;
    const uint32_t* y;
    if (KEYED) {
      // an index outside [0, nkeys) decodes key 0's supports and stores nothing
      const uint32_t ki = (uint32_t)__ldg(a.key_idx + it);
      ok = ki < (uint64_t)a.nkeys;
      y = a.y + (ok ? (int64_t)ki : 0) * LV::w;
    } else {
      y = a.y + it * LV::w;
    }
    load_supports<LV::n, LV::w, 32 * T>(sup, y, tid);
    build_doubled<LV::n, LV::W_u_pitch, CS::U2W, 32 * T>(u2, a.u + it * LV::W_u_pitch, tid, sync);
    uint32_t acc[CS::WPT];
    rot_xor_product<CS::WPT, LV::w, !KEYED, true>(u2, sup, w0, acc);
    const uint32_t* v32 = reinterpret_cast<const uint32_t*>(a.v + it * LV::W_v);
#pragma unroll
    for (int k = 0; k < CS::WPT; k++)
      if (w0 + k < w_hi) acc[k] ^= __ldcs(v32 + w0 + k);
    sync();
#pragma unroll
    for (int k = 0; k < CS::WPT; k++)
      if (w0 + k < w_hi) u2[w0 + k] = acc[k];
    sync();
    const int j = b0 + (tid >> 1);
    const int jj = j < b1 ? j : b1 - 1;
    const uint32_t byte = rm_decode_pair<LV::mult>(u2 + jj * CS::NW, tid & 1);
    cluster_wait();  // A
    if (j < b1 && (tid & 1) == 0) st_cluster_u8(rbuf + j, 0u, byte);
    cluster_arrive();  // B
    cluster_wait();
    if (rank == 0) {
      rs_decode_team<LV, T>(gf, ws, rbuf, wt, lane, sync, ok, a.m + it * LV::k);
      sync();  // the RS scratch lives in u2: the next item rebuilds it
      after(it, ws, rbuf);
    }
  }
}

template <int LEVEL, bool KEYED, int C, int T>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(32 * T, 1) k_decrypt_latency_cluster(DecArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  cluster_items<LEVEL, KEYED, C, T>(a, smem, [](int64_t, uint32_t*, const uint8_t*) {});
}

// ---------------------------------------------------------------------------
// Items of one level taken from a mixed list
// ---------------------------------------------------------------------------
// Whether item `it` of a one-level list names valid rows, key and m bytes.
template <int LEVEL>
__device__ __forceinline__ bool item_rows(const MixedArgs& a, int64_t it, const uint64_t*& u, const uint64_t*& v,
                                          const uint32_t*& y, uint8_t*& m) {
  using LV = Level<LEVEL>;
  constexpr int li = LEVEL == 1 ? 0 : LEVEL == 3 ? 1 : 2;
  if (it >= a.count) return false;
  const MixedItem item = a.items[it];
  const bool ok = item.level == LEVEL && (uint32_t)item.key < (uint64_t)a.nkeys[li] && item.u_off >= 0 &&
                  (item.u_off & 1) == 0 && item.u_off + LV::W_u_pitch <= a.arena_words && item.v_off >= 0 &&
                  item.v_off + LV::W_v <= a.arena_words && item.m_off >= 0 && item.m_off + LV::k <= a.m_bytes;
  u = a.arena + (ok ? item.u_off : 0);
  v = a.arena + (ok ? item.v_off : 0);
  y = a.keys[li] + (ok ? (int64_t)item.key * LV::w : 0);
  m = a.m + (ok ? item.m_off : 0);
  return ok;
}

// The items of ONE level by single warps, G per warp per turn: block `blk`
// of `nblk`, warp `warp` of `nw` (the shared memory after the GF tables is
// nw slices of fused_warp_words<LV, G>, after the syndrome table if SYN).
template <int LEVEL, int G, bool SYN = false>
__device__ __forceinline__ void items_solo(const MixedArgs& a, uint8_t* smem, int64_t blk, int64_t nblk, int warp,
                                           int nw) {
  using LV = Level<LEVEL>;
  const int lane = threadIdx.x & 31;
  const GF gf(smem, lane);
  uint32_t* ws = reinterpret_cast<uint32_t*>(smem + GF_TABLE_BYTES + (SYN ? SYN_TABLE_BYTES : 0)) +
                 warp * fused_warp_words<LV, G>();
  const int64_t ngroups = (a.count + G - 1) / G;
  for (int64_t q = blk * nw + warp; q < ngroups; q += nblk * nw) {
    auto rows = [&](int g, const uint64_t*& u, const uint64_t*& v, const uint32_t*& y, uint8_t*& m) {
      return item_rows<LEVEL>(a, q * G + g, u, v, y, m);
    };
    decrypt_group<LV, G, false, SYN>(gf, ws, lane, rows, smem + GF_TABLE_BYTES);
  }
}

// The same with two-warp teams (nw even, at most 30): team t = warp / 2
// takes pairs of items.
template <int LEVEL>
__device__ __forceinline__ void items_team(const MixedArgs& a, uint8_t* smem, int64_t blk, int64_t nblk, int warp,
                                           int nw) {
  using LV = Level<LEVEL>;
  const int lane = threadIdx.x & 31;
  const int team = warp >> 1, wt = warp & 1, nteams = nw >> 1;
  const GF gf(smem, lane);
  uint32_t* ws = reinterpret_cast<uint32_t*>(smem + GF_TABLE_BYTES) + team * Team<LV>::WORDS;
  const TeamSync sync{(uint32_t)(1 + team)};
  const int64_t ngroups = (a.count + 1) / 2;
  for (int64_t q = blk * nteams + team; q < ngroups; q += nblk * nteams) {
    auto rows = [&](int g, const uint64_t*& u, const uint64_t*& v, const uint32_t*& y, uint8_t*& m) {
      return item_rows<LEVEL>(a, 2 * q + g, u, v, y, m);
    };
    decrypt_team<LV, false>(gf, ws, wt, lane, sync, rows);
  }
}

// Persistent kernels over the items of ONE level taken from a mixed list
// (the list was partitioned by level beforehand).  Static stride: every
// item of a level costs the same.  The level-partitioned plan runs one of
// these per level side by side in a CUDA graph.
template <int LEVEL, int G = FusedGroup<LEVEL>::G>
__global__ void __launch_bounds__(FusedBound<LEVEL>::threads, 1) k_decrypt_items(MixedArgs a) {
  constexpr bool SYN = FusedSyn<LEVEL>::on;
  extern __shared__ __align__(16) uint8_t smem[];
  gf_tables_init(smem, threadIdx.x, blockDim.x);
  if constexpr (SYN) syn_table_init(smem + GF_TABLE_BYTES, threadIdx.x, blockDim.x);
  __syncthreads();
  items_solo<LEVEL, G, SYN>(a, smem, blockIdx.x, gridDim.x, threadIdx.x >> 5, blockDim.x >> 5);
}

template <int LEVEL>
__global__ void __launch_bounds__(TeamBound<LEVEL>::threads, 1) k_decrypt_items_team(MixedArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  gf_tables_init(smem, threadIdx.x, blockDim.x);
  __syncthreads();
  items_team<LEVEL>(a, smem, blockIdx.x, gridDim.x, threadIdx.x >> 5, blockDim.x >> 5);
}

// ---------------------------------------------------------------------------
// Plain per-stage form.
// K1: product + XOR with v (warp per ciphertext), w (and t) to global.
// ---------------------------------------------------------------------------
constexpr int STAGE_THREADS = 256;

template <int LEVEL, bool KEYED, bool WITH_T>
__global__ void __launch_bounds__(STAGE_THREADS) k_stage_product(DecArgs a, uint64_t* w_out, uint64_t* t_out) {
  using LV = Level<LEVEL>;
  extern __shared__ __align__(16) uint8_t smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t it = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (it >= a.count) return;
  uint32_t* ws = reinterpret_cast<uint32_t*>(smem) + warp * LV::WARP_WORDS;
  const uint32_t* yrow;
  if (KEYED) {
    const uint32_t ki = (uint32_t)__ldg(a.key_idx + it);
    yrow = a.y + (ki < (uint64_t)a.nkeys ? (int64_t)ki : 0) * LV::w;
  } else {
    yrow = a.y + it * LV::w;
  }
  load_supports<LV::n, LV::w>(ws + LV::U2W, yrow, lane);
  build_doubled<LV::n, LV::W_u_pitch, LV::U2W>(ws, a.u + it * LV::W_u_pitch, lane);
  using PS = ProductStrips<LEVEL>;
  const int w0 = PS::start(lane), wn = PS::len(lane);
  uint32_t acc[PS::MAXLEN];
  rot_xor_product<PS::MAXLEN, LV::w, !KEYED>(ws, ws + LV::U2W, w0, acc);
  const uint32_t* v32 = reinterpret_cast<const uint32_t*>(a.v + it * LV::W_v);
  uint32_t* w32 = reinterpret_cast<uint32_t*>(w_out + it * LV::W_v);
  uint32_t* t32 = WITH_T ? reinterpret_cast<uint32_t*>(t_out + it * LV::W_v) : nullptr;
#pragma unroll
  for (int k = 0; k < PS::MAXLEN; k++) {
    const int i = w0 + k;
    if (k < wn && i < LV::W_v32) {
      if (WITH_T) t32[i] = acc[k];
      w32[i] = acc[k] ^ v32[i];
    }
  }
}

// K2: one lane pair per (ciphertext, RS symbol): duplicated RM decode.
template <int LEVEL>
__global__ void __launch_bounds__(STAGE_THREADS) k_stage_rm(int64_t count, const uint64_t* __restrict__ w,
                                                           uint8_t* __restrict__ r_out) {
  using LV = Level<LEVEL>;
  const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 1;  // pair index
  const int64_t total = count * LV::n1;
  const int64_t gg = g < total ? g : total - 1;  // both lanes of every pair stay active
  const int64_t it = gg / LV::n1;
  const int j = (int)(gg - it * LV::n1);
  const uint32_t* blk = reinterpret_cast<const uint32_t*>(w + it * LV::W_v) + j * (LV::n2 / 32);
  const uint32_t byte = rm_decode_pair<LV::mult, false>(blk, threadIdx.x & 1);
  if (g < total && (threadIdx.x & 1) == 0) r_out[it * LV::n1 + j] = (uint8_t)byte;
}

// K3: one warp per ciphertext: Reed-Solomon decode (and the debug dump).
constexpr int RS_SCRATCH_WORDS = 24 + RS_SCRATCH;  // the n1 received bytes, then the RS scratch

// With key_idx given, a ciphertext whose index is outside [0, nkeys) is
// skipped (its m row stays untouched), as in the fused kernels.
template <int LEVEL, bool DEBUG>
__global__ void __launch_bounds__(STAGE_THREADS) k_stage_rs(int64_t count, const uint8_t* __restrict__ r_in,
                                                           uint8_t* __restrict__ m_out, DebugArgs d,
                                                           const int32_t* __restrict__ key_idx, int64_t nkeys) {
  using LV = Level<LEVEL>;
  static_assert(LV::n1 <= 96, "received bytes fit in 24 words");
  extern __shared__ __align__(16) uint8_t smem[];
  gf_tables_init(smem, threadIdx.x, blockDim.x);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t it = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (it >= count) return;
  if (key_idx && (uint32_t)__ldg(key_idx + it) >= (uint64_t)nkeys) return;
  const GF gf(smem, lane);
  uint32_t* base = reinterpret_cast<uint32_t*>(smem + GF_TABLE_BYTES) + warp * RS_SCRATCH_WORDS;
  uint8_t* rb = reinterpret_cast<uint8_t*>(base);
  for (int j = lane; j < LV::n1; j += 32) rb[j] = r_in[it * LV::n1 + j];
  __syncwarp();
  if (DEBUG) {
    RSDebugRow row{d.S + it * LV::NR, d.lam + it * LV::CAP, d.L + it,  d.errmask + it * LV::n1,
                   d.errval + it * LV::n1, d.cw + it * LV::n1, d.flag + it};
    rs_decode_seg<LV, 32, true>(gf, base + 24, rb, lane, true, m_out + it * LV::k, &row);
  } else {
    rs_decode_seg<LV, 32, false>(gf, base + 24, rb, lane, true, m_out + it * LV::k, nullptr);
  }
}

// ---------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------
template <int LEVEL>
[[maybe_unused]] static size_t fused_smem(int warps) {
  return (size_t)fused_fixed_bytes<LEVEL>() + (size_t)warps * fused_words<LEVEL>() * 4;
}

[[maybe_unused]] static std::mutex g_shape_mu;
static std::map<std::pair<const void*, int>, size_t> g_shape_attr;
static std::map<std::tuple<const void*, int, int, size_t>, int> g_shape_occ;

static inline int device_props(int* sms, int* smem_optin) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return dev;
}

// per_warp: shared bytes per warp (for teams: per team / 2); teams: the
// warp count must be even and at most 30 (15 named barriers); fixed: the
// block's bytes before the warps' slices (the GF tables, and for some
// kernels the syndrome table).
template <class KernelT>
static cudaError_t shape_for(KernelT kern, int max_threads, size_t per_warp, const LaunchCfg& cfg, int* warps,
                             int* ctas, int* grid, size_t* smem_bytes, bool teams = false,
                             size_t fixed = GF_TABLE_BYTES) {
  int sms = 0, optin = 0;
  const int dev = device_props(&sms, &optin);
  int nw = cfg.warps_per_cta;
  if (nw <= 0) {
    nw = (int)((optin - fixed) / per_warp);
    if (nw > max_threads / 32) nw = max_threads / 32;
    if (teams) nw = std::min(nw & ~1, 30);
  }
  if (nw < 1 || (teams && (nw & 1))) return cudaErrorInvalidValue;
  if (nw > max_threads / 32 || (teams && nw > 30)) return cudaErrorInvalidValue;
  const size_t sm = fixed + (size_t)nw * per_warp;
  if (sm > (size_t)optin) return cudaErrorInvalidValue;
  // the shared-memory attribute only grows, and occupancies are looked up
  // once per (kernel, device, warps, bytes): repeated launches of small
  // batches pay no runtime queries
  const void* kp = reinterpret_cast<const void*>(kern);
  int occ = 0;
  {
    std::lock_guard<std::mutex> lock(g_shape_mu);
    size_t& attr = g_shape_attr[{kp, dev}];
    if (sm > attr) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
      attr = sm;
    }
    const auto key = std::make_tuple(kp, dev, nw, sm);
    const auto hit = g_shape_occ.find(key);
    if (hit != g_shape_occ.end()) {
      occ = hit->second;
    } else {
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, nw * 32, sm);
      if (e != cudaSuccess) return e;
      g_shape_occ[key] = occ;
    }
  }
  if (occ < 1) return cudaErrorInvalidConfiguration;
  int c = cfg.ctas_per_sm > 0 ? cfg.ctas_per_sm : occ;
  if (c > occ) c = occ;
  *warps = nw;
  *ctas = c;
  *grid = sms * c;
  *smem_bytes = sm;
  return cudaSuccess;
}

}  // namespace hqc

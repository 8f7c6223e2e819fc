// The plain one-kernel-per-stage decryption (product, RM, RS as three
// launches with intermediates in global memory), the debug path that dumps
// every intermediate, and debug forms of the latency and throughput
// kernels that dump what their own RS stage held.
#include <cuda_runtime.h>

#include <algorithm>

#include "hqc_kernels.cuh"

namespace hqc {

template <int LEVEL, bool KEYED, bool DEBUG>
static cudaError_t staged_level(const DecArgs& a, uint64_t* w, uint8_t* r, const DebugArgs* d, cudaStream_t st) {
  using LV = Level<LEVEL>;
  if (a.count == 0) return cudaSuccess;
  const int wpb = STAGE_THREADS / 32;
  // K1
  {
    auto kern = k_stage_product<LEVEL, KEYED, DEBUG>;
    const size_t sm = (size_t)wpb * LV::WARP_WORDS * 4;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (a.count + wpb - 1) / wpb;
    kern<<<(unsigned)blocks, STAGE_THREADS, sm, st>>>(a, w, DEBUG ? d->t : nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // K2
  {
    const int64_t threads = 2 * a.count * LV::n1;
    const int64_t blocks = (threads + STAGE_THREADS - 1) / STAGE_THREADS;
    k_stage_rm<LEVEL><<<(unsigned)blocks, STAGE_THREADS, 0, st>>>(a.count, w, r);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // K3
  {
    auto kern = k_stage_rs<LEVEL, DEBUG>;
    const size_t sm = GF_TABLE_BYTES + (size_t)wpb * RS_SCRATCH_WORDS * 4;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (a.count + wpb - 1) / wpb;
    DebugArgs dd{};
    if (DEBUG) dd = *d;
    kern<<<(unsigned)blocks, STAGE_THREADS, sm, st>>>(a.count, r, a.m, dd, KEYED ? a.key_idx : nullptr, a.nkeys);
    return cudaGetLastError();
  }
}

cudaError_t launch_staged(int level, bool keyed, const DecArgs& a, uint64_t* w, uint8_t* r, cudaStream_t st) {
  switch (level) {
    case 1: return keyed ? staged_level<1, true, false>(a, w, r, nullptr, st) : staged_level<1, false, false>(a, w, r, nullptr, st);
    case 3: return keyed ? staged_level<3, true, false>(a, w, r, nullptr, st) : staged_level<3, false, false>(a, w, r, nullptr, st);
    case 5: return keyed ? staged_level<5, true, false>(a, w, r, nullptr, st) : staged_level<5, false, false>(a, w, r, nullptr, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_debug(int level, const DecArgs& a, const DebugArgs& d, cudaStream_t st) {
  switch (level) {
    case 1: return staged_level<1, false, true>(a, d.w, d.r, &d, st);
    case 3: return staged_level<3, false, true>(a, d.w, d.r, &d, st);
    case 5: return staged_level<5, false, true>(a, d.w, d.r, &d, st);
  }
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Debug forms of the latency kernels: the same per-item code as
// k_decrypt_latency and k_decrypt_latency_cluster (literal supports), then
// the block that ran RS copies the item's RM bytes and, from the RS
// scratch, its syndromes and Lambda to d (r, S, lam).
// ---------------------------------------------------------------------------
template <class LV>
__device__ __forceinline__ void dump_team_item(int64_t it, uint32_t* rs, const uint8_t* rbuf, const DebugArgs& d,
                                               const uint8_t* smem) {
  constexpr int NR = LV::NR;
  const GF gf(smem, threadIdx.x & 31);
  const uint16_t* logS = rs_team_logS(rs);
  const uint16_t* logLam = rs_team_logLam(rs);
  for (int j = threadIdx.x; j < LV::n1; j += blockDim.x) d.r[it * LV::n1 + j] = rbuf[j];
  for (int i = threadIdx.x; i < NR; i += blockDim.x) d.S[it * NR + i] = (uint8_t)gf.exp(logS[i]);
  for (int c = threadIdx.x; c < NR + 1; c += blockDim.x) d.lam[it * (NR + 1) + c] = (uint8_t)gf.exp(logLam[c]);
  __syncthreads();  // the next item rebuilds the scratch
}

template <int LEVEL>
__global__ void __launch_bounds__(32 * LAT_TEAM, 4) k_debug_latency(DecArgs a, DebugArgs d) {
  using LV = Level<LEVEL>;
  extern __shared__ __align__(16) uint8_t smem[];
  latency_items<LEVEL, false, LAT_TEAM>(a, smem, [&](int64_t it, uint32_t* ws) {
    dump_team_item<LV>(it, ws, Team<LV, LAT_TEAM, 1>::rbuf(ws), d, smem);
  });
}

template <int LEVEL>
__global__ void __cluster_dims__(4, 1, 1) __launch_bounds__(32 * LAT_TEAM, 1) k_debug_cluster(DecArgs a, DebugArgs d) {
  extern __shared__ __align__(16) uint8_t smem[];
  cluster_items<LEVEL, false, 4, LAT_TEAM>(a, smem, [&](int64_t it, uint32_t* ws, const uint8_t* rbuf) {
    dump_team_item<Level<LEVEL>>(it, ws, rbuf, d, smem);
  });
}

// ---------------------------------------------------------------------------
// Debug form of the persistent throughput kernels: the same per-turn code
// as k_decrypt_fused (solo warps, G words per turn; for HQC-1 with the
// syndrome table and Horner syndromes) or, for HQC-5, k_decrypt_team
// (two-warp teams, one word's RS per warp), with literal supports.  After
// each turn the warp that ran a word's RS copies its RM bytes and, from
// rs_decode_seg's scratch (log S at halfword 64 of word 48, log Lambda at
// word 112), its syndromes and Lambda to d, before the next turn reuses the
// shared memory.  Blocks of DEBUG_FUSED_WARPS warps; the decoding does not
// depend on the block shape.
// ---------------------------------------------------------------------------
constexpr int DEBUG_FUSED_WARPS = 4;

template <class LV>
__device__ __forceinline__ void dump_seg_item(int64_t it, const uint32_t* rs, const uint8_t* rb, const DebugArgs& d,
                                              const GF& gf, int lane) {
  constexpr int NR = LV::NR;
  const uint16_t* logS = reinterpret_cast<const uint16_t*>(rs + 48) + 64;
  const uint16_t* logLam = reinterpret_cast<const uint16_t*>(rs + 112);
  for (int j = lane; j < LV::n1; j += 32) d.r[it * LV::n1 + j] = rb[j];
  for (int i = lane; i < NR; i += 32) d.S[it * NR + i] = (uint8_t)gf.exp(logS[i]);
  for (int c = lane; c < NR + 1; c += 32) d.lam[it * (NR + 1) + c] = (uint8_t)gf.exp(logLam[c]);
}

template <int LEVEL>
__global__ void __launch_bounds__(32 * DEBUG_FUSED_WARPS) k_debug_fused(DecArgs a, DebugArgs d) {
  using LV = Level<LEVEL>;
  extern __shared__ __align__(16) uint8_t smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  auto literal = [&](int64_t it0, int64_t first, const uint64_t*& u, const uint64_t*& v, const uint32_t*& y,
                     uint8_t*& m) {
    const bool ok = it0 < a.count;
    const int64_t it = ok ? it0 : first;
    u = a.u + it * LV::W_u_pitch;
    v = a.v + it * LV::W_v;
    y = a.y + it * LV::w;
    m = a.m + it * LV::k;
    return ok;
  };
  if constexpr (UseTeam<LEVEL>::value) {
    using TT = Team<LV>;
    gf_tables_init(smem, threadIdx.x, blockDim.x);
    __syncthreads();
    const GF gf(smem, lane);
    const int team = warp >> 1, wt = warp & 1, nteams = nw >> 1;
    uint32_t* ws = reinterpret_cast<uint32_t*>(smem + GF_TABLE_BYTES) + team * TT::WORDS;
    const TeamSync sync{(uint32_t)(1 + team)};
    const int64_t ngroups = (a.count + 1) / 2;
    for (int64_t q = (int64_t)blockIdx.x * nteams + team; q < ngroups; q += (int64_t)gridDim.x * nteams) {
      decrypt_team<LV, true>(gf, ws, wt, lane, sync,
                             [&](int g, const uint64_t*& u, const uint64_t*& v, const uint32_t*& y, uint8_t*& m) {
                               return literal(2 * q + g, 2 * q, u, v, y, m);
                             });
      // decrypt_team ends with the team barrier; its RS scratch is intact
      // until the next turn's product
      if (2 * q + wt < a.count) dump_seg_item<LV>(2 * q + wt, ws + wt * RS_SCRATCH, TT::rbuf(ws) + wt * TT::RB, d, gf, lane);
      sync();
    }
  } else {
    constexpr int G = FusedGroup<LEVEL>::G;
    constexpr bool SYN = FusedSyn<LEVEL>::on;
    constexpr int RB = cdiv(LV::n1, 4) * 4;
    gf_tables_init(smem, threadIdx.x, blockDim.x);
    if constexpr (SYN) syn_table_init(smem + GF_TABLE_BYTES, threadIdx.x, blockDim.x);
    __syncthreads();
    const GF gf(smem, lane);
    uint32_t* ws = reinterpret_cast<uint32_t*>(smem + fused_fixed_bytes<LEVEL>()) + warp * fused_warp_words<LV, G>();
    const uint8_t* rbuf = reinterpret_cast<const uint8_t*>(ws + LV::U2W + LV::WP);
    const int64_t ngroups = (a.count + G - 1) / G;
    for (int64_t q = (int64_t)blockIdx.x * nw + warp; q < ngroups; q += (int64_t)gridDim.x * nw) {
      decrypt_group<LV, G, true, SYN>(gf, ws, lane,
                                      [&](int g, const uint64_t*& u, const uint64_t*& v, const uint32_t*& y,
                                          uint8_t*& m) { return literal(q * G + g, q * G, u, v, y, m); },
                                      smem + GF_TABLE_BYTES);
      for (int g = 0; g < G; g++)
        if (q * G + g < a.count) dump_seg_item<LV>(q * G + g, ws + g * RS_SCRATCH, rbuf + g * RB, d, gf, lane);
      __syncwarp();
    }
  }
}

template <int LEVEL>
static cudaError_t debug_fused_level(const DecArgs& a, const DebugArgs& d, cudaStream_t st) {
  using LV = Level<LEVEL>;
  constexpr int NW = DEBUG_FUSED_WARPS;
  size_t sm;
  int64_t per_block;
  if constexpr (UseTeam<LEVEL>::value) {
    sm = GF_TABLE_BYTES + (size_t)(NW / 2) * Team<LV>::WORDS * 4;
    per_block = NW;  // NW / 2 teams, two words each
  } else {
    constexpr int G = FusedGroup<LEVEL>::G;
    sm = (size_t)fused_fixed_bytes<LEVEL>() + (size_t)NW * fused_warp_words<LV, G>() * 4;
    per_block = (int64_t)NW * G;
  }
  cudaError_t e = cudaFuncSetAttribute(k_debug_fused<LEVEL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  // at most 64 blocks: several turns per warp when the batch is larger
  const int64_t grid = std::min<int64_t>(64, (a.count + per_block - 1) / per_block);
  k_debug_fused<LEVEL><<<(unsigned)grid, 32 * NW, sm, st>>>(a, d);
  return cudaGetLastError();
}

template <int LEVEL>
static cudaError_t debug_team_level(int form, const DecArgs& a, const DebugArgs& d, cudaStream_t st) {
  using LV = Level<LEVEL>;
  if (a.count == 0) return cudaSuccess;
  if (form == 2) return debug_fused_level<LEVEL>(a, d, st);
  if (form == 0) {
    constexpr size_t sm = GF_TABLE_BYTES + (size_t)Team<LV, LAT_TEAM, 1>::WORDS * 4;
    cudaError_t e = cudaFuncSetAttribute(k_debug_latency<LEVEL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int64_t grid = std::min<int64_t>(a.count, MAX_LATENCY_GRID);
    k_debug_latency<LEVEL><<<(unsigned)grid, 32 * LAT_TEAM, sm, st>>>(a, d);
  } else {
    constexpr size_t sm = GF_TABLE_BYTES + (size_t)ClusterShare<LV, 4, LAT_TEAM>::WORDS * 4;
    cudaError_t e = cudaFuncSetAttribute(k_debug_cluster<LEVEL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int64_t clusters = std::min<int64_t>(a.count, MAX_LATENCY_GRID / 4);
    k_debug_cluster<LEVEL><<<(unsigned)(clusters * 4), 32 * LAT_TEAM, sm, st>>>(a, d);
  }
  return cudaGetLastError();
}

cudaError_t launch_debug_team(int level, int form, const DecArgs& a, const DebugArgs& d, cudaStream_t st) {
  if (form < 0 || form > 2) return cudaErrorInvalidValue;
  switch (level) {
    case 1: return debug_team_level<1>(form, a, d, st);
    case 3: return debug_team_level<3>(form, a, d, st);
    case 5: return debug_team_level<5>(form, a, d, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hqc

// The plain one-kernel-per-stage decryption (product, RM, RS as three
// launches with intermediates in global memory) and the debug path that
// dumps every intermediate.
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

template <int LEVEL>
static cudaError_t debug_team_level(int form, const DecArgs& a, const DebugArgs& d, cudaStream_t st) {
  using LV = Level<LEVEL>;
  if (a.count == 0) return cudaSuccess;
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
  if (form != 0 && form != 1) return cudaErrorInvalidValue;
  switch (level) {
    case 1: return debug_team_level<1>(form, a, d, st);
    case 3: return debug_team_level<3>(form, a, d, st);
    case 5: return debug_team_level<5>(form, a, d, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hqc

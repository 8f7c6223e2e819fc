// The plain one-kernel-per-stage decryption (product, RM, RS as three
// launches with intermediates in global memory) and the debug path that
// dumps every intermediate.
#include <cuda_runtime.h>

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

}  // namespace hqc

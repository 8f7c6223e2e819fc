// S5-S7 (duplicated RM(1,7) decoding, Sec. II-A) on the tensor cores: the
// Walsh-Hadamard transform of every block written as one dense product
// F = S H with H the 128 x 128 matrix of (-1)^popcount(a & i), run by
// tcgen05.mma (kind::f16, fp32 accumulators in tensor memory) on tiles of
// 128 RM blocks.  A measured alternative to the register butterflies of
// rm_decode_pair (k_stage_rm); both give the same bytes.
//
// Exactness.  Row t of the A tile holds, for block t, 512 + cnt_i as fp16
// (cnt_i = copies with bit i set, at most 5: exact, bit pattern 0x6000 +
// 2 cnt_i).  With D = A H^T accumulated in fp32 (every partial sum is an
// integer below 2^17, exact):
//   D(a) = C(a) for a > 0 and D(0) = 65536 + C(0), C = the transform of
//   cnt; since s_i = mult - 2 cnt_i, F(a) = -2 D(a) for a > 0 and
//   F(0) = 2 (mult 64 + 65536 - D(0)).
// The argmax over |F| (ties to the smaller a) and the sign of F there use
// one fp32 key per column: |F| / 2 * 256 + (127 - a) * 2 + [F < 0], at most
// 320 * 256 + 255 < 2^24, so every key is an exact integer in fp32.
//
// Tensor-core details.  Both operands are K-major in the canonical layout
// without swizzle: core matrices of 8 rows x 16 bytes, K-adjacent ones 128
// bytes apart (the descriptor's leading offset), 8-row groups 2048 bytes
// apart (its stride offset).  A block holds four groups of four warps that
// share the H tile (160 KB of shared memory, all 512 tensor-memory columns:
// one block per SM, 16 warps).  In each group one thread issues the eight
// K = 16 steps and commits them to the group's mbarrier; the group's four
// warps then read their 32 TMEM lanes (rows) with tcgen05.ld.  Each thread
// loads its block's words for the group's next tile one turn ahead.
// Every wait on an mbarrier is bounded: on a timeout the kernel records it
// in a device flag, stops, frees its tensor memory and returns.
#include <cuda_runtime.h>

#include "hqc_kernels.cuh"

namespace hqc {

namespace {

constexpr int RMTC_ROWS = 128;                    // RM blocks per tile (MMA M)
constexpr int RMTC_TILE_BYTES = 128 * 128 * 2;    // one fp16 operand tile
constexpr int RMTC_GROUPS = 4;                    // four-warp groups per block, one tile each
constexpr int RMTC_SMEM = (RMTC_GROUPS + 1) * RMTC_TILE_BYTES + 64;  // A per group, H, mbarriers, TMEM address
constexpr uint32_t RMTC_TMEM_COLS = 128 * RMTC_GROUPS;  // one 128-column fp32 accumulator per group
constexpr int RMTC_MAX_SPIN = 1 << 22;

__device__ int g_rm_tc_timeouts = 0;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (row, k) in a K-major 128 x 128 fp16 tile
__device__ __forceinline__ int tile_off(int row, int k) {
  return (row >> 3) * 2048 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// shared-memory matrix descriptor: start, leading and stride byte offsets
// (all in 16-byte units), descriptor version 1, no swizzle, base offset 0
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | (uint64_t)(128u >> 4) << 16 | (uint64_t)(2048u >> 4) << 32 |
         1ull << 46;
}

// kind::f16 instruction descriptor: D f32, A and B f16, both K-major,
// N = 128, M = 128
constexpr uint32_t RMTC_IDESC = (1u << 4) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// barrier of the 128 threads of group g (named barrier 1 + g); the AND of p
__device__ __forceinline__ void group_sync(int g) {
  asm volatile("bar.sync %0, 128;" ::"r"(1 + g) : "memory");
}
__device__ __forceinline__ bool group_and(int g, bool p) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred a, b;\n\tsetp.ne.u32 a, %2, 0;\n\tbar.red.and.pred b, %1, 128, a;\n\tselp.u32 %0, 1, 0, b;\n\t}"
      : "=r"(r)
      : "r"(1 + g), "r"((uint32_t)p)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity) {
  uint32_t done = 0;
  for (int spin = 0; spin < RMTC_MAX_SPIN && !done; spin++) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
  }
  return done != 0;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// counts of 32 consecutive positions of the MULT copies b[] as fp16
// patterns 0x6000 + 2 cnt, two per word: word m holds positions 2m, 2m + 1
template <int MULT>
__device__ __forceinline__ void count_pairs(const uint32_t (&b)[MULT], uint32_t (&out)[16]) {
  static_assert(MULT == 3 || MULT == 5, "HQC duplicates RM codewords 3 or 5 times");
  // bit-sliced population count: cnt = p0 + 2 p1 (+ 4 p2)
  const uint32_t s1 = b[0] ^ b[1] ^ b[2];
  const uint32_t k1 = (b[0] & b[1]) | (b[2] & (b[0] ^ b[1]));
  if constexpr (MULT == 3) {
    // z0: the count of position 2m at bits 2m, 2m + 1; z1: that of 2m + 1
    const uint32_t z0 = (s1 & 0x55555555u) | ((k1 & 0x55555555u) << 1);
    const uint32_t z1 = ((s1 & 0xAAAAAAAAu) >> 1) | (k1 & 0xAAAAAAAAu);
#pragma unroll
    for (int m = 0; m < 16; m++) {
      const uint32_t lo = (m == 0 ? z0 << 1 : z0 >> (2 * m - 1)) & 0x6u;
      const uint32_t hi = (2 * m <= 17 ? z1 << (17 - 2 * m) : z1 >> (2 * m - 17)) & 0x60000u;
      out[m] = 0x60006000u | lo | hi;
    }
  } else {
    const uint32_t d = b[MULT > 3 ? 3 : 0], e = b[MULT > 4 ? 4 : 0];
    const uint32_t k2 = (s1 & d) | (e & (s1 ^ d));
    const uint32_t p0 = s1 ^ d ^ e, p1 = k1 ^ k2, p2 = k1 & k2;
    // z[rr]: the count of position 4u + rr at bits 4u .. 4u + 2
    uint32_t z[4];
#pragma unroll
    for (int rr = 0; rr < 4; rr++) {
      const uint32_t mk = 0x11111111u << rr;
      z[rr] = ((p0 & mk) >> rr) | (((p1 & mk) >> rr) << 1) | (((p2 & mk) >> rr) << 2);
    }
#pragma unroll
    for (int m = 0; m < 16; m++) {
      const int u = m >> 1, r0 = (2 * m) & 3;  // positions 2m = 4u + r0 and 2m + 1
      const uint32_t ze = z[r0], zo = z[r0 + 1];
      const uint32_t lo = (u == 0 ? ze << 1 : ze >> (4 * u - 1)) & 0xEu;
      const uint32_t hi = (4 * u <= 17 ? zo << (17 - 4 * u) : zo >> (4 * u - 17)) & 0xE0000u;
      out[m] = 0x60006000u | lo | hi;
    }
  }
}

template <int LEVEL>
__global__ void __launch_bounds__(128 * RMTC_GROUPS, 1) k_rm_tc(int64_t count, const uint64_t* __restrict__ w,
                                                               uint8_t* __restrict__ r_out) {
  using LV = Level<LEVEL>;
  constexpr int MULT = LV::mult, NW = LV::n2 / 32;
  static_assert(LV::n2 == 128 * MULT, "one RM block is MULT copies of 128 bits");
  extern __shared__ __align__(1024) uint8_t smem[];
  // four groups of four warps share H; group g owns A tile g, mbarrier g
  // and accumulator columns [128 g, 128 g + 128)
  uint8_t* sh = smem + RMTC_GROUPS * RMTC_TILE_BYTES;
  uint64_t* mbars = reinterpret_cast<uint64_t*>(smem + (RMTC_GROUPS + 1) * RMTC_TILE_BYTES);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + (RMTC_GROUPS + 1) * RMTC_TILE_BYTES + 8 * RMTC_GROUPS);
  const int grp = threadIdx.x >> 7, tid = threadIdx.x & 127, warp = tid >> 5;
  uint8_t* sa = smem + grp * RMTC_TILE_BYTES;
  uint64_t* mbar = mbars + grp;
  // B: row n of H, (-1)^popcount(n & k) as fp16 (rows split over the groups)
  for (int r = threadIdx.x; r < 128 * 16; r += blockDim.x) {
    const int n = r >> 4, k8 = r & 15;
    uint32_t p[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int k0 = 8 * k8 + 2 * q;
      const uint32_t lo = (__popc(n & k0) & 1) ? 0xBC00u : 0x3C00u;
      const uint32_t hi = (__popc(n & (k0 + 1)) & 1) ? 0xBC00u : 0x3C00u;
      p[q] = lo | (hi << 16);
    }
    *reinterpret_cast<uint4*>(sh + tile_off(n, 8 * k8)) = make_uint4(p[0], p[1], p[2], p[3]);
  }
  if (threadIdx.x < RMTC_GROUPS) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbars + threadIdx.x)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(RMTC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot + 128u * grp;
  const int64_t total = count * LV::n1;
  const int64_t ntiles = (total + RMTC_ROWS - 1) / RMTC_ROWS;
  const int64_t first = (int64_t)blockIdx.x * RMTC_GROUPS + grp, stride = (int64_t)gridDim.x * RMTC_GROUPS;
  uint32_t parity = 0;
  bool ok = true;
  // the words of this thread's RM block of a tile (row tid; the tail of the
  // last tile repeats the last block, and its byte is not stored)
  uint32_t words[MULT][4];
  auto fetch = [&](int64_t tile) {
    const int64_t g = tile * RMTC_ROWS + tid;
    const int64_t gg = g < total ? g : total - 1;
    const int64_t it = gg / LV::n1;
    const int j = (int)(gg - it * LV::n1);
    const uint32_t* blk = reinterpret_cast<const uint32_t*>(w + it * LV::W_v) + j * NW;
#pragma unroll
    for (int c = 0; c < MULT; c++)
#pragma unroll
      for (int q = 0; q < 4; q++) words[c][q] = __ldg(blk + 4 * c + q);
  };
  if (first < ntiles) fetch(first);
  for (int64_t tile = first; tile < ntiles && ok; tile += stride) {
    const int64_t g = tile * RMTC_ROWS + tid;
#pragma unroll
    for (int q = 0; q < 4; q++) {
      uint32_t b[MULT];
#pragma unroll
      for (int c = 0; c < MULT; c++) b[c] = words[c][q];
      uint32_t pk[16];
      count_pairs<MULT>(b, pk);
#pragma unroll
      for (int u = 0; u < 4; u++)
        *reinterpret_cast<uint4*>(sa + tile_off(tid, 32 * q + 8 * u)) =
            make_uint4(pk[4 * u], pk[4 * u + 1], pk[4 * u + 2], pk[4 * u + 3]);
    }
    // the next tile's words load while this tile's product and argmax run
    if (tile + stride < ntiles) fetch(tile + stride);
    // generic-proxy stores -> visible to the tensor core's reads
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    group_sync(grp);
    tc_fence_after();
    if (tid == 0) {
#pragma unroll
      for (int kk = 0; kk < 8; kk++) {
        const uint64_t ad = smem_desc(smem_u32(sa) + 256u * kk);
        const uint64_t bd = smem_desc(smem_u32(sh) + 256u * kk);
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(RMTC_IDESC), "r"((uint32_t)(kk > 0)));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(mbar))
                   : "memory");
    }
    const bool done = mbar_wait_bounded(smem_u32(mbar), parity);
    parity ^= 1u;
    ok = group_and(grp, done);
    tc_fence_after();
    if (ok) {
      constexpr float H0 = (float)(MULT * 64 + 65536);
      float best = -1.f;
#pragma unroll
      for (int c0 = 0; c0 < 128; c0 += 32) {
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
        for (int jj = 0; jj < 32; jj++) {
          const int a = c0 + jj;
          const float d = __uint_as_float(v[jj]);
          if (a == 0) {
            // F = 2 (H0 - D): |F| / 2 = |H0 - D|, F < 0 iff H0 < D
            const float half = H0 - d;
            best = fmaxf(best, fmaf(fabsf(half), 256.f, 254.f + (half < 0.f ? 1.f : 0.f)));
          } else {
            // F = -2 D: the key is D 256 + (254 - 2a) + 1 when D > 0 (F < 0)
            // and -D 256 + (254 - 2a) when D < 0, the larger of the two;
            // D = 0 gives 255 - 2a, below column 0's key whenever every F
            // is 0, so its low bit never decides
            const float c = (float)(254 - 2 * a);
            best = fmaxf(best, fmaxf(fmaf(d, 256.f, c + 1.f), fmaf(d, -256.f, c)));
          }
        }
      }
      const int kb = (int)best;
      const uint32_t byte = (uint32_t)(127 - ((kb & 255) >> 1)) | ((uint32_t)(kb & 1) << 7);
      if (g < total) r_out[g] = (uint8_t)byte;
    }
    tc_fence_before();
    group_sync(grp);
  }
  if (!ok && tid == 0) atomicAdd(&g_rm_tc_timeouts, 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tslot), "r"(RMTC_TMEM_COLS));
}

template <int LEVEL>
cudaError_t rm_tc_level(int64_t count, const uint64_t* w, uint8_t* r, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_rm_tc<LEVEL>, cudaFuncAttributeMaxDynamicSharedMemorySize, RMTC_SMEM);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int64_t tiles = (count * Level<LEVEL>::n1 + RMTC_ROWS - 1) / RMTC_ROWS;
  // one 160 KB block of four groups per SM, holding all 512 tensor-memory columns
  const int64_t grid = std::min<int64_t>((tiles + RMTC_GROUPS - 1) / RMTC_GROUPS, (int64_t)sms);
  k_rm_tc<LEVEL><<<(unsigned)grid, 128 * RMTC_GROUPS, RMTC_SMEM, st>>>(count, w, r);
  return cudaGetLastError();
}

template <int LEVEL>
cudaError_t rm_fht_level(int64_t count, const uint64_t* w, uint8_t* r, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  const int64_t threads = 2 * count * Level<LEVEL>::n1;
  const int64_t blocks = (threads + STAGE_THREADS - 1) / STAGE_THREADS;
  k_stage_rm<LEVEL><<<(unsigned)blocks, STAGE_THREADS, 0, st>>>(count, w, r);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rm_decode(int level, int64_t count, const uint64_t* w, uint8_t* r, bool tensor_cores,
                             cudaStream_t st) {
  switch (level) {
    case 1: return tensor_cores ? rm_tc_level<1>(count, w, r, st) : rm_fht_level<1>(count, w, r, st);
    case 3: return tensor_cores ? rm_tc_level<3>(count, w, r, st) : rm_fht_level<3>(count, w, r, st);
    case 5: return tensor_cores ? rm_tc_level<5>(count, w, r, st) : rm_fht_level<5>(count, w, r, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t rm_tc_take_timeouts(int* out) {
  int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(out, g_rm_tc_timeouts, sizeof(int));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(g_rm_tc_timeouts, &zero, sizeof(int));
}

}  // namespace hqc

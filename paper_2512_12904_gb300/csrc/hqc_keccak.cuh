// Keccak-f[1600] and SHAKE256 for one message per thread (FIPS 202), the
// PRNG and hash behind HQC's sampler and its G and K functions (Sec. II-A),
// batched as the paper batches its Keccak calls (Sec. III-C).
//
// State: 25 lanes a[x + 5 y] of 64 bits, held in registers.  The round
// constants (FIPS 202 Algorithm 5/6) and the rho offsets (Algorithm 2) are
// computed at compile time from their definitions.
#pragma once
#include <cstdint>

namespace hqc {

constexpr int SHAKE256_RATE = 136;           // bytes
constexpr int SHAKE256_RATE_WORDS = 17;      // 64-bit lanes absorbed per block

// rc(t): the degree-8 LFSR x^8 + x^6 + x^5 + x^4 + 1 stepped t times from
// R = 1000 0000; bit i of R below is the register's i-th bit.
__host__ __device__ constexpr uint32_t keccak_rc_bit(int t) {
  const int steps = t % 255;
  uint32_t R = 1u;
  for (int i = 0; i < steps; i++) {
    R <<= 1u;
    const uint32_t top = (R >> 8) & 1u;
    R ^= top * 0x71u;   // feedback into bits 0, 4, 5, 6
    R &= 0xFFu;
  }
  return R & 1u;
}

__host__ __device__ constexpr uint64_t keccak_round_constant(int ir) {
  uint64_t rc = 0;
  for (int j = 0; j <= 6; j++)
    if (keccak_rc_bit(j + 7 * ir)) rc |= 1ull << ((1 << j) - 1);
  return rc;
}

// rho offset of lane (x, y): the walk (x, y) -> (y, 2x + 3y) from (1, 0)
// assigns (t + 1)(t + 2) / 2 mod 64 at step t.
__host__ __device__ constexpr int keccak_rho(int lane) {
  if (lane == 0) return 0;
  int x = 1, y = 0;
  for (int t = 0; t < 24; t++) {
    if (x + 5 * y == lane) return ((t + 1) * (t + 2) / 2) % 64;
    const int nx = y, ny = (2 * x + 3 * y) % 5;
    x = nx;
    y = ny;
  }
  return 0;
}

static __constant__ uint64_t c_keccak_rc[24] = {
    keccak_round_constant(0),  keccak_round_constant(1),  keccak_round_constant(2),  keccak_round_constant(3),
    keccak_round_constant(4),  keccak_round_constant(5),  keccak_round_constant(6),  keccak_round_constant(7),
    keccak_round_constant(8),  keccak_round_constant(9),  keccak_round_constant(10), keccak_round_constant(11),
    keccak_round_constant(12), keccak_round_constant(13), keccak_round_constant(14), keccak_round_constant(15),
    keccak_round_constant(16), keccak_round_constant(17), keccak_round_constant(18), keccak_round_constant(19),
    keccak_round_constant(20), keccak_round_constant(21), keccak_round_constant(22), keccak_round_constant(23)};

template <int R>
__device__ __forceinline__ uint64_t rotl64c(uint64_t v) {
  if constexpr ((R & 63) == 0) {
    return v;
  } else {
    return (v << (R & 63)) | (v >> (64 - (R & 63)));
  }
}

// One round on the registers a[25]: theta, rho + pi, chi, iota.
__device__ __forceinline__ void keccak_round(uint64_t (&a)[25], uint64_t rc) {
  uint64_t C[5];
#pragma unroll
  for (int x = 0; x < 5; x++) C[x] = a[x] ^ a[x + 5] ^ a[x + 10] ^ a[x + 15] ^ a[x + 20];
#pragma unroll
  for (int x = 0; x < 5; x++) {
    const uint64_t D = C[(x + 4) % 5] ^ rotl64c<1>(C[(x + 1) % 5]);
#pragma unroll
    for (int y = 0; y < 5; y++) a[x + 5 * y] ^= D;
  }
  // pi moves lane (x, y) to (y, 2x + 3y) after its rho rotation
  uint64_t b[25];
#define HQC_RHO_PI(x, y) b[(y) + 5 * ((2 * (x) + 3 * (y)) % 5)] = rotl64c<keccak_rho((x) + 5 * (y))>(a[(x) + 5 * (y)]);
#define HQC_RHO_PI_ROW(y) HQC_RHO_PI(0, y) HQC_RHO_PI(1, y) HQC_RHO_PI(2, y) HQC_RHO_PI(3, y) HQC_RHO_PI(4, y)
  HQC_RHO_PI_ROW(0) HQC_RHO_PI_ROW(1) HQC_RHO_PI_ROW(2) HQC_RHO_PI_ROW(3) HQC_RHO_PI_ROW(4)
#undef HQC_RHO_PI_ROW
#undef HQC_RHO_PI
#pragma unroll
  for (int y = 0; y < 5; y++)
#pragma unroll
    for (int x = 0; x < 5; x++) a[x + 5 * y] = b[x + 5 * y] ^ (~b[(x + 1) % 5 + 5 * y] & b[(x + 2) % 5 + 5 * y]);
  a[0] ^= rc;
}

__device__ __forceinline__ void keccak_f1600(uint64_t (&a)[25]) {
#pragma unroll 2
  for (int ir = 0; ir < 24; ir++) keccak_round(a, c_keccak_rc[ir]);
}

// SHAKE256 absorb of a `len`-byte message whose little-endian 64-bit word q
// is word(q) (bytes at or past len inside the last word must be zero):
// M || 1111 || pad10*1 in 136-byte blocks.  word(q) is called once per q,
// in increasing q.  The words of block b + 1 are fetched before block b is
// permuted, so their loads overlap the permutation.  len is the same for
// every thread of a launch, so the control flow is uniform.
template <class WordFn>
__device__ __forceinline__ void shake256_absorb(uint64_t (&a)[25], int len, WordFn word) {
#pragma unroll
  for (int i = 0; i < 25; i++) a[i] = 0;
  const int nblocks = len / SHAKE256_RATE + 1;
  const int qpad = len >> 3;
  auto fetch = [&](int blk, uint64_t (&w)[SHAKE256_RATE_WORDS]) {
#pragma unroll
    for (int i = 0; i < SHAKE256_RATE_WORDS; i++) {
      const int q = blk * SHAKE256_RATE_WORDS + i;
      w[i] = q < qpad || (q == qpad && (len & 7)) ? word(q) : 0ull;
    }
  };
  uint64_t w[SHAKE256_RATE_WORDS];
  fetch(0, w);
  for (int blk = 0; blk < nblocks; blk++) {
#pragma unroll
    for (int i = 0; i < SHAKE256_RATE_WORDS; i++) {
      const int q = blk * SHAKE256_RATE_WORDS + i;
      uint64_t wv = w[i];
      if (q == qpad) wv ^= 0x1Full << (8 * (len & 7));
      if (i == SHAKE256_RATE_WORDS - 1 && blk == nblocks - 1) wv ^= 0x80ull << 56;
      a[i] ^= wv;
    }
    if (blk + 1 < nblocks) fetch(blk + 1, w);
    keccak_f1600(a);
  }
}

// ---------------------------------------------------------------------------
// The same permutation on a lane pair: lane h (= lane & 1) of the pair holds
// the h-th 32-bit half of each of the 25 lanes (h = 0: bits 0..31), so a
// batch of messages keeps twice as many warps busy for the same ALU work.
// A 64-bit rotation by r needs the partner's half of the lane, one shuffle:
//   r in [1, 31]:  mine' = funnel_l(other, mine, r)   (both halves alike)
//   r in [33, 63]: mine' = funnel_l(mine, other, r - 32)
// Every lane of the warp must take part (the shuffles name all 32 lanes).
// ---------------------------------------------------------------------------
template <int R>
__device__ __forceinline__ uint32_t rotl64_half(uint32_t mine, uint32_t other) {
  constexpr int r = R & 63;
  if constexpr (r == 0) {
    return mine;
  } else if constexpr (r < 32) {
    return __funnelshift_l(other, mine, r);
  } else if constexpr (r == 32) {
    return other;
  } else {
    return __funnelshift_l(mine, other, r - 32);
  }
}

__device__ __forceinline__ void keccak_round_pair(uint32_t (&a)[25], uint32_t rc_half) {
  uint32_t C[5], Cp[5];
#pragma unroll
  for (int x = 0; x < 5; x++) C[x] = a[x] ^ a[x + 5] ^ a[x + 10] ^ a[x + 15] ^ a[x + 20];
#pragma unroll
  for (int x = 0; x < 5; x++) Cp[x] = __shfl_xor_sync(0xFFFFFFFFu, C[x], 1);
#pragma unroll
  for (int x = 0; x < 5; x++) {
    const uint32_t D = C[(x + 4) % 5] ^ rotl64_half<1>(C[(x + 1) % 5], Cp[(x + 1) % 5]);
#pragma unroll
    for (int y = 0; y < 5; y++) a[x + 5 * y] ^= D;
  }
  uint32_t p[25];
#pragma unroll
  for (int i = 0; i < 25; i++) p[i] = keccak_rho(i) % 64 == 0 ? 0u : __shfl_xor_sync(0xFFFFFFFFu, a[i], 1);
  uint32_t b[25];
#define HQC_RHO_PI_H(x, y) \
  b[(y) + 5 * ((2 * (x) + 3 * (y)) % 5)] = rotl64_half<keccak_rho((x) + 5 * (y))>(a[(x) + 5 * (y)], p[(x) + 5 * (y)]);
#define HQC_RHO_PI_H_ROW(y) HQC_RHO_PI_H(0, y) HQC_RHO_PI_H(1, y) HQC_RHO_PI_H(2, y) HQC_RHO_PI_H(3, y) HQC_RHO_PI_H(4, y)
  HQC_RHO_PI_H_ROW(0) HQC_RHO_PI_H_ROW(1) HQC_RHO_PI_H_ROW(2) HQC_RHO_PI_H_ROW(3) HQC_RHO_PI_H_ROW(4)
#undef HQC_RHO_PI_H_ROW
#undef HQC_RHO_PI_H
#pragma unroll
  for (int y = 0; y < 5; y++)
#pragma unroll
    for (int x = 0; x < 5; x++) a[x + 5 * y] = b[x + 5 * y] ^ (~b[(x + 1) % 5 + 5 * y] & b[(x + 2) % 5 + 5 * y]);
  a[0] ^= rc_half;
}

__device__ __forceinline__ void keccak_f1600_pair(uint32_t (&a)[25], uint32_t h) {
#pragma unroll 2
  for (int ir = 0; ir < 24; ir++) {
    const uint64_t rc = c_keccak_rc[ir];
    keccak_round_pair(a, h ? (uint32_t)(rc >> 32) : (uint32_t)rc);
  }
}

// shake256_absorb on a lane pair: word(q) returns the whole 64-bit word
// (both lanes of the pair read the same address) and each lane keeps its
// half.
template <class WordFn>
__device__ __forceinline__ void shake256_absorb_pair(uint32_t (&a)[25], int len, uint32_t h, WordFn word) {
#pragma unroll
  for (int i = 0; i < 25; i++) a[i] = 0;
  const int nblocks = len / SHAKE256_RATE + 1;
  const int qpad = len >> 3;
  auto fetch = [&](int blk, uint32_t (&wh)[SHAKE256_RATE_WORDS]) {
#pragma unroll
    for (int i = 0; i < SHAKE256_RATE_WORDS; i++) {
      const int q = blk * SHAKE256_RATE_WORDS + i;
      const uint64_t wv = q < qpad || (q == qpad && (len & 7)) ? word(q) : 0ull;
      wh[i] = h ? (uint32_t)(wv >> 32) : (uint32_t)wv;
    }
  };
  uint32_t wh[SHAKE256_RATE_WORDS];
  fetch(0, wh);
  for (int blk = 0; blk < nblocks; blk++) {
#pragma unroll
    for (int i = 0; i < SHAKE256_RATE_WORDS; i++) {
      const int q = blk * SHAKE256_RATE_WORDS + i;
      uint64_t pad = 0;
      if (q == qpad) pad ^= 0x1Full << (8 * (len & 7));
      if (i == SHAKE256_RATE_WORDS - 1 && blk == nblocks - 1) pad ^= 0x80ull << 56;
      a[i] ^= wh[i] ^ (h ? (uint32_t)(pad >> 32) : (uint32_t)pad);
    }
    if (blk + 1 < nblocks) fetch(blk + 1, wh);
    keccak_f1600_pair(a, h);
  }
}

}  // namespace hqc

// The KEM's K function of one item on a lane pair (Sec. II-A: the
// domain-separated hash of HHK with implicit rejection), shared by the
// stand-alone K kernel and the fused re-encryption kernel of decapsulation.
//   K = SHAKE256(x || U || V || salt || 0x04)[0:32]
// x = m (the decrypted message) or sigma (the key's rejection secret), U
// the ceil(n/8) bytes of u with bits >= n cleared, V the n1 n2 / 8 bytes of
// v.
#pragma once
#include <cstdint>

#include "hqc_keccak.cuh"

namespace hqc {

constexpr int KEM_SALT = 16;
constexpr int KEM_KBYTES = 32;

// Lane half h of the pair absorbs the message into the 32-bit halves a[]
// of the state (keccak_f1600_pair); both lanes of the pair must call it
// together.  x = m where keep is all ones, sigma where keep is zero (a mask,
// not a branch).  Message words: x (k/8 words), then the u words up to the
// one that holds the last byte of U (bits >= n cleared), then, from word P1
// on, a stream shifted by r = (k + ceil(n/8)) mod 8 bytes over T = [last u
// word, v[0..W_v), salt, 0x04]: word P1 + i = (T[i+1] << 8r) | (T[i] >>
// (64 - 8r)).  The previous T word is carried, so each message word costs
// one load.  On return a[0..8) hold K as 32-bit halves: K word i = a[i]
// of lane 0 | a[i] of lane 1 << 32.
template <class LV>
__device__ __forceinline__ void kem_K_pair(uint32_t h, uint64_t keep, const uint64_t* __restrict__ mrow,
                                           const uint64_t* __restrict__ grow, const uint64_t* __restrict__ urow,
                                           const uint64_t* __restrict__ vrow, const uint64_t* __restrict__ srow,
                                           uint32_t (&a)[25]) {
  constexpr int KW = LV::k / 8;
  constexpr int UB = (LV::n + 7) / 8, VB = LV::n1 * LV::n2 / 8;
  constexpr int OFF_V = LV::k + UB;
  constexpr int LEN = OFF_V + VB + KEM_SALT + 1;
  constexpr int P1 = OFF_V / 8, R8 = 8 * (OFF_V % 8);
  constexpr int NT = LV::W_v + 4;  // T[1..NT): v words, two salt words, the domain byte
  static_assert(P1 == KW + LV::W_u - 1 && R8 > 0, "U ends inside its last word");
  constexpr uint64_t UMASK = (LV::n & 63) ? (1ull << (LV::n & 63)) - 1ull : ~0ull;
  // T[0] = last u word placed so that T[0] >> (64 - 8r) is its U bytes
  uint64_t prev = (__ldg(urow + LV::W_u - 1) & UMASK) << (64 - R8);
  auto tword = [&](int i) {  // T[i], i >= 1
    return i <= LV::W_v ? __ldg(vrow + i - 1) : i <= LV::W_v + 2 ? __ldg(srow + i - 1 - LV::W_v) : 0x04ull;
  };
  shake256_absorb_pair(a, LEN, h, [&](int q) {
    uint64_t w;
    if (q < KW) {
      w = (__ldg(mrow + q) & keep) | (__ldg(grow + q) & ~keep);
    } else if (q < P1) {
      w = __ldg(urow + q - KW);
    } else {
      const int i = q - P1 + 1;
      const uint64_t cur = i < NT ? tword(i) : 0ull;
      w = (cur << R8) | (prev >> (64 - R8));
      prev = cur;
    }
    return w;
  });
}

}  // namespace hqc

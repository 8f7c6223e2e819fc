// Batched HQC.PKE key generation core (Algorithm 3: s = x + h*y) and
// encryption (Algorithm 1: u = r1 + h*r2, v = first n1*n2 bits of
// mG + s*r2 + e) on the same rotate-XOR product as decryption.  One warp
// per item; used to build synthetic ciphertexts on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <utility>

#include "hqc_device.cuh"
#include "hqc_internal.h"

namespace hqc {

constexpr int ENC_THREADS = 256;  // key generation

// Encryption: as many warps per block as shared memory holds (one u2 region
// per warp), one block per SM.
template <int LEVEL> struct EncBound;
template <> struct EncBound<1> { static constexpr int threads = 1024; };
template <> struct EncBound<3> { static constexpr int threads = 704; };
template <> struct EncBound<5> { static constexpr int threads = 448; };

// Products of the RS generator's coefficients by a byte, in shared memory
// for the encoder: lane l of a warp owns coefficients c = l + 32 x, and
// g_c * b = T[x][0][b & 15] ^ T[x][1][b >> 4] with T[x][h][j] = g_c *
// (j << 4 h).  Entry (x, h, j) of lane l sits at byte ((2 x + h) 16 + j) 32
// + l: the warp looks up one j (the feedback byte is the same for every
// lane), its 32 bytes fill 8 words in 8 different banks, so the access
// pattern does not depend on the (secret) byte.  NX <= 2: 2 KB per block.
constexpr int ENC_GF_BYTES = 2 * 1024;

// RS generator g(x) = prod_{i=1}^{2 delta} (x - alpha^i) over GF(2^8) mod
// x^8 + x^4 + x^3 + x^2 + 1, alpha = x, computed at compile time; the
// encoder uses the logs of its coefficients (511 for a zero coefficient).
__host__ __device__ constexpr uint32_t ce_gf_mul(uint32_t a, uint32_t b) {
  uint32_t r = 0;
  for (int i = 0; i < 8; i++) {
    if ((b >> i) & 1u) r ^= a;
    a <<= 1;
    if (a & 0x100u) a ^= 0x11Du;
  }
  return r;
}
__host__ __device__ constexpr uint32_t ce_gf_pow_alpha(int e) {
  uint32_t r = 1;
  for (int i = 0; i < e; i++) r = ce_gf_mul(r, 2u);
  return r;
}
template <int NR>
struct RsGenLog {
  uint32_t lg[NR + 1];
  __host__ __device__ constexpr RsGenLog() : lg() {
    uint32_t g[NR + 1] = {};
    g[0] = 1;
    for (int i = 1; i <= NR; i++) {
      const uint32_t root = ce_gf_pow_alpha(i);
      for (int d = i; d >= 0; d--) g[d] = (d > 0 ? g[d - 1] : 0u) ^ ce_gf_mul(g[d], root);
    }
    uint32_t logt[256] = {};
    uint32_t p = 1;
    for (int e = 0; e < 255; e++) {
      logt[p] = (uint32_t)e;
      p = ce_gf_mul(p, 2u);
    }
    for (int d = 0; d <= NR; d++) lg[d] = g[d] ? logt[g[d]] : 511u;
  }
};
template <int NR, int C>
struct RsGenAt {
  static constexpr uint32_t lg = RsGenLog<NR>().lg[C];
  static constexpr uint32_t value = lg == 511u ? 0u : ce_gf_pow_alpha((int)lg);
};
// g_c for a runtime c (0 past the degree NR), as a chain of selects between
// compile-time immediates (no table in memory)
template <int NR, int... C>
__device__ __forceinline__ uint32_t rs_gen_select(int c, std::integer_sequence<int, C...>) {
  uint32_t v = 0u;
  ((v = (c == C) ? RsGenAt<NR, C>::value : v), ...);
  return v;
}

// Fill the encoder's product tables (all threads of the block, then
// __syncthreads).  Only the NR parity coefficients c < NR are used.
template <class LV>
__device__ inline void enc_tab_init(uint8_t* tab, int tid, int nthreads) {
  constexpr int NX = cdiv(LV::NR, 32);
  static_assert(NX <= 2, "two coefficient columns per lane at most");
  for (int i = tid; i < NX * 1024; i += nthreads) {
    const int l = i & 31, j = (i >> 5) & 15, h = (i >> 9) & 1, x = i >> 10;
    const uint32_t g = rs_gen_select<LV::NR>(l + 32 * x, std::make_integer_sequence<int, LV::NR>{});
    tab[i] = (uint8_t)ce_gf_mul(g, h ? (uint32_t)j << 4 : (uint32_t)j);
  }
}

// Product of the dense row `dense` by the support `supp` (w entries, may
// be invalid -> masked) over the full n bits, left in u2[0, N32) with the
// bits >= n of the last word cleared.
template <class LV, int W, bool MASKED = true>
__device__ __forceinline__ void full_product_to_smem(uint32_t* u2, uint32_t* sup, const uint64_t* dense,
                                                     const uint32_t* supp, int lane) {
  constexpr int N32 = LV::N32, R = LV::n & 31, WPT = LV::WPT_FULL;
  constexpr uint32_t LAST = R ? (1u << R) - 1u : ~0u;
  load_supports<LV::n, W>(sup, supp, lane);
  build_doubled<LV::n, LV::W_u_pitch, LV::U2W_FULL>(u2, dense, lane);
  uint32_t acc[WPT];
  rot_xor_product<WPT, W, MASKED>(u2, sup, lane * WPT, acc);
  __syncwarp();
#pragma unroll
  for (int k = 0; k < WPT; k++) {
    const int i = lane * WPT + k;
    if (i < N32) u2[i] = i == N32 - 1 ? (acc[k] & LAST) : acc[k];
  }
  __syncwarp();
}

// The W_v32 words of the product truncated to n1 n2 bits, left in
// u2[0, W_v32).
template <class LV, int W, bool MASKED>
__device__ __forceinline__ void truncated_product_to_smem(uint32_t* u2, const uint32_t* sup, int lane) {
  using PS = ProductStrips<LV::level>;
  constexpr int WPT = PS::MAXLEN;
  const int w0 = PS::start(lane), wn = PS::len(lane);
  uint32_t acc[WPT];
  rot_xor_product<WPT, W, MASKED>(u2, sup, w0, acc);
  __syncwarp();
#pragma unroll
  for (int k = 0; k < WPT; k++) {
    const int i = w0 + k;
    if (k < wn && i < LV::W_v32) u2[i] = acc[k];
  }
  __syncwarp();
}

// XOR the bits of a W-entry support into out (NBITS bits).  Lanes writing
// at once would collide in banks according to the secret positions, so the
// entries are applied one per step by lane 0 alone, with one shared load
// and one store every step; an entry at or past NBITS adds 0 to word 0.
// The accesses and their timing do not depend on the positions.
template <int W, int NBITS>
__device__ __forceinline__ void xor_support_bits(uint32_t* out, const uint32_t* supp, int lane) {
  constexpr int NJ = cdiv(W, 32);
  uint32_t pj[NJ];
#pragma unroll
  for (int j = 0; j < NJ; j++) pj[j] = lane + 32 * j < W ? __ldg(supp + lane + 32 * j) : 0u;
#pragma unroll
  for (int t = 0; t < W; t++) {
    const uint32_t p = __shfl_sync(FULL_MASK, pj[t >> 5], t & 31);
    const bool ok = p < (uint32_t)NBITS;
    const uint32_t q = sel(ok, p >> 5, 0u);
    const uint32_t bit = sel(ok, 1u << (p & 31), 0u);
    if (lane == 0) out[q] ^= bit;
  }
  __syncwarp();
}

template <int PITCH64, int NWORDS32>
__device__ __forceinline__ void store_row(uint64_t* dst, const uint32_t* src, int lane) {
  uint32_t* d32 = reinterpret_cast<uint32_t*>(dst);
  for (int i = lane; i < 2 * PITCH64; i += 32) d32[i] = i < NWORDS32 ? src[i] : 0u;
}

template <int LEVEL>
__global__ void __launch_bounds__(ENC_THREADS) k_keygen(int64_t nkeys, const uint64_t* __restrict__ h,
                                                       const uint32_t* __restrict__ x, const uint32_t* __restrict__ y,
                                                       uint64_t* __restrict__ s) {
  using LV = Level<LEVEL>;
  constexpr int WARP_W = LV::U2W_FULL + LV::WP;
  extern __shared__ __align__(16) uint8_t smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t it = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (it >= nkeys) return;
  uint32_t* u2 = reinterpret_cast<uint32_t*>(smem) + warp * WARP_W;
  uint32_t* sup = u2 + LV::U2W_FULL;
  full_product_to_smem<LV, LV::w>(u2, sup, h + it * LV::W_u_pitch, y + it * LV::w, lane);
  xor_support_bits<LV::w, LV::n>(u2, x + it * LV::w, lane);
  store_row<LV::W_u_pitch, LV::N32>(s + it * LV::W_u_pitch, u2, lane);
}

// Codeword bits of one byte B = a + 128 b, word t of 4: bit q is
// b ^ parity(a & (32 t + q)).
__device__ __forceinline__ uint32_t rm_codeword_word(uint32_t B, int t) {
  const uint32_t a = B & 127u;
  uint32_t w = 0;
  w ^= 0xAAAAAAAAu & (0u - (a & 1u));
  w ^= 0xCCCCCCCCu & (0u - ((a >> 1) & 1u));
  w ^= 0xF0F0F0F0u & (0u - ((a >> 2) & 1u));
  w ^= 0xFF00FF00u & (0u - ((a >> 3) & 1u));
  w ^= 0xFFFF0000u & (0u - ((a >> 4) & 1u));
  w ^= 0u - ((a >> 5) & 1u & (uint32_t)t);
  w ^= 0u - ((a >> 6) & 1u & ((uint32_t)t >> 1));
  w ^= 0u - (B >> 7);
  return w;
}

// RS systematic encoding of the k-byte row m by the division register (one
// warp; lane owns parity coefficient c = lane + 32 x, tab the block's
// product tables), written as the codeword (parity || message) to cw.
template <class LV>
__device__ __forceinline__ void enc_rs_encode(const uint8_t* __restrict__ mrow, const uint8_t* tab, int lane,
                                              uint8_t* cw) {
  constexpr int NR = LV::NR, k = LV::k, NX = cdiv(NR, 32);
  uint32_t par[NX];
#pragma unroll
  for (int x = 0; x < NX; x++) par[x] = 0;
  const uint8_t* tl = tab + lane;
  for (int i = k - 1; i >= 0; i--) {
    const uint32_t top = __shfl_sync(FULL_MASK, par[(NR - 1) / 32], (NR - 1) % 32);
    const uint32_t fb = (uint32_t)mrow[i] ^ top;  // the feedback byte, the same in every lane
    const uint32_t lo = (fb & 15u) << 5, hi = 512u + ((fb >> 4) << 5);
    uint32_t nxt[NX];
#pragma unroll
    for (int x = 0; x < NX; x++) {
      const uint32_t up = __shfl_up_sync(FULL_MASK, par[x], 1);
      const uint32_t carry = x > 0 ? __shfl_sync(FULL_MASK, par[x > 0 ? x - 1 : 0], 31) : 0u;
      const int c = lane + 32 * x;
      const uint32_t prev = lane == 0 ? carry : up;
      const uint32_t gfb = (uint32_t)tl[1024 * x + lo] ^ (uint32_t)tl[1024 * x + hi];  // g_c * fb
      nxt[x] = c < NR ? (prev ^ gfb) : 0u;
    }
#pragma unroll
    for (int x = 0; x < NX; x++) par[x] = nxt[x];
  }
#pragma unroll
  for (int x = 0; x < NX; x++) {
    const int c = lane + 32 * x;
    if (c < NR) cw[c] = (uint8_t)par[x];
  }
  for (int i = lane; i < k; i += 32) cw[NR + i] = mrow[i];
}

// Duplicated RM(1,7) encoding of every codeword byte (at u2 + W_v32), added
// into the truncated product in u2; NT threads, tid in [0, NT).
template <class LV, int NT>
__device__ __forceinline__ void enc_rm_encode(uint32_t* u2, int tid) {
  const uint8_t* cw = reinterpret_cast<const uint8_t*>(u2 + LV::W_v32);
  for (int j = tid; j < LV::n1; j += NT) {
    const uint32_t B = cw[j];
#pragma unroll
    for (int t = 0; t < 4; t++) {
      const uint32_t cwt = rm_codeword_word(B, t);
#pragma unroll
      for (int rcp = 0; rcp < LV::mult; rcp++) u2[j * (LV::n2 / 32) + 4 * rcp + t] ^= cwt;
    }
  }
}

// One item by one warp (its key index already checked): u = r1 + h r2 and
// v = first n1 n2 bits of mG + s r2 + e in the warp's shared slice u2 /
// sup.  CMP: instead of storing (u, v), compare them with (u_in, v_in) on
// the n and n1 n2 bits (padding of u_in ignored); returns true, on every
// lane, when they match (the re-encryption check of decapsulation).
// VALID: the supports are known to hold distinct positions < n (drawn by
// the sampler), so the product takes the unmasked two-entries-per-pass
// path.
template <class LV, bool CMP, bool VALID>
__device__ __forceinline__ bool encrypt_item(const uint8_t* smem, uint32_t* u2, uint32_t* sup, int lane, int64_t it,
                                             int64_t key, const uint64_t* __restrict__ h,
                                             const uint64_t* __restrict__ s, const uint8_t* __restrict__ m,
                                             const uint32_t* __restrict__ r1, const uint32_t* __restrict__ r2,
                                             const uint32_t* __restrict__ e, uint64_t* __restrict__ u,
                                             uint64_t* __restrict__ v, const uint64_t* __restrict__ u_in,
                                             const uint64_t* __restrict__ v_in) {
  // u = r1 + h * r2
  full_product_to_smem<LV, LV::wr, !VALID>(u2, sup, h + key * LV::W_u_pitch, r2 + it * LV::wr, lane);
  xor_support_bits<LV::wr, LV::n>(u2, r1 + it * LV::wr, lane);
  uint32_t diff = 0;
  if constexpr (CMP) {
    constexpr int R = LV::n & 31;
    const uint32_t* ui = reinterpret_cast<const uint32_t*>(u_in + it * LV::W_u_pitch);
    for (int i = lane; i < LV::N32; i += 32) {
      uint32_t x = __ldg(ui + i);
      if (R && i == LV::N32 - 1) x &= (1u << R) - 1u;
      diff |= x ^ u2[i];
    }
  } else {
    store_row<LV::W_u_pitch, LV::N32>(u + it * LV::W_u_pitch, u2, lane);
  }
  __syncwarp();

  // s * r2, truncated to n1*n2 bits, plus e
  build_doubled<LV::n, LV::W_u_pitch, LV::U2W_FULL>(u2, s + key * LV::W_u_pitch, lane);
  truncated_product_to_smem<LV, LV::wr, !VALID>(u2, sup, lane);
  xor_support_bits<LV::we, LV::n1 * LV::n2>(u2, e + it * LV::we, lane);

  enc_rs_encode<LV>(m + it * LV::k, smem, lane, reinterpret_cast<uint8_t*>(u2 + LV::W_v32));
  __syncwarp();
  enc_rm_encode<LV, 32>(u2, lane);
  __syncwarp();
  bool same = false;
  if constexpr (CMP) {
    const uint32_t* vi = reinterpret_cast<const uint32_t*>(v_in + it * LV::W_v);
    for (int i = lane; i < LV::W_v32; i += 32) diff |= __ldg(vi + i) ^ u2[i];
    same = !__any_sync(FULL_MASK, diff != 0u);
  } else {
    store_row<LV::W_v, LV::W_v32>(v + it * LV::W_v, u2, lane);
  }
  __syncwarp();
  return same;
}

// Persistent: each warp encrypts items it, it + (warps in the grid), ...
// (encrypt_item); with CMP it stores ok[item] = 1 on a match, 0 otherwise.
template <int LEVEL, bool CMP, bool VALID>
__global__ void __launch_bounds__(EncBound<LEVEL>::threads, 1) k_encrypt(int64_t count, const uint64_t* __restrict__ h,
                                                        const uint64_t* __restrict__ s, int64_t nkeys,
                                                        const int32_t* __restrict__ key_idx,
                                                        const uint8_t* __restrict__ m, const uint32_t* __restrict__ r1,
                                                        const uint32_t* __restrict__ r2, const uint32_t* __restrict__ e,
                                                        uint64_t* __restrict__ u, uint64_t* __restrict__ v,
                                                        const uint64_t* __restrict__ u_in,
                                                        const uint64_t* __restrict__ v_in, uint32_t* __restrict__ ok) {
  using LV = Level<LEVEL>;
  constexpr int WARP_W = LV::U2W_FULL + LV::WP_R;
  extern __shared__ __align__(16) uint8_t smem[];
  enc_tab_init<LV>(smem, threadIdx.x, blockDim.x);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t* u2 = reinterpret_cast<uint32_t*>(smem + ENC_GF_BYTES) + warp * WARP_W;
  uint32_t* sup = u2 + LV::U2W_FULL;
  for (int64_t it = (int64_t)blockIdx.x * nw + warp; it < count; it += (int64_t)gridDim.x * nw) {
    const uint32_t ki = (uint32_t)key_idx[it];
    if (ki >= (uint64_t)nkeys) continue;  // skipped item: outputs untouched (the index is public)
    const bool same =
        encrypt_item<LV, CMP, VALID>(smem, u2, sup, lane, it, (int64_t)ki, h, s, m, r1, r2, e, u, v, u_in, v_in);
    if (CMP && lane == 0) ok[it] = same ? 1u : 0u;
  }
}

// Two-warp teams (HQC-5): the team's warps share one doubled operand and
// each computes half of both products' words (strips of ETeam::WPT2 words
// over 64 lanes), so a block holds twice the items in shared memory.  The
// RS encoder runs on the team's first warp; members synchronise with a
// 64-thread named barrier.
template <class LV>
struct ETeam {
  static constexpr int WPT2 = odd_at_least(cdiv(cmax(LV::N32, LV::W_v32), 64));
  static constexpr int U2W = round_up(cmax(cdiv(2 * LV::n, 32), 64 * WPT2 + (LV::n >> 5) + 1), 4);
  static constexpr int WORDS = U2W + LV::WP_R + 4;  // u2, supports, the team's compare flag
  static_assert(LV::W_v32 + cdiv(LV::n1, 4) <= U2W, "codeword bytes fit after the product");
};
template <int LEVEL> struct EncTeamBound { static constexpr int threads = 896; };

template <int LEVEL, bool CMP, bool VALID>
__global__ void __launch_bounds__(EncTeamBound<LEVEL>::threads, 1)
    k_encrypt_team(int64_t count, const uint64_t* __restrict__ h, const uint64_t* __restrict__ s, int64_t nkeys,
                   const int32_t* __restrict__ key_idx, const uint8_t* __restrict__ m,
                   const uint32_t* __restrict__ r1, const uint32_t* __restrict__ r2, const uint32_t* __restrict__ e,
                   uint64_t* __restrict__ u, uint64_t* __restrict__ v, const uint64_t* __restrict__ u_in,
                   const uint64_t* __restrict__ v_in, uint32_t* __restrict__ ok) {
  using LV = Level<LEVEL>;
  using T = ETeam<LV>;
  constexpr int WPT = T::WPT2, RB = LV::n & 31;
  extern __shared__ __align__(16) uint8_t smem[];
  enc_tab_init<LV>(smem, threadIdx.x, blockDim.x);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int team = warp >> 1, wt = warp & 1, tid = wt * 32 + lane, nteams = blockDim.x >> 6;
  uint32_t* u2 = reinterpret_cast<uint32_t*>(smem + ENC_GF_BYTES) + team * T::WORDS;
  uint32_t* sup = u2 + T::U2W;
  uint32_t* flag = sup + LV::WP_R;
  const TeamSync sync{(uint32_t)(1 + team)};
  for (int64_t it = (int64_t)blockIdx.x * nteams + team; it < count; it += (int64_t)gridDim.x * nteams) {
    const uint32_t ki = (uint32_t)key_idx[it];
    // skipped item: outputs untouched; both warps of the team see the same
    // index, so they skip together and no barrier is left waiting
    if (ki >= (uint64_t)nkeys) continue;
    const int64_t key = (int64_t)ki;
    if (tid == 0) *flag = 0u;
    // u = r1 + h * r2
    load_supports<LV::n, LV::wr, 64>(sup, r2 + it * LV::wr, tid);
    build_doubled<LV::n, LV::W_u_pitch, T::U2W, 64, TeamSync>(u2, h + key * LV::W_u_pitch, tid, sync);
    uint32_t acc[WPT];
    rot_xor_product<WPT, LV::wr, !VALID>(u2, sup, tid * WPT, acc);
    sync();
#pragma unroll
    for (int kk = 0; kk < WPT; kk++) {
      const int i = tid * WPT + kk;
      if (i < LV::N32) u2[i] = (RB && i == LV::N32 - 1) ? (acc[kk] & ((1u << RB) - 1u)) : acc[kk];
    }
    sync();
    if (wt == 0) xor_support_bits<LV::wr, LV::n>(u2, r1 + it * LV::wr, lane);
    sync();
    uint32_t diff = 0;
    if constexpr (CMP) {
      const uint32_t* ui = reinterpret_cast<const uint32_t*>(u_in + it * LV::W_u_pitch);
      for (int i = tid; i < LV::N32; i += 64) {
        uint32_t x = __ldg(ui + i);
        if (RB && i == LV::N32 - 1) x &= (1u << RB) - 1u;
        diff |= x ^ u2[i];
      }
    } else {
      uint32_t* d32 = reinterpret_cast<uint32_t*>(u + it * LV::W_u_pitch);
      for (int i = tid; i < 2 * LV::W_u_pitch; i += 64) d32[i] = i < LV::N32 ? u2[i] : 0u;
    }
    sync();
    // s * r2, truncated to n1*n2 bits, plus e
    build_doubled<LV::n, LV::W_u_pitch, T::U2W, 64, TeamSync>(u2, s + key * LV::W_u_pitch, tid, sync);
    rot_xor_product<WPT, LV::wr, !VALID>(u2, sup, tid * WPT, acc);
    sync();
#pragma unroll
    for (int kk = 0; kk < WPT; kk++) {
      const int i = tid * WPT + kk;
      if (i < LV::W_v32) u2[i] = acc[kk];
    }
    sync();
    if (wt == 0) {
      xor_support_bits<LV::we, LV::n1 * LV::n2>(u2, e + it * LV::we, lane);
      enc_rs_encode<LV>(m + it * LV::k, smem, lane, reinterpret_cast<uint8_t*>(u2 + LV::W_v32));
    }
    sync();
    enc_rm_encode<LV, 64>(u2, tid);
    sync();
    if constexpr (CMP) {
      const uint32_t* vi = reinterpret_cast<const uint32_t*>(v_in + it * LV::W_v);
      for (int i = tid; i < LV::W_v32; i += 64) diff |= __ldg(vi + i) ^ u2[i];
      // every warp adds its result, 0 or 1: no branch on the comparison
      const uint32_t differs = __any_sync(FULL_MASK, diff != 0u) ? 1u : 0u;
      if (lane == 0) atomicOr(flag, differs);
      sync();
      if (tid == 0) ok[it] = *flag ? 0u : 1u;
    } else {
      uint32_t* d32 = reinterpret_cast<uint32_t*>(v + it * LV::W_v);
      for (int i = tid; i < 2 * LV::W_v; i += 64) d32[i] = u2[i];
    }
    sync();
  }
}

template <int LEVEL>
static cudaError_t keygen_level(int64_t nkeys, const uint64_t* h, const uint32_t* x, const uint32_t* y, uint64_t* s,
                                cudaStream_t st) {
  using LV = Level<LEVEL>;
  if (nkeys == 0) return cudaSuccess;
  const int wpb = ENC_THREADS / 32;
  const size_t sm = (size_t)wpb * (LV::U2W_FULL + LV::WP) * 4;
  cudaError_t e = cudaFuncSetAttribute(k_keygen<LEVEL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_keygen<LEVEL><<<(unsigned)((nkeys + wpb - 1) / wpb), ENC_THREADS, sm, st>>>(nkeys, h, x, y, s);
  return cudaGetLastError();
}

template <int LEVEL, bool CMP, bool VALID>
static cudaError_t encrypt_team_level(int64_t count, const uint64_t* h, const uint64_t* s, int64_t nkeys,
                                      const int32_t* ki, const uint8_t* m, const uint32_t* r1, const uint32_t* r2,
                                      const uint32_t* e, uint64_t* u, uint64_t* v, const uint64_t* u_in,
                                      const uint64_t* v_in, uint32_t* ok, cudaStream_t st) {
  using T = ETeam<Level<LEVEL>>;
  auto kern = k_encrypt_team<LEVEL, CMP, VALID>;
  int dev = 0, sms = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  constexpr size_t per_team = (size_t)T::WORDS * 4;
  int teams = (int)((optin - ENC_GF_BYTES) / per_team);
  if (teams > EncTeamBound<LEVEL>::threads / 64) teams = EncTeamBound<LEVEL>::threads / 64;
  if (teams > 15) teams = 15;  // named barriers 1..15
  if (teams < 1) return cudaErrorInvalidConfiguration;
  if (count < (int64_t)sms * teams) teams = (int)((count + sms - 1) / sms);
  const size_t sm = ENC_GF_BYTES + (size_t)teams * per_team;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (err != cudaSuccess) return err;
  int occ = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, teams * 64, sm);
  if (err != cudaSuccess) return err;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  int64_t grid = (int64_t)sms * occ;
  const int64_t need = (count + teams - 1) / teams;
  if (need < grid) grid = need;
  kern<<<(unsigned)grid, teams * 64, sm, st>>>(count, h, s, nkeys, ki, m, r1, r2, e, u, v, u_in, v_in, ok);
  return cudaGetLastError();
}

template <int LEVEL> struct EncUseTeam { static constexpr bool value = LEVEL == 5; };

template <int LEVEL, bool CMP, bool VALID>
static cudaError_t encrypt_level(int64_t count, const uint64_t* h, const uint64_t* s, int64_t nkeys, const int32_t* ki,
                                 const uint8_t* m, const uint32_t* r1, const uint32_t* r2, const uint32_t* e,
                                 uint64_t* u, uint64_t* v, const uint64_t* u_in, const uint64_t* v_in, uint32_t* ok,
                                 cudaStream_t st) {
  using LV = Level<LEVEL>;
  if (count == 0) return cudaSuccess;
  if constexpr (EncUseTeam<LEVEL>::value)
    return encrypt_team_level<LEVEL, CMP, VALID>(count, h, s, nkeys, ki, m, r1, r2, e, u, v, u_in, v_in, ok, st);
  auto kern = k_encrypt<LEVEL, CMP, VALID>;
  int dev = 0, sms = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  constexpr size_t per_warp = (size_t)(LV::U2W_FULL + LV::WP_R) * 4;
  int wpb = (int)((optin - ENC_GF_BYTES) / per_warp);
  if (wpb > EncBound<LEVEL>::threads / 32) wpb = EncBound<LEVEL>::threads / 32;
  if (wpb < 1) return cudaErrorInvalidConfiguration;
  // fewer items than one wave: fewer warps per block, so every SM gets work
  if (count < (int64_t)sms * wpb) wpb = (int)((count + sms - 1) / sms);
  const size_t sm = ENC_GF_BYTES + (size_t)wpb * per_warp;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (err != cudaSuccess) return err;
  int occ = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, wpb * 32, sm);
  if (err != cudaSuccess) return err;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  int64_t grid = (int64_t)sms * occ;
  const int64_t need = (count + wpb - 1) / wpb;
  if (need < grid) grid = need;
  kern<<<(unsigned)grid, wpb * 32, sm, st>>>(count, h, s, nkeys, ki, m, r1, r2, e, u, v, u_in, v_in, ok);
  return cudaGetLastError();
}

cudaError_t launch_keygen(int level, int64_t nkeys, const uint64_t* h, const uint32_t* x, const uint32_t* y,
                          uint64_t* s, cudaStream_t st) {
  switch (level) {
    case 1: return keygen_level<1>(nkeys, h, x, y, s, st);
    case 3: return keygen_level<3>(nkeys, h, x, y, s, st);
    case 5: return keygen_level<5>(nkeys, h, x, y, s, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_encrypt(int level, int64_t count, const uint64_t* h, const uint64_t* s, int64_t nkeys,
                           const int32_t* key_idx, const uint8_t* m, const uint32_t* r1, const uint32_t* r2,
                           const uint32_t* e, uint64_t* u, uint64_t* v, cudaStream_t st) {
  switch (level) {
    case 1: return encrypt_level<1, false, false>(count, h, s, nkeys, key_idx, m, r1, r2, e, u, v, 0, 0, 0, st);
    case 3: return encrypt_level<3, false, false>(count, h, s, nkeys, key_idx, m, r1, r2, e, u, v, 0, 0, 0, st);
    case 5: return encrypt_level<5, false, false>(count, h, s, nkeys, key_idx, m, r1, r2, e, u, v, 0, 0, 0, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_encrypt_compare(int level, int64_t count, const uint64_t* h, const uint64_t* s, int64_t nkeys,
                                   const int32_t* key_idx, const uint8_t* m, const uint32_t* r1, const uint32_t* r2,
                                   const uint32_t* e, const uint64_t* u_in, const uint64_t* v_in, uint32_t* ok,
                                   cudaStream_t st) {
  switch (level) {
    case 1: return encrypt_level<1, true, true>(count, h, s, nkeys, key_idx, m, r1, r2, e, 0, 0, u_in, v_in, ok, st);
    case 3: return encrypt_level<3, true, true>(count, h, s, nkeys, key_idx, m, r1, r2, e, 0, 0, u_in, v_in, ok, st);
    case 5: return encrypt_level<5, true, true>(count, h, s, nkeys, key_idx, m, r1, r2, e, 0, 0, u_in, v_in, ok, st);
  }
  return cudaErrorInvalidValue;
}

// Encryption with sampler-drawn supports (the KEM's encapsulation).
cudaError_t launch_encrypt_valid(int level, int64_t count, const uint64_t* h, const uint64_t* s, int64_t nkeys,
                                 const int32_t* key_idx, const uint8_t* m, const uint32_t* r1, const uint32_t* r2,
                                 const uint32_t* e, uint64_t* u, uint64_t* v, cudaStream_t st) {
  switch (level) {
    case 1: return encrypt_level<1, false, true>(count, h, s, nkeys, key_idx, m, r1, r2, e, u, v, 0, 0, 0, st);
    case 3: return encrypt_level<3, false, true>(count, h, s, nkeys, key_idx, m, r1, r2, e, u, v, 0, 0, 0, st);
    case 5: return encrypt_level<5, false, true>(count, h, s, nkeys, key_idx, m, r1, r2, e, u, v, 0, 0, 0, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hqc

// Device building blocks of batched HQC.PKE decryption on sm_103a.
//
// Every routine is warp- or thread-level, has a fixed trip count that
// depends only on the (public) level, and selects with masks instead of
// branching on ciphertext or key data, so the control flow of a
// decryption does not depend on secrets (HQC's constant-time requirement,
// Sec. III-B and III-D of the paper).
#pragma once
#include <cstdint>
#include <type_traits>

#include "hqc_params.cuh"

namespace hqc {

constexpr unsigned FULL_MASK = 0xFFFFFFFFu;

// ---------------------------------------------------------------------------
// GF(2^8) = GF(2)[x]/(x^8+x^4+x^3+x^2+1), alpha = x.
// Log/antilog tables live in shared memory, replicated once per lane so a
// warp's 32 lookups always hit 32 different banks: the access time does not
// depend on the (secret) indices.
//   exp: entries e in [0, 512): alpha^(e mod 255) for e < 511, exp[511] = 0
//   log: entries a in [0, 256): log_alpha(a), log[0] = 511
// With log 0 = 511, a*b = exp[min(log a + log b, 511)] for all a, b.
// ---------------------------------------------------------------------------
constexpr int GF_EXP_BYTES = 512 * 32;
constexpr int GF_LOG_BYTES = 256 * 32 * 2;
constexpr int GF_TABLE_BYTES = GF_EXP_BYTES + GF_LOG_BYTES;
constexpr uint32_t GF_LOG_ZERO = 511;

// c ? a : b as one predicated select (no branch).
__device__ __forceinline__ uint32_t sel(bool c, uint32_t a, uint32_t b) {
  uint32_t d;
  asm("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %3, 0;\n\tselp.b32 %0, %1, %2, p;\n\t}"
      : "=r"(d)
      : "r"(a), "r"(b), "r"((uint32_t)c));
  return d;
}

__device__ __forceinline__ uint32_t gf_xtime(uint32_t a) {
  return ((a << 1) ^ (0x11Du & (0u - (a >> 7)))) & 0xFFu;
}

// The two tables packed as the 32-bit words one lane's column holds:
// exp4[q] = exp[4q .. 4q+3] as bytes, log2[p] = log[2p], log[2p+1] as
// halfwords.  Computed at compile time (GF(2^8) mod x^8+x^4+x^3+x^2+1,
// alpha = x) into global memory; a block copies each word into all 32
// lane columns.
struct GfPacked {
  uint32_t exp4[128];
  uint32_t log2[128];
  __host__ __device__ constexpr GfPacked() : exp4(), log2() {
    uint32_t ex[512] = {};
    uint32_t lg[256] = {};
    uint32_t x = 1;
    for (int e = 0; e < 255; e++) {
      ex[e] = x;
      ex[e + 255] = x;
      lg[x] = (uint32_t)e;
      x = ((x << 1) ^ ((x >> 7) ? 0x11Du : 0u)) & 0xFFu;
    }
    ex[510] = ex[0];
    ex[511] = 0;
    lg[0] = GF_LOG_ZERO;
    for (int q = 0; q < 128; q++)
      exp4[q] = ex[4 * q] | ex[4 * q + 1] << 8 | ex[4 * q + 2] << 16 | ex[4 * q + 3] << 24;
    for (int p = 0; p < 128; p++) log2[p] = lg[2 * p] | lg[2 * p + 1] << 16;
  }
};
static __device__ const GfPacked g_gf_packed = GfPacked();

// Fill both tables; called by every thread of the block, then
// __syncthreads.  Word w of either table belongs to lane w mod 32 and holds
// packed word w / 32, so each 128-byte row is one packed word 32 times.
// Thread q of the first 256 reads packed word q (exp rows, then log rows)
// with its own load -- all rows arrive after one memory round trip -- and
// writes the row as eight 16-byte stores, in an order rotated by the
// thread so the eight threads of a store phase hit eight different banks.
__device__ inline void gf_tables_init(uint8_t* smem, int tid, int nthreads) {
  const uint32_t* packed = reinterpret_cast<const uint32_t*>(&g_gf_packed);
  uint4* rows = reinterpret_cast<uint4*>(smem);  // 128 exp rows, then 128 log rows
  static_assert(GF_EXP_BYTES == 128 * 128 && sizeof(GfPacked) == 256 * 4, "table layout");
  for (int q = tid; q < 256; q += nthreads) {
    const uint32_t w = __ldg(packed + q);
    const uint4 v = make_uint4(w, w, w, w);
#pragma unroll
    for (int j = 0; j < 8; j++) rows[8 * q + ((j + q) & 7)] = v;
  }
}

struct GF {
  const uint8_t* ex;   // this lane's column: exp table + 4 * lane
  const uint16_t* lg;  // this lane's column: log table + 2 * lane (halfwords)
  uint32_t lane;
  __device__ __forceinline__ GF(const uint8_t* smem, uint32_t lane_)
      : ex(smem + 4 * lane_), lg(reinterpret_cast<const uint16_t*>(smem + GF_EXP_BYTES) + 2 * lane_), lane(lane_) {}
  // e in [0, 511].  Entry e sits at byte ((e & ~3) << 5) + (e & 3) of the
  // lane's column, i.e. 32 e - 31 (e & 3): written as multiplies so the
  // address arithmetic can run on the multiply-add pipe.
  __device__ __forceinline__ uint32_t exp(uint32_t e) const { return ex[e * 32u - (e & 3u) * 31u]; }
  // a in [0, 255]: halfword 32 a - 31 (a & 1) of the lane's column
  __device__ __forceinline__ uint32_t log(uint32_t a) const { return lg[a * 32u - (a & 1u) * 31u]; }
  // product of two elements given by their logs (511 = zero)
  __device__ __forceinline__ uint32_t mul_l(uint32_t la, uint32_t lb) const {
    return exp(min(la + lb, GF_LOG_ZERO));
  }
  __device__ __forceinline__ uint32_t mul(uint32_t a, uint32_t b) const { return mul_l(log(a), log(b)); }
  // a / b from logs, with x / 0 := 0 and 0 / x = 0
  __device__ __forceinline__ uint32_t div_l(uint32_t la, uint32_t lb) const {
    const uint32_t e = la + 255u - lb;
    return exp(sel(max(la, lb) >= GF_LOG_ZERO, GF_LOG_ZERO, e));
  }
};

// ---------------------------------------------------------------------------
// S1/S2: stage u in shared memory as the doubled 2n-bit string u || u.
// Bits of u at positions >= n (the padding of the last word and the pad
// word) are cleared, so garbage there never reaches the product.
// PITCH64 = 64-bit words per HBM row (even, 16-byte aligned rows).
// ---------------------------------------------------------------------------
struct WarpSync {
  __device__ __forceinline__ void operator()() const { __syncwarp(); }
};

// NT threads (tid in [0, NT)) build it together; sync() orders their
// shared-memory writes (__syncwarp for one warp, a named barrier for a team).
template <int N, int PITCH64, int U2W, int NT = 32, class Sync = WarpSync>
__device__ __forceinline__ void build_doubled(uint32_t* u2, const uint64_t* __restrict__ urow, int tid,
                                              const Sync& sync = Sync()) {
  constexpr int N32 = (N + 31) / 32, R = N & 31, F = N >> 5;
  const uint4* src = reinterpret_cast<const uint4*>(urow);
  uint4* dst = reinterpret_cast<uint4*>(u2);
#pragma unroll 2
  for (int i = tid; i < PITCH64 / 2; i += NT) {
    uint4 x = __ldcs(src + i);
    uint32_t wv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int c = 0; c < 4; c++) {
      const int idx = 4 * i + c;
      uint32_t keep = idx < F ? 0xFFFFFFFFu : 0u;
      if (R) keep = idx == F ? ((1u << R) - 1u) : keep;
      wv[c] &= keep;
    }
    dst[i] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
  }
  sync();
  // second copy: word a >= N32 holds bits [32a - N, 32a - N + 32) of u
#pragma unroll 2
  for (int a = N32 + tid; a < U2W; a += NT) {
    const int o = 32 * a - N;
    const int kw = o >> 5, sh = o & 31;
    const uint32_t lo = kw < N32 ? u2[kw] : 0u;
    const uint32_t hi = kw + 1 < N32 ? u2[kw + 1] : 0u;
    u2[a] = __funnelshift_r(lo, hi, sh);
  }
  sync();
  // straddle word: the first bits of the second copy start at bit R of word F
  if (R && tid == 0) u2[F] |= u2[0] << R;
  sync();
}

// Support entry p -> two words: with q0 = n - p the rotation by p reads u2
// from bit 32 i + q0, i.e. word i + (q0 >> 5) at shift q0 & 31.  Stored as
// sup[2t] = 4 (q0 >> 5) (a byte offset) and sup[2t+1] = (q0 & 31) | (p < n)
// << 31; an entry p >= n stores offset 0 and no flag, and its contribution
// is masked off.  (Funnel shifts use the shift modulo 32, so the flag bit
// can stay in place.)
template <int N, int W, int NT = 32>
__device__ __forceinline__ void load_supports(uint32_t* sup, const uint32_t* __restrict__ yrow, int tid) {
  for (int t = tid; t < W; t += NT) {
    const uint32_t p = __ldg(yrow + t);
    const bool ok = p < (uint32_t)N;
    const uint32_t q0 = (uint32_t)N - p;
    *reinterpret_cast<uint2*>(sup + 2 * t) = make_uint2(sel(ok, (q0 >> 5) << 2, 0u), sel(ok, (q0 & 31u) | 0x80000000u, 0u));
  }
}

// ---------------------------------------------------------------------------
// S3 (Eq. 1): t = XOR over p in Supp(y) of x^p u, truncated to the first
// (strips)*32*WPT bits.  Strip l (a lane, or a lane of a team) owns output
// words [l*WPT, l*WPT + WPT).
// Word i of x^p u is the 32-bit window of u2 at bit 32 i + n - p: two
// neighbouring u2 words joined by one funnel shift.  The lane's strip of
// WPT + 1 u2 words is read once per support entry; WPT odd keeps the
// warp's reads on 32 distinct banks for every rotation.  Every lane of a
// load works on the same support entry, so its 32 addresses are one fixed
// pattern shifted by that entry's offset: one wavefront whatever the
// secret positions.  (Lanes working on different entries at once, e.g. to
// share out a few leftover words, would collide in banks depending on the
// positions, so the strips cover the product with odd WPT and no tail.)
// PREFETCH (validated supports only): the next pair of entries is read one
// pass ahead, so a pass's window loads need not wait for its entries.
// Worth it where a scheduler holds one or two warps (the latency teams);
// elsewhere other warps hide that wait and the registers are scarcer.
// ---------------------------------------------------------------------------
template <int WPT, int W, bool MASKED, bool PREFETCH = false>
__device__ __forceinline__ void rot_xor_product(const uint32_t* u2, const uint32_t* sup, int w0,
                                                uint32_t (&acc)[WPT]) {
#pragma unroll
  for (int k = 0; k < WPT; k++) acc[k] = 0;
  const char* base = reinterpret_cast<const char*>(u2 + w0);
  if (MASKED) {
#pragma unroll 1
    for (int t = 0; t < W; t++) {
      const uint2 e = *reinterpret_cast<const uint2*>(sup + 2 * t);
      const uint32_t msk = (uint32_t)((int32_t)e.y >> 31);
      const uint32_t* src = reinterpret_cast<const uint32_t*>(base + e.x);
      uint32_t lo = src[0];
#pragma unroll
      for (int k = 0; k < WPT; k++) {
        const uint32_t hi = src[k + 1];
        acc[k] ^= __funnelshift_r(lo, hi, e.y) & msk;
        lo = hi;
      }
    }
  } else {
    // validated supports: two entries per pass so each accumulator update
    // is a single three-input XOR
    uint4 en = *reinterpret_cast<const uint4*>(sup);
#pragma unroll 1
    for (int t = 0; t + 1 < W; t += 2) {
      uint4 e;
      if constexpr (PREFETCH) {
        // the last pass re-reads the last pair (an even index keeps the
        // 16-byte load aligned and inside the W entries)
        constexpr int LASTPAIR = (W - 2) & ~1;
        e = en;
        en = *reinterpret_cast<const uint4*>(sup + 2 * (t + 2 < LASTPAIR ? t + 2 : LASTPAIR));
      } else {
        e = *reinterpret_cast<const uint4*>(sup + 2 * t);
      }
      const uint32_t* a0 = reinterpret_cast<const uint32_t*>(base + e.x);
      const uint32_t* a1 = reinterpret_cast<const uint32_t*>(base + e.z);
      uint32_t lo0 = a0[0], lo1 = a1[0];
#pragma unroll
      for (int k = 0; k < WPT; k++) {
        const uint32_t hi0 = a0[k + 1], hi1 = a1[k + 1];
        acc[k] ^= __funnelshift_r(lo0, hi0, e.y) ^ __funnelshift_r(lo1, hi1, e.w);
        lo0 = hi0;
        lo1 = hi1;
      }
    }
    if (W & 1) {
      const uint2 e = *reinterpret_cast<const uint2*>(sup + 2 * (W - 1));
      const uint32_t* src = reinterpret_cast<const uint32_t*>(base + e.x);
      uint32_t lo = src[0];
#pragma unroll
      for (int k = 0; k < WPT; k++) {
        const uint32_t hi = src[k + 1];
        acc[k] ^= __funnelshift_r(lo, hi, e.y);
        lo = hi;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// S5-S7: decode one duplicated RM(1,7) block (mult copies of 128 bits at
// blk, 16-byte aligned) to one byte, with a PAIR of lanes per block.
//   s_i = mult - 2 * #(copies with bit i set)           (S5)
//   F(a) = sum_i s_i (-1)^{popcount(a & i)}, 7 butterfly stages (S6)
//   byte = a* + 128 [F(a*) < 0], a* = argmax |F|, ties -> smallest a (S7)
// Lane hb (= lane & 1) of the pair holds the 64 elements with index bit 6
// equal to hb, as 32 registers of two 16-bit halves.  Register r = 16 tt +
// q holds indices q | tt << 5 | hb << 6 (low half) and the same | 16 (high
// half).  Stages on index bits 0-3 and 5 are packed adds inside a lane.
// For mult 3 a register there is the integer 65536 hi + lo of its two
// signed halves, which sums and differences keep exact (a negative low half
// borrows from the high half, and is lent back when the bias is added), so
// a butterfly is a plain add and a plain subtract; bit 6, one shuffle with
// the partner lane, adds the bias 640 to both halves.  With SIGNED false
// every stage keeps both halves biased by 640 (a butterfly adds or
// subtracts the bias too).  Measured: the signed form is 3.6 % faster in
// the HQC-1 fused kernel (it removes a spill at 64 registers), the biased
// one 0.6-0.8 % faster for mult 5, and in the stand-alone RM stage kernel
// (48 against 54 registers, so more warps per SM) 8 % faster for mult 3
// too.  Either way, after bit 6 each half is F + 640 as an unsigned
// 16-bit value (|F| <= 640, and F is even: a sum of 128 odd s_i); bit 4
// (the halves) is the last stage.
// The argmax runs on 16-bit keys (F + 640) / 2 * 64 + (63 - r6) -- score,
// then smaller index -- with packed unsigned max, once for +F (b = 0) and
// once for -F (b = 1); the half bit and b stay implicit in where the key
// sits.  Both lanes of the pair return the byte.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t vmax_u16x2(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}

// max of three pairs of unsigned 16-bit halves
__device__ __forceinline__ uint32_t vmax3_u16x2(uint32_t a, uint32_t b, uint32_t c) {
  return __vimax3_u16x2(a, b, c);
}

template <int MULT, bool SIGNED = MULT == 3>
__device__ __forceinline__ uint32_t rm_decode_pair(const uint32_t* blk, uint32_t hb) {
  constexpr uint32_t BIAS = 640u;
  constexpr uint32_t BP = BIAS * 0x10001u;
  constexpr uint32_t K = (SIGNED ? MULT : BIAS + MULT) * 0x10001u;  // K - 2 c = s_i (+ bias) in both halves
  constexpr uint32_t SB = SIGNED ? 0u : BP;
  constexpr uint32_t KN = 2u * BP * 32u;  // (1280 per half) * 32
  uint32_t p0[2], p1[2], p2[2];
  {
    uint2 cp[MULT];
#pragma unroll
    for (int c = 0; c < MULT; c++) cp[c] = *reinterpret_cast<const uint2*>(blk + 4 * c + 2 * hb);
#pragma unroll
    for (int tt = 0; tt < 2; tt++) {
      uint32_t b[MULT];
#pragma unroll
      for (int c = 0; c < MULT; c++) b[c] = tt == 0 ? cp[c].x : cp[c].y;
      // bit-sliced population count of the copies
      const uint32_t s1 = b[0] ^ b[1] ^ b[2];
      const uint32_t k1 = (b[0] & b[1]) | (b[2] & (b[0] ^ b[1]));
      if (MULT == 3) {
        p0[tt] = s1;
        p1[tt] = k1;
        p2[tt] = 0;
      } else {
        const uint32_t d = b[MULT > 3 ? 3 : 0], e = b[MULT > 4 ? 4 : 0];
        const uint32_t k2 = (s1 & d) | (e & (s1 ^ d));
        p0[tt] = s1 ^ d ^ e;
        p1[tt] = k1 ^ k2;
        p2[tt] = k1 & k2;
      }
    }
  }
  // Packed counts of positions q and q + 16: the count planes are first
  // bit-interleaved so one shift and one mask extract a whole count
  // (positions q, q+1 for mult 3; q..q+2 in residue classes mod 4 for 5).
  uint32_t R[32];
#pragma unroll
  for (int tt = 0; tt < 2; tt++) {
    if (MULT == 3) {
      const uint32_t z0 = (p0[tt] & 0x55555555u) | ((p1[tt] & 0x55555555u) << 1);  // even q
      const uint32_t z1 = ((p0[tt] & 0xAAAAAAAAu) >> 1) | (p1[tt] & 0xAAAAAAAAu);  // odd q
#pragma unroll
      for (int q = 0; q < 16; q++) {
        const uint32_t cnt = ((q & 1 ? z1 : z0) >> (q & ~1)) & 0x00030003u;
        R[16 * tt + q] = K - 2u * cnt;
      }
    } else {
      uint32_t z[4];
#pragma unroll
      for (int rr = 0; rr < 4; rr++) {
        const uint32_t mk = 0x11111111u << rr;
        z[rr] = ((p0[tt] & mk) >> rr) | (((p1[tt] & mk) >> rr) << 1) | (((p2[tt] & mk) >> rr) << 2);
      }
#pragma unroll
      for (int q = 0; q < 16; q++) {
        const uint32_t cnt = (z[q & 3] >> (q & ~3)) & 0x00070007u;
        R[16 * tt + q] = K - 2u * cnt;
      }
    }
  }
#pragma unroll
  for (int b = 0; b < 5; b++) {
#pragma unroll
    for (int r = 0; r < 32; r++) {
      if (!(r & (1 << b))) {
        const uint32_t X = R[r], Y = R[r | (1 << b)];
        R[r] = X + Y - SB;
        R[r | (1 << b)] = X - Y + SB;
      }
    }
  }
  // index bit 6: lane 0 keeps x + y, lane 1 keeps y - x (x = own value,
  // y = partner's), both biased: own * (+-1) + (y + cst), one multiply-add
  // (cst adds the bias for unbiased inputs, corrects it for biased ones)
  const uint32_t sgn = hb ? 0xFFFFFFFFu : 1u;
  const uint32_t cst = SIGNED ? BP : hb ? BP : (0u - BP);
#pragma unroll
  for (int r = 0; r < 32; r++) {
    const uint32_t Y = __shfl_xor_sync(FULL_MASK, R[r], 1);
    R[r] = R[r] * sgn + (Y + cst);
  }
  uint32_t mp[4] = {0, 0, 0, 0}, mn[4] = {0, 0, 0, 0};
  const uint32_t cbase = (63u - 32u * hb) * 0x10001u;
#pragma unroll
  for (int r = 0; r < 32; r += 2) {
    // index bit 4: low half -> lo + hi - bias, high half -> lo - hi + bias,
    // as lo * 0x10001 + hi * (1 - 2^16) + bias * (2^16 - 1) (mod 2^32)
    uint32_t kp[2], kn[2];
#pragma unroll
    for (int d = 0; d < 2; d++) {
      const uint32_t X = R[r + d];
      const uint32_t P = (X & 0xFFFFu) * 0x10001u + (X >> 16) * 0xFFFF0001u + (BIAS * 0xFFFFu);
      const uint32_t C = cbase - (uint32_t)(r + d) * 0x10001u;
      kp[d] = P * 32u + C;
      kn[d] = (KN + C) - P * 32u;
    }
    const int a = (r >> 1) & 3;
    mp[a] = vmax3_u16x2(mp[a], kp[0], kp[1]);
    mn[a] = vmax3_u16x2(mn[a], kn[0], kn[1]);
  }
  uint32_t MP = vmax3_u16x2(mp[0], mp[1], vmax_u16x2(mp[2], mp[3]));
  uint32_t MN = vmax3_u16x2(mn[0], mn[1], vmax_u16x2(mn[2], mn[3]));
  MP = vmax_u16x2(MP, __shfl_xor_sync(FULL_MASK, MP, 1));
  MN = vmax_u16x2(MN, __shfl_xor_sync(FULL_MASK, MN, 1));
  uint32_t best = 0;
#pragma unroll
  for (int c = 0; c < 4; c++) {
    const uint32_t M = c < 2 ? MP : MN;
    const uint32_t h = c & 1, b = c >> 1;
    const uint32_t key = h ? (M >> 16) : (M & 0xFFFFu);
    const uint32_t s = key >> 6, r6 = 63u - (key & 63u);
    const uint32_t a = (r6 & 15u) | (h << 4) | ((r6 >> 4) << 5);
    best = max(best, (s << 8) | ((127u - a) << 1) | (1u - b));
  }
  const uint32_t a = 127u - ((best >> 1) & 127u);
  return a | ((1u - (best & 1u)) << 7);
}

// All n1 blocks of one ciphertext by NP lane pairs (16 for one warp, 32
// for a two-warp team), tid in [0, 2 NP).
// w: the n1*n2-bit word vector (shared or global, 16-byte aligned).
template <class LV, int NP = 16>
__device__ __forceinline__ void rm_decode_warp(const uint32_t* w, uint8_t* r, int tid) {
  const uint32_t hb = tid & 1;
#pragma unroll 1
  for (int j0 = 0; j0 < LV::n1; j0 += NP) {
    const int j = j0 + (tid >> 1);
    const int jj = j < LV::n1 ? j : LV::n1 - 1;
    const uint32_t byte = rm_decode_pair<LV::mult>(w + jj * (LV::n2 / 32), hb);
    if (j < LV::n1 && hb == 0) r[j] = (uint8_t)byte;
  }
}

// ---------------------------------------------------------------------------
// S8-S9: Reed-Solomon decoding, SEG lanes per received word (a warp decodes
// 32 / SEG words side by side; all shuffles stay inside a segment).
//   syndromes S_i = sum_j r_j alpha^{i j}, i = 1..2 delta    (Sec. III-D)
//   Berlekamp-Massey, exactly 2 delta iterations, Lambda and x^m B kept
//   with 2 delta + 1 coefficients spread over the segment's lanes
//   Chien: position j in error iff Lambda(alpha^{-j}) = 0
//   Forney: e_j = Omega(alpha^{-j}) / Lambda'(alpha^{-j}), Omega = S Lambda
//   mod x^{2 delta}
// r: the n1 received bytes of this segment's word; rs: RS_SCRATCH words of
// shared scratch for it.  With ALL_POS false only the k message positions
// are evaluated (m is all the decryption returns); with ALL_POS true every
// position is evaluated and the intermediates are written to dbg.  A
// segment with active == false computes but stores nothing.
// ---------------------------------------------------------------------------
struct RSDebugRow {
  uint8_t* S;        // 2 delta
  uint8_t* lam;      // 2 delta + 1
  int32_t* L;        // 1
  uint8_t* errmask;  // n1
  uint8_t* errval;   // n1
  uint8_t* cw;       // n1
  int32_t* flag;     // 1
};

// words: log r (96 halfwords), log S behind 64 halfwords of log-zero padding
// (128), log Lambda and log Omega (64 halfwords each)
constexpr int RS_SCRATCH = 176;

// ---------------------------------------------------------------------------
// Syndromes by Horner's rule on per-lane multiply tables (the table-driven
// syndromes of Sec. III-D, in a GPU layout).  For one received word
//   S_i = sum_j r_j alpha^{i j}
//       = (...((r_{n1-1}) alpha^i + r_{n1-2}) alpha^i + ...) alpha^i + r_0,
// so lane L, which owns S_{L+1}, only ever multiplies by alpha^{L+1}: a
// 256-entry table of its own, in its own bank.  An element x travels as
// its byte offset in the table block,
//   o_L(x) = spread(x) | 4 L,  spread(x) = ((x >> 1) << 7) | ((x & 1) << 1)
// (entry x of lane L is halfword x & 1 of word 32 (x >> 1) + L).  spread
// is linear over GF(2) and leaves bits 2..6 free for 4 L, so
//   o_L(x alpha^{L+1} + r) = T_L[o_L(x)] ^ spread(r),
// with T_L[o_L(x)] = o_L(x alpha^{L+1}) stored in the table: a Horner step
// is one shared load and one XOR, with no exponent arithmetic.  Every
// offset stays inside the 16 KB block (spread(255) | 124 + 2 < 16384)
// whatever the bytes, and a warp's 32 loads hit 32 banks.
// ---------------------------------------------------------------------------
constexpr int SYN_TABLE_BYTES = 256 * 32 * 2;

__host__ __device__ constexpr uint32_t syn_spread(uint32_t x) { return ((x >> 1) << 7) | ((x & 1u) << 1); }
__host__ __device__ constexpr uint32_t syn_unspread(uint32_t o) { return ((o >> 6) & 0xFEu) | ((o >> 1) & 1u); }
static_assert(syn_unspread(syn_spread(0xA5u) | 4u * 31u) == 0xA5u && syn_spread(255u) + 4u * 31u + 2u <= 16384u,
              "syndrome table offsets");

// Fill a block's syndrome table: column L multiplies by alpha^{L+1}.  Reads
// the packed GF tables from global memory, so it needs no barrier after the
// shared GF tables and can share theirs.
__device__ inline void syn_table_init(uint8_t* tab, int tid, int nthreads) {
  const uint32_t* packed = reinterpret_cast<const uint32_t*>(&g_gf_packed);
  for (int e = tid; e < 32 * 256; e += nthreads) {
    const uint32_t L = (uint32_t)e & 31u, x = (uint32_t)e >> 5;
    const uint32_t lg = (__ldg(packed + 128 + (x >> 1)) >> (16 * (x & 1u))) & 0xFFFFu;
    const uint32_t ex = lg + L + 1u;  // <= 254 + 32: inside the doubled exp table
    const uint32_t y = x == 0 ? 0u : (__ldg(packed + (ex >> 2)) >> (8 * (ex & 3u))) & 0xFFu;
    *reinterpret_cast<uint16_t*>(tab + (syn_spread(x) | 4u * L)) = (uint16_t)(syn_spread(y) | 4u * L);
  }
}

// S_1..S_{2 delta} of a warp's G received words (lane L computes S_{L+1}
// of each: G Horner chains side by side), stored as logs where
// rs_decode_seg<..., HAVE_S = true> expects them.  rs: the words' scratch
// areas (RS_SCRATCH words apart); r: their RM bytes (RB bytes apart).  The
// spread bytes go where rs_decode_seg would keep log r.  Lanes past
// 2 delta run the chains and store nothing.
template <class LV, int G>
__device__ __forceinline__ void rs_syndromes_horner(const GF& gf, const uint8_t* syn, uint32_t* rs,
                                                    const uint8_t* r, int RB, int lane) {
  constexpr int n1 = LV::n1, NR = LV::NR;
  static_assert(NR <= 32 && n1 <= 96, "one syndrome per lane; spread bytes fit the log r area");
#pragma unroll
  for (int g = 0; g < G; g++)
    for (int j = lane; j < n1; j += 32)
      reinterpret_cast<uint16_t*>(rs + g * RS_SCRATCH)[j] = (uint16_t)syn_spread(r[g * RB + j]);
  __syncwarp();
  uint32_t o[G];
#pragma unroll
  for (int g = 0; g < G; g++) o[g] = (4u * (uint32_t)lane) ^ reinterpret_cast<const uint16_t*>(rs + g * RS_SCRATCH)[n1 - 1];
#pragma unroll
  for (int j = n1 - 2; j >= 0; j--) {
#pragma unroll
    for (int g = 0; g < G; g++)
      o[g] = (uint32_t)*reinterpret_cast<const uint16_t*>(syn + o[g]) ^
             reinterpret_cast<const uint16_t*>(rs + g * RS_SCRATCH)[j];
  }
  if (lane < NR) {
#pragma unroll
    for (int g = 0; g < G; g++)
      (reinterpret_cast<uint16_t*>(rs + g * RS_SCRATCH + 48) + 64)[lane] = (uint16_t)gf.log(syn_unspread(o[g]));
  }
}

// Berlekamp-Massey (S8) on SEG lanes: exactly 2 delta iterations over the
// syndromes logS (log form, with log-zero padding below index 0); writes the
// logs of Lambda_0..Lambda_{2 delta} to logLam and returns the LFSR length L.
template <class LV, int SEG, bool ALL_POS>
__device__ __forceinline__ uint32_t rs_bm(const GF& gf, const uint16_t* logS, uint16_t* logLam, int lane, bool active,
                                          const RSDebugRow* dbg) {
  constexpr int NR = LV::NR, CAP = LV::CAP;
  const int sl = lane % SEG;
  // Berlekamp-Massey; lane owns coefficient c = sl + SEG x.  x^m B is only
  // ever multiplied, so it is carried in log form (lbp, 511 = zero): it
  // shifts with the same shuffles and, when replaced by Lambda, takes the
  // logs of Lambda already computed for the discrepancy.
  // At the start of iteration r, deg Lambda <= r and deg x^m B <= r + 1, so
  // coefficient block x (c in [SEG x, SEG x + SEG)) is still all zero in
  // both while r + 2 <= SEG x: iteration r works on the first
  // NA(r) = min(NC, floor((r + 2) / SEG) + 1) blocks only.  r is public,
  // so the trip counts stay independent of the data.
  constexpr int NC = cdiv(CAP, SEG);
  uint32_t lam[NC], lbp[NC];
#pragma unroll
  for (int x = 0; x < NC; x++) {
    const int c = sl + SEG * x;
    lam[x] = c == 0;
    lbp[x] = c == 1 ? 0u : GF_LOG_ZERO;  // x^m B with m = 1, B = 1
  }
  uint32_t lb = 0, L = 0;  // log b (b = 1), LFSR length
  auto bm_iter = [&](auto na, int rr) {
    constexpr int NA = decltype(na)::value;
    uint32_t llam[NA];
    uint32_t part = 0;
#pragma unroll
    for (int x = 0; x < NA; x++) {
      const int c = sl + SEG * x;  // rr - c >= -64: padding covers c > rr
      llam[x] = gf.log(lam[x]);
      part ^= gf.mul_l(llam[x], logS[rr - c]);
    }
    if constexpr (SEG == 32) {
      part = __reduce_xor_sync(FULL_MASK, part);  // one warp-wide reduction
    } else if constexpr (SEG == 16) {
      // two warp-wide reductions, each over one half's partial sums
      const uint32_t lo = __reduce_xor_sync(FULL_MASK, lane < 16 ? part : 0u);
      const uint32_t hi = __reduce_xor_sync(FULL_MASK, lane < 16 ? 0u : part);
      part = lane < 16 ? lo : hi;
    } else {
#pragma unroll
      for (int o = SEG / 2; o > 0; o >>= 1) part ^= __shfl_xor_sync(FULL_MASK, part, o, SEG);
    }
    const uint32_t d = part;
    const uint32_t ld = gf.log(d);
    const uint32_t lcoef = sel(d == 0, GF_LOG_ZERO, sel(ld >= lb, ld - lb, ld + 255u - lb));
    const bool cond = (d != 0) & (2 * L <= (uint32_t)rr);
    uint32_t src[NA];
#pragma unroll
    for (int x = 0; x < NA; x++) {
      lam[x] ^= gf.mul_l(lcoef, lbp[x]);
      src[x] = sel(cond, llam[x], lbp[x]);
    }
#pragma unroll
    for (int x = 0; x < NA; x++) {
      const uint32_t up = __shfl_up_sync(FULL_MASK, src[x], 1, SEG);
      const uint32_t carry = x > 0 ? __shfl_sync(FULL_MASK, src[x > 0 ? x - 1 : 0], SEG - 1, SEG) : GF_LOG_ZERO;
      const uint32_t nb = sl == 0 ? carry : up;
      lbp[x] = (sl + SEG * x) < CAP ? nb : GF_LOG_ZERO;
    }
    lb = sel(cond, ld, lb);
    L = sel(cond, (uint32_t)rr + 1u - L, L);
  };
  // phase p runs iterations [max(0, SEG p - 2), SEG (p + 1) - 2) on p + 1
  // blocks (the last phase runs to NR)
  auto bm_phase = [&](auto na) {
    constexpr int NA = decltype(na)::value;
    constexpr int R0 = NA == 1 ? 0 : cmin(NR, SEG * (NA - 1) - 2);
    constexpr int R1 = NA == NC ? NR : cmin(NR, SEG * NA - 2);
#pragma unroll 1
    for (int rr = R0; rr < R1; rr++) bm_iter(na, rr);
  };
  static_assert(NC >= 1 && NC <= 8, "BM phases");
  bm_phase(std::integral_constant<int, 1>{});
  if constexpr (NC >= 2) bm_phase(std::integral_constant<int, 2>{});
  if constexpr (NC >= 3) bm_phase(std::integral_constant<int, 3>{});
  if constexpr (NC >= 4) bm_phase(std::integral_constant<int, 4>{});
  if constexpr (NC >= 5) bm_phase(std::integral_constant<int, 5>{});
  if constexpr (NC >= 6) bm_phase(std::integral_constant<int, 6>{});
  if constexpr (NC >= 7) bm_phase(std::integral_constant<int, 7>{});
  if constexpr (NC >= 8) bm_phase(std::integral_constant<int, 8>{});
#pragma unroll
  for (int x = 0; x < NC; x++) {
    const int c = sl + SEG * x;
    if (c < CAP) {
      logLam[c] = (uint16_t)gf.log(lam[x]);
      if (ALL_POS && active) dbg->lam[c] = (uint8_t)lam[x];
    }
  }
  if (ALL_POS && active && sl == 0) *dbg->L = (int32_t)L;
  __syncwarp();
  return L;
}

// HAVE_S: the syndromes' logs are already in rs (rs_syndromes_horner).
template <class LV, int SEG, bool ALL_POS, bool HAVE_S = false>
__device__ __forceinline__ void rs_decode_seg(const GF& gf, uint32_t* rs, const uint8_t* r, int lane, bool active,
                                              uint8_t* __restrict__ m_out, const RSDebugRow* dbg) {
  constexpr int n1 = LV::n1, k = LV::k, NR = LV::NR, CAP = LV::CAP, delta = LV::delta;
  static_assert(n1 <= 96 && CAP <= 64, "RS scratch sizes");
  static_assert(!(HAVE_S && ALL_POS), "the debug path computes its own syndromes");
  const int sl = lane % SEG;
  uint16_t* logr = reinterpret_cast<uint16_t*>(rs);
  // logS[i] for i in [-64, 64): negative indices read log 0, so terms of
  // Lambda_c S_{r+1-c} with c > r vanish without a select
  uint16_t* logS = reinterpret_cast<uint16_t*>(rs + 48) + 64;
  uint16_t* logLam = reinterpret_cast<uint16_t*>(rs + 112);
  uint16_t* logOm = reinterpret_cast<uint16_t*>(rs + 144);

  if constexpr (!HAVE_S)
    for (int j = sl; j < n1; j += SEG) logr[j] = (uint16_t)gf.log(r[j]);
  for (int j = sl; j < 64; j += SEG) logS[j - 64] = (uint16_t)GF_LOG_ZERO;
  __syncwarp();

  // syndromes: lane owns i = sl + 1 + SEG s; each log r_j is loaded once
  // for all of the lane's syndromes
  constexpr int NS = cdiv(NR, SEG);
  if constexpr (!HAVE_S) {
    uint32_t acc[NS], e[NS];
#pragma unroll
    for (int s = 0; s < NS; s++) acc[s] = e[s] = 0;
#pragma unroll 2
    for (int j = 0; j < n1; j++) {
      const uint32_t lr = logr[j];
#pragma unroll
      for (int s = 0; s < NS; s++) {
        acc[s] ^= gf.exp(min(lr + e[s], GF_LOG_ZERO));
        e[s] += (uint32_t)(sl + 1 + SEG * s);
        e[s] = e[s] >= 255u ? e[s] - 255u : e[s];
      }
    }
#pragma unroll
    for (int s = 0; s < NS; s++) {
      const uint32_t i = (uint32_t)(sl + 1 + SEG * s);
      if (i <= (uint32_t)NR) {
        logS[i - 1] = (uint16_t)gf.log(acc[s]);
        if (ALL_POS && active) dbg->S[i - 1] = (uint8_t)acc[s];
      }
    }
  }
  __syncwarp();

  const uint32_t L = rs_bm<LV, SEG, ALL_POS>(gf, logS, logLam, lane, active, dbg);

  // Omega_k = sum_{c <= k} Lambda_c S_{k+1-c}, k < 2 delta.  The lanes of
  // block x hold k < SEG (x + 1), so terms c >= SEG (x + 1) vanish for all
  // of them: block x sums over c < min(2 delta, SEG (x + 1)).
#pragma unroll
  for (int x = 0; x < NS; x++) {
    const int kk = sl + SEG * x;
    uint32_t om = 0;
    const int cend = cmin(NR, SEG * (x + 1));
#pragma unroll 4
    for (int c = 0; c < cend; c++) {
      const int idx = kk < NR ? kk - c : -1;  // c > kk reads the log-zero padding
      om ^= gf.mul_l(logLam[c], logS[idx]);
    }
    if (kk < NR) logOm[kk] = (uint16_t)gf.log(om);
  }
  __syncwarp();

  // Chien + Forney at position j: powers of X = alpha^{-j}.  In
  // characteristic 2 the odd part of Lambda is X Lambda'(X), so one sum of
  // the terms Lambda_c X^c gives both Lambda(X) (all terms) and Lambda'(X)
  // (odd terms divided by X), and e_j = Omega(X) X / Lambda_odd(X).
  constexpr int NPOS = ALL_POS ? cdiv(n1, SEG) : cdiv(k, SEG);
  uint32_t roots = 0;
#pragma unroll
  for (int y = 0; y < NPOS; y++) {
    const int pos = sl + SEG * y;
    const int j = ALL_POS ? pos : (n1 - k) + pos;
    const bool valid = ALL_POS ? pos < n1 : pos < k;
    const uint32_t jj = valid ? (uint32_t)j : 0u;
    const uint32_t step = jj == 0 ? 0u : 255u - jj;  // log X
    uint32_t ec = 0, lev = 0, lod = 0, omv = 0;
#pragma unroll
    for (int c = 0; c < CAP; c++) {
      const uint32_t t = gf.exp(min((uint32_t)logLam[c] + ec, GF_LOG_ZERO));
      if (c & 1) lod ^= t; else lev ^= t;
      if (c < NR) omv ^= gf.exp(min((uint32_t)logOm[c] + ec, GF_LOG_ZERO));
      ec += step;
      ec = ec >= 255u ? ec - 255u : ec;
    }
    const bool root = (lev ^ lod) == 0;
    // log(Omega X) = log Omega + log X mod 255 (Omega = 0 keeps log zero)
    const uint32_t lom = gf.log(omv);
    uint32_t lomx = lom + step;
    lomx = lomx >= 255u ? lomx - 255u : lomx;
    lomx = sel(lom >= GF_LOG_ZERO, GF_LOG_ZERO, lomx);
    const uint32_t ev = sel(root, gf.div_l(lomx, gf.log(lod)), 0u);
    const uint32_t cwj = (uint32_t)r[jj] ^ ev;
    if (ALL_POS) {
      const uint32_t segmask = SEG == 32 ? FULL_MASK : (((1u << SEG) - 1u) << (lane - sl));
      roots += __popc(__ballot_sync(FULL_MASK, root && valid) & segmask);
      if (valid && active) {
        dbg->errmask[j] = (uint8_t)root;
        dbg->errval[j] = (uint8_t)ev;
        dbg->cw[j] = (uint8_t)cwj;
        if (j >= n1 - k) m_out[j - (n1 - k)] = (uint8_t)cwj;
      }
    } else if (valid && active) {
      m_out[pos] = (uint8_t)cwj;
    }
  }
  if (ALL_POS && active && sl == 0) *dbg->flag = (int32_t)((L > (uint32_t)delta) || (roots != L));
}

// ---------------------------------------------------------------------------
// S1-S7 of one ciphertext by one warp: product, XOR with v, RM decode; the
// n1 RM bytes go to r_out.  ws: U2W + WP words owned by this warp.
// ---------------------------------------------------------------------------
template <class LV, bool MASKED>
__device__ __forceinline__ void product_rm_one(uint32_t* ws, int lane, const uint64_t* __restrict__ urow,
                                               const uint64_t* __restrict__ vrow, const uint32_t* __restrict__ yrow,
                                               uint8_t* r_out) {
  using PS = ProductStrips<LV::level>;
  constexpr int WPT = PS::MAXLEN, W_v32 = LV::W_v32;
  uint32_t* u2 = ws;
  uint32_t* sup = ws + LV::U2W;
  load_supports<LV::n, LV::w>(sup, yrow, lane);
  build_doubled<LV::n, LV::W_u_pitch, LV::U2W>(u2, urow, lane);
  const int w0 = PS::start(lane), wn = PS::len(lane);
  uint32_t acc[WPT];
  rot_xor_product<WPT, LV::w, MASKED>(u2, sup, w0, acc);
  // S4: w = v + t, truncated (only the first n1*n2 bits were computed)
  const uint32_t* v32 = reinterpret_cast<const uint32_t*>(vrow);
#pragma unroll
  for (int k = 0; k < WPT; k++) {
    const int i = w0 + k;
    if (k < wn && i < W_v32) acc[k] ^= __ldcs(v32 + i);
  }
  __syncwarp();
#pragma unroll
  for (int k = 0; k < WPT; k++) {
    const int i = w0 + k;
    if (k < wn && i < W_v32) u2[i] = acc[k];
  }
  __syncwarp();
  rm_decode_warp<LV>(u2, r_out, lane);
  __syncwarp();
}

// Per-warp shared memory of the fused kernels: u2 and the support list,
// then the RM bytes of up to G ciphertexts kept for the grouped RS stage.
// (a multiple of 4 words, so every warp's u2 stays 16-byte aligned for the
// vector stores that stage u)
template <class LV, int G>
__host__ __device__ constexpr int fused_warp_words() {
  return round_up(LV::U2W + LV::WP + G * cdiv(LV::n1, 4), 4);
}

// Whole decryption (S1-S9) of G ciphertexts by one warp: product and RM
// for each in turn, then Reed-Solomon for all G side by side on 32 / G
// lanes each.  rows(g, u, v, y, m) fills ciphertext g's rows and returns
// false for a slot past the end of the batch (skipped, nothing stored).
// HORNER: the syndromes come from the block's syndrome table syn (Horner
// chains on all 32 lanes) instead of SEG lanes' exponent sums.
template <class LV, int G, bool MASKED, bool HORNER = false, class Rows>
__device__ __forceinline__ void decrypt_group(const GF& gf, uint32_t* ws, int lane, const Rows& rows,
                                              const uint8_t* syn = nullptr) {
  constexpr int RB = cdiv(LV::n1, 4) * 4;  // bytes per stored RM word
  static_assert(G * RS_SCRATCH <= LV::U2W, "RS scratch of G words fits in u2");
  static_assert(fused_warp_words<LV, G>() % 4 == 0 && LV::U2W % 4 == 0 && LV::WP % 4 == 0, "16-byte alignment");
  uint8_t* rbuf = reinterpret_cast<uint8_t*>(ws + LV::U2W + LV::WP);
  const uint64_t* u;
  const uint64_t* v;
  const uint32_t* y;
  uint8_t* m;
#pragma unroll 1
  for (int g = 0; g < G; g++)
    if (rows(g, u, v, y, m)) product_rm_one<LV, MASKED>(ws, lane, u, v, y, rbuf + g * RB);
  constexpr int SEG = 32 / G;
  const int seg = lane / SEG;
  const bool act = rows(seg, u, v, y, m);
  if constexpr (HORNER) rs_syndromes_horner<LV, G>(gf, syn, ws, rbuf, RB, lane);
  rs_decode_seg<LV, SEG, false, HORNER>(gf, ws + seg * RS_SCRATCH, rbuf + seg * RB, lane, act, m, nullptr);
  __syncwarp();
}

// One ciphertext (G = 1), as used by the mixed-level kernel.
template <class LV, bool MASKED>
__device__ __forceinline__ void decrypt_one(const GF& gf, uint32_t* ws, int lane, const uint64_t* __restrict__ urow,
                                            const uint64_t* __restrict__ vrow, const uint32_t* __restrict__ yrow,
                                            uint8_t* __restrict__ mrow) {
  auto rows = [&](int, const uint64_t*& u, const uint64_t*& v, const uint32_t*& y, uint8_t*& m) {
    u = urow;
    v = vrow;
    y = yrow;
    m = mrow;
    return true;
  };
  decrypt_group<LV, 1, MASKED>(gf, ws, lane, rows);
}

// ---------------------------------------------------------------------------
// Teams of T warps.  The warps of a team share one doubled operand: each
// lane computes a strip of WPT2 of the product's output words over the
// team's 32 T lanes, the RM blocks spread over its 16 T lane pairs, and
// warp i < NI decodes the Reed-Solomon stage of the team's i-th ciphertext
// of the turn.  With T = 2, NI = 2 (throughput, HQC-5) a warp needs half
// the shared memory, so twice the warps fit on an SM; with NI = 1 (latency)
// one ciphertext's serial chain is split over the team.
// Members synchronise with a named barrier of 32 T threads.
// ---------------------------------------------------------------------------
struct TeamSync {
  uint32_t id;
  uint32_t threads = 64;
  __device__ __forceinline__ void operator()() const {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
  }
};

// Berlekamp-Massey on one warp (32 lanes, lane owns coefficient c = lane +
// 32 x) with the discrepancy carried ahead instead of summed at the top of
// each iteration.  With coef_r = d_r / b and x^m B written B_r:
//   Lambda_{r+1} = Lambda_r + coef_r B_r, so
//   d_{r+1} = sum_c Lambda_{r+1,c} S_{r+2-c} = P_r + coef_r Q_r, where
//   P_r = sum_c Lambda_{r,c} S_{r+2-c} and Q_r = sum_c B_{r,c} S_{r+2-c};
//   B_{r+1} = x (cond ? Lambda_r : B_r) gives Q_{r+1} = cond ? P_r : Q_r.
// So each iteration sums P_r from Lambda_r (off the serial path) while the
// serial path from d_r to d_{r+1} is one log, one product and one XOR;
// Lambda, B, b and L take exactly the textbook values.  d_0 = Q_0 = S_1.
// Same block skipping as rs_bm.  Returns L; writes log Lambda to logLam.
// d, b and Q are the same for every lane, so their lookups use the plain
// (one copy) tables lexp/llog: a warp-uniform address is one broadcast
// whatever its value, and the address is the index itself, which shortens
// the serial path (about 13 % fewer cycles per iteration than the
// lane-replicated tables).
template <class LV>
__device__ __forceinline__ uint32_t rs_bm_lookahead(const GF& gf, const uint8_t* lexp, const uint16_t* llog,
                                                   const uint16_t* logS, uint16_t* logLam, int lane) {
  constexpr int NR = LV::NR, CAP = LV::CAP, SEG = 32;
  constexpr int NC = cdiv(CAP, SEG);
  uint32_t lam[NC], lbp[NC];
#pragma unroll
  for (int x = 0; x < NC; x++) {
    const int c = lane + SEG * x;
    lam[x] = c == 0;
    lbp[x] = c == 1 ? 0u : GF_LOG_ZERO;  // B = x (m = 1, B = 1)
  }
  uint32_t lb = 0, L = 0;                 // log b (b = 1), LFSR length
  uint32_t d = lexp[logS[0]];             // d_0 = S_1
  uint32_t lq = logS[0];                  // log Q_0 = log S_1
  auto iter = [&](auto na, int rr) {
    constexpr int NA = decltype(na)::value;
    // log Q_r - log b (log-zero kept), formed off the serial path
    const uint32_t lqb = sel(lq >= GF_LOG_ZERO, GF_LOG_ZERO, sel(lq >= lb, lq - lb, lq + 255u - lb));
    uint32_t llam[NA];
    uint32_t part = 0;
#pragma unroll
    for (int x = 0; x < NA; x++) {
      const int c = lane + SEG * x;  // rr + 1 - c >= -64: padding covers c > rr + 1
      llam[x] = gf.log(lam[x]);
      part ^= gf.mul_l(llam[x], logS[rr + 1 - c]);
    }
    const uint32_t P = __reduce_xor_sync(FULL_MASK, part);
    const uint32_t ld = llog[d];
    const uint32_t lcoef = sel(d == 0, GF_LOG_ZERO, sel(ld >= lb, ld - lb, ld + 255u - lb));
    const bool cond = (d != 0) & (2 * L <= (uint32_t)rr);
    uint32_t src[NA];
#pragma unroll
    for (int x = 0; x < NA; x++) {
      lam[x] ^= gf.mul_l(lcoef, lbp[x]);
      src[x] = sel(cond, llam[x], lbp[x]);
    }
#pragma unroll
    for (int x = 0; x < NA; x++) {
      const uint32_t up = __shfl_up_sync(FULL_MASK, src[x], 1);
      const uint32_t carry = x > 0 ? __shfl_sync(FULL_MASK, src[x > 0 ? x - 1 : 0], SEG - 1) : GF_LOG_ZERO;
      const uint32_t nb = lane == 0 ? carry : up;
      lbp[x] = (lane + SEG * x) < CAP ? nb : GF_LOG_ZERO;
    }
    d = P ^ lexp[min(ld + lqb, GF_LOG_ZERO)];  // d_{r+1} = P_r + (d_r / b) Q_r
    lq = sel(cond, (uint32_t)llog[P], lq);     // log Q_{r+1}
    lb = sel(cond, ld, lb);
    L = sel(cond, (uint32_t)rr + 1u - L, L);
  };
  // block x of Lambda_r, B_r is zero while r + 2 <= SEG x; P_r reads
  // Lambda_r only (degree <= r), so the phases of rs_bm hold here too
  auto phase = [&](auto na) {
    constexpr int NA = decltype(na)::value;
    constexpr int R0 = NA == 1 ? 0 : cmin(NR, SEG * (NA - 1) - 2);
    constexpr int R1 = NA == NC ? NR : cmin(NR, SEG * NA - 2);
#pragma unroll 2
    for (int rr = R0; rr < R1; rr++) iter(na, rr);
  };
  static_assert(NC >= 1 && NC <= 2, "look-ahead BM phases");
  phase(std::integral_constant<int, 1>{});
  if constexpr (NC >= 2) phase(std::integral_constant<int, 2>{});
#pragma unroll
  for (int x = 0; x < NC; x++) {
    const int c = lane + SEG * x;
    if (c < CAP) logLam[c] = (uint16_t)gf.log(lam[x]);
  }
  __syncwarp();
  return L;
}

// S8-S9 of ONE received word by a team of T warps (tid = 32 wt + lane):
// the syndromes split by position over the warps, Berlekamp-Massey on warp
// 0 (the serial part), Omega by coefficient over the lanes, and Chien +
// Forney at the k message positions with each position's sums over the
// 2 delta + 1 coefficients split over the warps.  Partial sums meet in
// shared memory between team barriers.  Same field arithmetic as
// rs_decode_seg, with Berlekamp-Massey's discrepancy carried ahead
// (rs_bm_lookahead); only the order of the XORs differs.  rs:
// rs_team_scratch<T>() words of shared scratch (logs of r, S, Lambda and
// Omega, the partial sums, and plain copies of the exp and log tables for
// the warp-uniform lookups).  An inactive word is decoded but not stored.
template <int T>
__host__ __device__ constexpr int rs_team_scratch() { return 176 + 40 * T + 256; }

// Where rs_decode_team keeps log S (indices [-64, 64), log-zero below 0)
// and log Lambda in its scratch; the debug path reads them back from there.
__device__ __forceinline__ uint16_t* rs_team_logS(uint32_t* rs) { return reinterpret_cast<uint16_t*>(rs + 48) + 64; }
__device__ __forceinline__ uint16_t* rs_team_logLam(uint32_t* rs) { return reinterpret_cast<uint16_t*>(rs + 112); }

template <class LV, int T>
__device__ __forceinline__ void rs_decode_team(const GF& gf, uint32_t* rs, const uint8_t* r, int wt, int lane,
                                               const TeamSync& sync, bool active, uint8_t* __restrict__ m_out) {
  constexpr int n1 = LV::n1, k = LV::k, NR = LV::NR, CAP = LV::CAP;
  static_assert(n1 <= 96 && CAP <= 64 && k <= 32, "RS scratch sizes");
  const int tid = wt * 32 + lane;
  uint16_t* logr = reinterpret_cast<uint16_t*>(rs);
  uint16_t* logS = rs_team_logS(rs);
  uint16_t* logLam = rs_team_logLam(rs);
  uint16_t* logOm = reinterpret_cast<uint16_t*>(rs + 144);
  uint8_t* partS = reinterpret_cast<uint8_t*>(rs + 176);           // [T][64] partial syndromes
  uint8_t* partC = reinterpret_cast<uint8_t*>(rs + 176 + 16 * T);  // [T][3][32] partial Chien sums
  uint8_t* lexp = reinterpret_cast<uint8_t*>(rs + 176 + 40 * T);     // plain exp table, 512 bytes
  uint16_t* llog = reinterpret_cast<uint16_t*>(rs + 304 + 40 * T);   // plain log table, 256 halfwords

  for (int j = tid; j < n1; j += 32 * T) logr[j] = (uint16_t)gf.log(r[j]);
  for (int j = tid; j < 64; j += 32 * T) logS[j - 64] = (uint16_t)GF_LOG_ZERO;
  for (int e = tid; e < 512; e += 32 * T) lexp[e] = (uint8_t)gf.exp((uint32_t)e);
  for (int a = tid; a < 256; a += 32 * T) llog[a] = (uint16_t)gf.log((uint32_t)a);
  sync();

  // partial syndromes over positions [J0, J1): lane owns i = lane + 1 + 32 s
  constexpr int NS = cdiv(NR, 32);
  constexpr int JW = cdiv(n1, T);
  {
    const int J0 = wt * JW, J1 = cmin(n1, J0 + JW);
    uint32_t acc[NS], e[NS];
#pragma unroll
    for (int s = 0; s < NS; s++) {
      acc[s] = 0;
      e[s] = ((uint32_t)(lane + 1 + 32 * s) * (uint32_t)J0) % 255u;  // log of alpha^{i J0}
    }
#pragma unroll 2
    for (int j = J0; j < J1; j++) {
      const uint32_t lr = logr[j];
#pragma unroll
      for (int s = 0; s < NS; s++) {
        acc[s] ^= gf.exp(min(lr + e[s], GF_LOG_ZERO));
        e[s] += (uint32_t)(lane + 1 + 32 * s);
        e[s] = e[s] >= 255u ? e[s] - 255u : e[s];
      }
    }
#pragma unroll
    for (int s = 0; s < NS; s++) {
      const int i = lane + 1 + 32 * s;
      if (i <= NR) partS[wt * 64 + i - 1] = (uint8_t)acc[s];
    }
  }
  sync();
  if (wt == 0) {
#pragma unroll
    for (int s = 0; s < NS; s++) {
      const int i = lane + 1 + 32 * s;
      if (i <= NR) {
        uint32_t S = 0;
#pragma unroll
        for (int w = 0; w < T; w++) S ^= partS[w * 64 + i - 1];
        logS[i - 1] = (uint16_t)gf.log(S);
      }
    }
    __syncwarp();
    rs_bm_lookahead<LV>(gf, lexp, llog, logS, logLam, lane);
  }
  sync();

  // Omega_kk for kk = tid < 2 delta: warp wt holds kk < 32 (wt + 1), so it
  // sums over c < min(2 delta, 32 (wt + 1)); warps past 2 delta idle
  if (32 * wt < NR) {
    const int kk = tid;
    const int cend = cmin(NR, 32 * (wt + 1));
    uint32_t om = 0;
#pragma unroll 4
    for (int c = 0; c < cend; c++) {
      const int idx = kk < NR ? kk - c : -1;  // c > kk reads the log-zero padding
      om ^= gf.mul_l(logLam[c], logS[idx]);
    }
    if (kk < NR) logOm[kk] = (uint16_t)gf.log(om);
  }
  sync();

  // Chien + Forney: lane = message position; warp wt sums the terms
  // c in [C0, C1) of Lambda_even, Lambda_odd and Omega at X = alpha^{-j}
  constexpr int CW = cdiv(CAP, T);
  const int pos = lane;
  const uint32_t jj = (uint32_t)((n1 - k) + (pos < k ? pos : 0));
  const uint32_t step = jj == 0 ? 0u : 255u - jj;  // log X
  {
    const int C0 = wt * CW, C1 = cmin(CAP, C0 + CW);
    uint32_t ec = (step * (uint32_t)C0) % 255u;
    uint32_t lev = 0, lod = 0, omv = 0;
#pragma unroll 4
    for (int c = C0; c < C1; c++) {
      const uint32_t t = gf.exp(min((uint32_t)logLam[c] + ec, GF_LOG_ZERO));
      lod ^= (c & 1) ? t : 0u;
      lev ^= (c & 1) ? 0u : t;
      if (c < NR) omv ^= gf.exp(min((uint32_t)logOm[c] + ec, GF_LOG_ZERO));
      ec += step;
      ec = ec >= 255u ? ec - 255u : ec;
    }
    partC[(wt * 3 + 0) * 32 + lane] = (uint8_t)lev;
    partC[(wt * 3 + 1) * 32 + lane] = (uint8_t)lod;
    partC[(wt * 3 + 2) * 32 + lane] = (uint8_t)omv;
  }
  sync();
  if (wt == 0) {
    uint32_t lev = 0, lod = 0, omv = 0;
#pragma unroll
    for (int w = 0; w < T; w++) {
      lev ^= partC[(w * 3 + 0) * 32 + lane];
      lod ^= partC[(w * 3 + 1) * 32 + lane];
      omv ^= partC[(w * 3 + 2) * 32 + lane];
    }
    const bool root = (lev ^ lod) == 0;
    const uint32_t lom = gf.log(omv);
    uint32_t lomx = lom + step;
    lomx = lomx >= 255u ? lomx - 255u : lomx;
    lomx = sel(lom >= GF_LOG_ZERO, GF_LOG_ZERO, lomx);
    const uint32_t ev = sel(root, gf.div_l(lomx, gf.log(lod)), 0u);
    if (pos < k && active) m_out[pos] = (uint8_t)((uint32_t)r[jj] ^ ev);
  }
}

template <class LV, int T = 2, int NI = 2>
struct Team {
  static constexpr int WPT2 = odd_at_least(cdiv(LV::W_v32, 32 * T));
  static constexpr int U2W = round_up(cmax(cdiv(2 * LV::n, 32), 32 * T * WPT2 + (LV::n >> 5) + 1), 4);
  static constexpr int RB = cdiv(LV::n1, 4) * 4;  // bytes per stored RM word
  static constexpr int WORDS = round_up(U2W + LV::WP + NI * (RB / 4), 4);  // shared words per team
  // the RM bytes of the team's NI ciphertexts, RB bytes each, behind u2 and the supports
  __device__ static uint8_t* rbuf(uint32_t* ws) { return reinterpret_cast<uint8_t*>(ws + U2W + LV::WP); }
  static_assert(NI >= 1 && NI <= T, "one RS word per warp at most");
  static_assert(NI * RS_SCRATCH <= U2W && rs_team_scratch<T>() <= U2W, "the RS scratches fit in u2");
  static_assert(U2W % 4 == 0 && LV::WP % 4 == 0 && WORDS % 4 == 0, "16-byte alignment");
};

// S1-S7 of one ciphertext by a team (tid in [0, 32 T)).
template <class LV, bool MASKED, int T = 2>
__device__ __forceinline__ void product_rm_team(uint32_t* ws, int tid, const TeamSync& sync,
                                                const uint64_t* __restrict__ urow, const uint64_t* __restrict__ vrow,
                                                const uint32_t* __restrict__ yrow, uint8_t* r_out) {
  using TT = Team<LV, T>;
  constexpr int WPT = TT::WPT2, W_v32 = LV::W_v32;
  uint32_t* u2 = ws;
  uint32_t* sup = ws + TT::U2W;
  load_supports<LV::n, LV::w, 32 * T>(sup, yrow, tid);
  build_doubled<LV::n, LV::W_u_pitch, TT::U2W, 32 * T>(u2, urow, tid, sync);
  uint32_t acc[WPT];
  rot_xor_product<WPT, LV::w, MASKED, (T >= 4)>(u2, sup, tid * WPT, acc);
  const uint32_t* v32 = reinterpret_cast<const uint32_t*>(vrow);
#pragma unroll
  for (int k = 0; k < WPT; k++) {
    const int i = tid * WPT + k;
    if (i < W_v32) acc[k] ^= __ldcs(v32 + i);
  }
  sync();
#pragma unroll
  for (int k = 0; k < WPT; k++) {
    const int i = tid * WPT + k;
    if (i < W_v32) u2[i] = acc[k];
  }
  sync();
  rm_decode_warp<LV, 16 * T>(u2, r_out, tid);
  sync();
}

// NI ciphertexts per turn: product and RM of each by the whole team, then
// warp wt < NI of the team runs the RS stage of ciphertext wt.
template <class LV, bool MASKED, int T = 2, int NI = 2, class Rows>
__device__ __forceinline__ void decrypt_team(const GF& gf, uint32_t* ws, int wt, int lane, const TeamSync& sync,
                                             const Rows& rows) {
  using TT = Team<LV, T, NI>;
  const int tid = (wt << 5) | lane;
  uint8_t* rbuf = TT::rbuf(ws);
  const uint64_t* u;
  const uint64_t* v;
  const uint32_t* y;
  uint8_t* m;
#pragma unroll 1
  for (int g = 0; g < NI; g++)
    if (rows(g, u, v, y, m)) product_rm_team<LV, MASKED, T>(ws, tid, sync, u, v, y, rbuf + g * TT::RB);
  if constexpr (NI == 1 && T > 1) {
    // one ciphertext per turn: the whole team shares its RS stage
    const bool act = rows(0, u, v, y, m);
    rs_decode_team<LV, T>(gf, ws, rbuf, wt, lane, sync, act, m);
  } else if (wt < NI) {
    const bool act = rows(wt, u, v, y, m);
    rs_decode_seg<LV, 32, false>(gf, ws + wt * RS_SCRATCH, rbuf + wt * TT::RB, lane, act, m, nullptr);
  }
  sync();  // the RS scratch lives in u2: the next turn rebuilds it
}

}  // namespace hqc

// Per-level constants of HQC-1/3/5 (Table I of the paper) and the sizes of
// the GB300 data layout derived from them.  Host and device share this
// header; the CPU oracle keeps its own copy of Table I.
#pragma once
#include <cstdint>

namespace hqc {

// Table I: N, omega, omega_r = omega_e, RS [n1, k, 2 delta + 1],
// duplicated RM(1,7) [n2 = 128 mult, 8, 64 mult].
template <int LEVEL> struct LevelConst;
template <> struct LevelConst<1> {
  static constexpr int n = 17669, w = 66, wr = 75, we = 75;
  static constexpr int n1 = 46, k = 16, delta = 15, mult = 3;
};
template <> struct LevelConst<3> {
  static constexpr int n = 35851, w = 100, wr = 114, we = 114;
  static constexpr int n1 = 56, k = 24, delta = 16, mult = 5;
};
template <> struct LevelConst<5> {
  static constexpr int n = 57637, w = 131, wr = 149, we = 149;
  static constexpr int n1 = 90, k = 32, delta = 29, mult = 5;
};

__host__ __device__ constexpr int cdiv(int a, int b) { return (a + b - 1) / b; }
__host__ __device__ constexpr int odd_at_least(int x) { return x | 1; }
__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }
__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int round_up(int a, int b) { return cdiv(a, b) * b; }

// Layout in HBM (bit i of a vector = bit i%64 of 64-bit word i/64):
//   u  [count][W_u_pitch] uint64  (pitch even -> rows 16-byte aligned)
//   v  [count][W_v]       uint64  (n1*n2 bits exactly)
//   m  [count][k]         uint8
// Layout in shared memory for one ciphertext (32-bit words):
//   u2[U2W]   the 2n-bit string u||u (second copy starts at bit n) so a
//             rotation by p is the 32-bit window at bit offset 32 i + n - p;
//   sup[WP]   two words per support entry: the byte offset of the
//             window's first u2 word and the bit shift (see load_supports).
// After the product the w = v + u*y words overwrite u2[0, W_v32); once the
// RM bytes are out, u2 is scratch for the Reed-Solomon stage.
template <int LEVEL> struct Level : LevelConst<LEVEL> {
  using C = LevelConst<LEVEL>;
  static constexpr int level = LEVEL;
  static constexpr int n2 = 128 * C::mult;
  static constexpr int NR = 2 * C::delta;           // syndromes = n1 - k
  static constexpr int CAP = NR + 1;                // Lambda coefficients
  static constexpr int N32 = cdiv(C::n, 32);
  static constexpr int W_u = cdiv(C::n, 64);
  static constexpr int W_u_pitch = W_u + (W_u & 1);
  static constexpr int W_v = C::n1 * n2 / 64;
  static constexpr int W_v32 = C::n1 * n2 / 32;
  // output words of the truncated product per lane (odd -> a warp's
  // strided shared-memory reads hit 32 distinct banks)
  static constexpr int WPT = odd_at_least(cdiv(W_v32, 32));
  // highest u2 word a lane may read: 32*WPT - 1 + (n >> 5) + 1
  static constexpr int U2W = round_up(cmax(cdiv(2 * C::n, 32), 32 * WPT + (C::n >> 5) + 1), 4);
  static constexpr int WP = round_up(2 * C::w, 4);    // two words per support entry
  static constexpr int WARP_WORDS = U2W + WP;       // u2 and the support list
  // full-length (n-bit) product used by key generation and encryption
  static constexpr int WPT_FULL = odd_at_least(cdiv(N32, 32));
  static constexpr int U2W_FULL = round_up(cmax(cdiv(2 * C::n, 32), 32 * WPT_FULL + (C::n >> 5) + 1), 4);
  static constexpr int WP_R = round_up(2 * C::wr, 4);
  static_assert(C::n1 * n2 % 64 == 0, "v is a whole number of words");
  static_assert(C::n1 - C::k == NR, "RS code has n1 - k = 2 delta");
  static_assert(C::k <= 32, "one message byte per lane");
  static_assert(C::n1 <= 96 && CAP <= 64, "RS scratch sizes");
};

// Strips of the truncated product (W_v32 output words) over the 32 lanes of
// a warp: lane l computes words [start(l), start(l) + len(l)).  At step k
// the warp loads u2 words start(l) + k + offset, so one load instruction
// hits 32 distinct banks (one wavefront, whatever the support entry's
// offset) exactly when the 32 starts are distinct modulo 32, which uniform
// odd strips (start = l WPT) give.  (For HQC-1, whose 552 words are
// 32 x 17.25, strips of 16-18 words with 32 distinct start residues exist
// and cut the longest strip to 18, but measured 1.4 % slower on GB300 than
// the uniform 19.)
template <int LEVEL> struct ProductStrips {
  static constexpr int MAXLEN = Level<LEVEL>::WPT;
  __host__ __device__ static constexpr int len(int) { return MAXLEN; }
  __host__ __device__ static constexpr int start(int l) { return l * MAXLEN; }
};

// Every strip within MAXLEN, starts distinct modulo 32, words [0, W_v32)
// covered, and every window a strip can read inside the U2W words of the
// doubled operand.
template <int LEVEL>
__host__ __device__ constexpr bool product_strips_ok() {
  using LV = Level<LEVEL>;
  using PS = ProductStrips<LEVEL>;
  bool seen[32] = {};
  int end = 0;
  for (int l = 0; l < 32; l++) {
    const int st = PS::start(l), ln = PS::len(l);
    if (ln < 1 || ln > PS::MAXLEN || st != end || seen[st % 32]) return false;
    seen[st % 32] = true;
    end = st + ln;
    if (st + PS::MAXLEN + (LV::n >> 5) + 1 > LV::U2W) return false;
  }
  return end >= LV::W_v32;
}
static_assert(product_strips_ok<1>() && product_strips_ok<3>() && product_strips_ok<5>(), "product strips");

}  // namespace hqc

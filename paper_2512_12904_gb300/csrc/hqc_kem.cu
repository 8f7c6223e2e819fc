// HQC.KEM around the PKE kernels (Sec. II-A: SHAKE-based sampling, the
// domain-separated G and K functions, HHK with implicit rejection;
// Algorithms 1-3), one message per thread for every SHAKE256 call:
//
//   k_shake256        batched SHAKE256 over fixed-length rows
//   k_kem_seed_keys   h, x, y of a key pair from its two 32-byte seeds
//   k_kem_derive      theta = G(m, salt), then r1, r2, e from the theta
//                     stream through the constant-weight sampler
//   k_kem_K2          K = SHAKE256(x || U || V || salt || 4), x = m, or
//                     sigma where the re-encryption did not match
//
// Encapsulation = derive, encrypt, K.  Decapsulation = the fused decryption,
// derive, encrypt-and-compare (k_encrypt with the compare epilogue), K.
//
// Domain bytes and draw order (this library's reading of the paper's G, K
// and sampler):
//   theta   = SHAKE256(m || salt || 0x03)[0:32]
//   r1 r2 e = the 32-bit words of SHAKE256(theta || 0x01), in that order,
//             through the sampler below
//   K       = SHAKE256(x || U || V || salt || 0x04)[0:32], U the ceil(n/8)
//             bytes of u with bits >= n cleared, V the n1 n2 / 8 bytes of v
//   h       = first n bits of SHAKE256(seed_pk || 0x02)
//   x, y    = SHAKE256(seed_sk || 0x01) words through the sampler (x first)
// Constant-weight sampler on 32-bit draws R_i: pos_i = i + floor(R_i (n - i)
// / 2^32), then from i = w - 2 down to 0 pos_i becomes i when it already
// occurs among pos_{i+1..w-1} (Floyd's subset sampling, constant-time form).
#include <cuda_runtime.h>

#include "hqc_device.cuh"
#include "hqc_internal.h"
#include "hqc_keccak.cuh"
#include "hqc_kem_k.cuh"

namespace hqc {

constexpr int KEM_THREADS = 128;
constexpr int KEM_K2_THREADS = 128;  // 64 lane pairs per block: 1,024 blocks for 65,536 items
constexpr int KEM_SEED = 32;

// ---------------------------------------------------------------------------
// Batched SHAKE256 of fixed-length rows (msg [count][len] -> out
// [count][outlen]), bytes assembled one at a time: a general entry point.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(KEM_THREADS) k_shake256(int64_t count, const uint8_t* __restrict__ msg, int len,
                                                         uint8_t* __restrict__ out, int outlen) {
  const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= count) return;
  const uint8_t* row = msg + it * (int64_t)len;
  uint64_t a[25];
  shake256_absorb(a, len, [&](int q) {
    uint64_t v = 0;
#pragma unroll
    for (int b = 0; b < 8; b++) {
      const int o = 8 * q + b;
      if (o < len) v |= (uint64_t)__ldg(row + o) << (8 * b);
    }
    return v;
  });
  uint8_t* orow = out + it * (int64_t)outlen;
  for (int o = 0; o < outlen; o += SHAKE256_RATE) {
#pragma unroll
    for (int i = 0; i < SHAKE256_RATE_WORDS; i++)
#pragma unroll
      for (int b = 0; b < 8; b++) {
        const int p = o + 8 * i + b;
        if (p < outlen) orow[p] = (uint8_t)(a[i] >> (8 * b));
      }
    if (o + SHAKE256_RATE < outlen) keccak_f1600(a);
  }
}

// ---------------------------------------------------------------------------
// Draws from a SHAKE256 stream and the constant-weight sampler.  Each
// thread owns `stride` words of shared memory: 34 words of squeezed output,
// then the positions of the support being drawn as 16-bit halves (n <
// 2^16).  stride is odd, so same-index accesses of a warp hit 32 banks.
// ---------------------------------------------------------------------------
template <int WMAX>
struct DrawSpace {
  static constexpr int BUF = 2 * SHAKE256_RATE_WORDS;  // 34 words per permutation
  static constexpr int stride = (BUF + cdiv(WMAX + 1, 2)) | 1;  // positions and one pad half
};

struct Stream {
  uint64_t a[25];
  uint32_t* buf;  // 34 words of this thread
  int used;

  __device__ __forceinline__ void spill() {
#pragma unroll
    for (int i = 0; i < SHAKE256_RATE_WORDS; i++) {
      buf[2 * i] = (uint32_t)a[i];
      buf[2 * i + 1] = (uint32_t)(a[i] >> 32);
    }
    used = 0;
  }
  // start squeezing: the state holds the absorbed, permuted seed
  __device__ __forceinline__ void begin(uint32_t* b) {
    buf = b;
    spill();
  }
  __device__ __forceinline__ uint32_t next() {
    if (used == 2 * SHAKE256_RATE_WORDS) {
      keccak_f1600(a);
      spill();
    }
    return buf[used++];
  }
};

// Draw one support of weight W over [0, N) into pos (16-bit halves, pos[W]
// = 0xFFFF as a pad that matches nothing) and write it to dst[0..W).  The
// collision test reads the later positions two halves per 32-bit word and
// finds an equal half as a zero half of (pair ^ v v): (t - 0x00010001) &
// ~t & 0x80008000 is nonzero iff some 16-bit half of t is zero.
template <int N, int W>
__device__ __forceinline__ void draw_support(Stream& st, uint16_t* pos, uint32_t* __restrict__ dst) {
  static_assert(N < 0xFFFF, "positions and the pad fit in 16 bits");
  for (int i = 0; i < W; i++) {
    const uint32_t R = st.next();
    pos[i] = (uint16_t)(i + __umulhi(R, (uint32_t)(N - i)));
  }
  pos[W] = 0xFFFFu;
  const uint32_t* pairs = reinterpret_cast<const uint32_t*>(pos);
  constexpr int NP = (W + 1) / 2;  // pairs covering indices 0..W (W odd) or 0..W-1
  for (int i = W - 2; i >= 0; i--) {
    const uint32_t v = pos[i];
    const uint32_t vv = v * 0x10001u;
    const int p0 = (i + 1) >> 1;
    // i even: the first pair holds index i itself in its low half, so only
    // its high half is compared (the zero-half test flags a pair, not which
    // half, once a borrow crosses from a zero low half)
    const uint32_t first = pairs[p0];
    uint32_t t = first ^ vv;
    uint32_t hit = (i & 1) ? ((t - 0x00010001u) & ~t & 0x80008000u) : (uint32_t)((first >> 16) == v);
    for (int p = p0 + 1; p < NP; p++) {
      t = pairs[p] ^ vv;
      hit |= (t - 0x00010001u) & ~t & 0x80008000u;
    }
    pos[i] = (uint16_t)sel(hit != 0u, (uint32_t)i, v);
  }
  for (int i = 0; i < W; i++) dst[i] = pos[i];
}

template <int LEVEL>
__global__ void __launch_bounds__(KEM_THREADS) k_kem_seed_keys(int64_t nkeys, const uint8_t* __restrict__ seed_sk,
                                                              const uint8_t* __restrict__ seed_pk,
                                                              uint64_t* __restrict__ h, uint32_t* __restrict__ x,
                                                              uint32_t* __restrict__ y) {
  using LV = Level<LEVEL>;
  using DS = DrawSpace<LV::w>;
  extern __shared__ __align__(16) uint32_t kem_smem[];
  const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= nkeys) return;
  uint32_t* mine = kem_smem + threadIdx.x * DS::stride;
  // h: first n bits of SHAKE256(seed_pk || 0x02)
  {
    const uint64_t* sp = reinterpret_cast<const uint64_t*>(seed_pk + it * KEM_SEED);
    uint64_t a[25];
    shake256_absorb(a, KEM_SEED + 1, [&](int q) { return q < 4 ? __ldg(sp + q) : 0x02ull; });
    uint64_t* hrow = h + it * LV::W_u_pitch;
    for (int base = 0; base < LV::W_u; base += SHAKE256_RATE_WORDS) {
#pragma unroll
      for (int i = 0; i < SHAKE256_RATE_WORDS; i++) {
        const int wi = base + i;
        uint64_t v = a[i];
        if ((LV::n & 63) && wi == LV::W_u - 1) v &= (1ull << (LV::n & 63)) - 1ull;
        if (wi < LV::W_u) hrow[wi] = v;
      }
      if (base + SHAKE256_RATE_WORDS < LV::W_u) keccak_f1600(a);
    }
    for (int wi = LV::W_u; wi < LV::W_u_pitch; wi++) hrow[wi] = 0;
  }
  // x then y from SHAKE256(seed_sk || 0x01)
  const uint64_t* ss = reinterpret_cast<const uint64_t*>(seed_sk + it * KEM_SEED);
  Stream st;
  shake256_absorb(st.a, KEM_SEED + 1, [&](int q) { return q < 4 ? __ldg(ss + q) : 0x01ull; });
  st.begin(mine);
  uint16_t* pos = reinterpret_cast<uint16_t*>(mine + DS::BUF);
  draw_support<LV::n, LV::w>(st, pos, x + it * LV::w);
  draw_support<LV::n, LV::w>(st, pos, y + it * LV::w);
}

template <int LEVEL>
__global__ void __launch_bounds__(KEM_THREADS) k_kem_derive(int64_t count, const uint8_t* __restrict__ m,
                                                           const uint8_t* __restrict__ salt, uint32_t* __restrict__ r1,
                                                           uint32_t* __restrict__ r2, uint32_t* __restrict__ e) {
  using LV = Level<LEVEL>;
  using DS = DrawSpace<LV::wr>;
  static_assert(LV::we == LV::wr && LV::k % 8 == 0, "Table I: w_e = w_r; k whole words");
  extern __shared__ __align__(16) uint32_t kem_smem[];
  const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= count) return;
  uint32_t* mine = kem_smem + threadIdx.x * DS::stride;
  constexpr int KW = LV::k / 8;
  const uint64_t* mrow = reinterpret_cast<const uint64_t*>(m + it * LV::k);
  const uint64_t* srow = reinterpret_cast<const uint64_t*>(salt + it * KEM_SALT);
  // theta = SHAKE256(m || salt || 0x03)[0:32]
  uint64_t th[25];
  shake256_absorb(th, LV::k + KEM_SALT + 1, [&](int q) {
    return q < KW ? __ldg(mrow + q) : q < KW + 2 ? __ldg(srow + q - KW) : 0x03ull;
  });
  Stream st;
  shake256_absorb(st.a, 33, [&](int q) {
    return q == 0 ? th[0] : q == 1 ? th[1] : q == 2 ? th[2] : q == 3 ? th[3] : 0x01ull;
  });
  st.begin(mine);
  uint16_t* pos = reinterpret_cast<uint16_t*>(mine + DS::BUF);
  draw_support<LV::n, LV::wr>(st, pos, r1 + it * LV::wr);
  draw_support<LV::n, LV::wr>(st, pos, r2 + it * LV::wr);
  draw_support<LV::n, LV::we>(st, pos, e + it * LV::we);
}

// K on lane pairs (kem_K_pair): lane h of the pair keeps the h-th 32-bit
// half of every state lane, so 65,536 messages fill 4,096 warps instead of
// 2,048 (one thread per message measured 0.7 % slower on HQC-1
// decapsulation: the pair's 29 shuffles per round cost most of what the
// warps gain).  x is m, or sigma where the re-encryption did not match
// (ok given and 0), chosen by mask.  Lanes past the batch, and items with a
// key index outside [0, nkeys), hash the last item's (or key 0's) data and
// store nothing: every lane takes part in the shuffles.
template <int LEVEL>
__global__ void __launch_bounds__(KEM_K2_THREADS) k_kem_K2(int64_t count, const uint8_t* __restrict__ m,
                                                          const uint32_t* __restrict__ ok,
                                                          const uint8_t* __restrict__ sigma,
                                                          const int32_t* __restrict__ key_idx, int64_t nkeys,
                                                          const uint64_t* __restrict__ u,
                                                          const uint64_t* __restrict__ v,
                                                          const uint8_t* __restrict__ salt, uint8_t* __restrict__ K) {
  using LV = Level<LEVEL>;
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t h = (uint32_t)(gt & 1);
  const bool in = (gt >> 1) < count;
  const int64_t it = in ? (gt >> 1) : count - 1;
  const uint32_t ki = (uint32_t)__ldg(key_idx + it);
  const bool store = in && ki < (uint64_t)nkeys;  // a skipped item: K untouched (the index is public)
  const uint64_t* mrow = reinterpret_cast<const uint64_t*>(m + it * LV::k);
  uint64_t keep = ~0ull;
  const uint64_t* grow = mrow;
  if (ok) {
    keep = 0ull - (uint64_t)(__ldg(ok + it) != 0u);
    grow = reinterpret_cast<const uint64_t*>(sigma + (int64_t)(ki < (uint64_t)nkeys ? ki : 0u) * LV::k);
  }
  uint32_t a[25];
  kem_K_pair<LV>(h, keep, mrow, grow, u + it * LV::W_u_pitch, v + it * LV::W_v,
                 reinterpret_cast<const uint64_t*>(salt + it * KEM_SALT), a);
  if (store) {
    uint32_t* krow = reinterpret_cast<uint32_t*>(K + it * KEM_KBYTES);
#pragma unroll
    for (int i = 0; i < KEM_KBYTES / 8; i++) krow[2 * i + h] = a[i];
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <class KernelT>
static cudaError_t set_smem(KernelT kern, size_t sm) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
}

static unsigned blocks_for(int64_t count) { return (unsigned)((count + KEM_THREADS - 1) / KEM_THREADS); }

cudaError_t launch_shake256(int64_t count, const uint8_t* msg, int len, uint8_t* out, int outlen, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  k_shake256<<<blocks_for(count), KEM_THREADS, 0, st>>>(count, msg, len, out, outlen);
  return cudaGetLastError();
}

template <int LEVEL>
static cudaError_t seed_keys_level(int64_t nkeys, const uint8_t* seed_sk, const uint8_t* seed_pk, uint64_t* h,
                                   uint32_t* x, uint32_t* y, cudaStream_t st) {
  using DS = DrawSpace<Level<LEVEL>::w>;
  const size_t sm = (size_t)KEM_THREADS * DS::stride * 4;
  cudaError_t e = set_smem(k_kem_seed_keys<LEVEL>, sm);
  if (e != cudaSuccess) return e;
  k_kem_seed_keys<LEVEL><<<blocks_for(nkeys), KEM_THREADS, sm, st>>>(nkeys, seed_sk, seed_pk, h, x, y);
  return cudaGetLastError();
}

template <int LEVEL>
static cudaError_t derive_level(int64_t count, const uint8_t* m, const uint8_t* salt, uint32_t* r1, uint32_t* r2,
                                uint32_t* e_out, cudaStream_t st) {
  using DS = DrawSpace<Level<LEVEL>::wr>;
  const size_t sm = (size_t)KEM_THREADS * DS::stride * 4;
  cudaError_t e = set_smem(k_kem_derive<LEVEL>, sm);
  if (e != cudaSuccess) return e;
  k_kem_derive<LEVEL><<<blocks_for(count), KEM_THREADS, sm, st>>>(count, m, salt, r1, r2, e_out);
  return cudaGetLastError();
}

cudaError_t launch_kem_seed_keys(int level, int64_t nkeys, const uint8_t* seed_sk, const uint8_t* seed_pk,
                                 uint64_t* h, uint32_t* x, uint32_t* y, cudaStream_t st) {
  if (nkeys == 0) return cudaSuccess;
  switch (level) {
    case 1: return seed_keys_level<1>(nkeys, seed_sk, seed_pk, h, x, y, st);
    case 3: return seed_keys_level<3>(nkeys, seed_sk, seed_pk, h, x, y, st);
    case 5: return seed_keys_level<5>(nkeys, seed_sk, seed_pk, h, x, y, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_kem_derive(int level, int64_t count, const uint8_t* m, const uint8_t* salt, uint32_t* r1,
                              uint32_t* r2, uint32_t* e, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  switch (level) {
    case 1: return derive_level<1>(count, m, salt, r1, r2, e, st);
    case 3: return derive_level<3>(count, m, salt, r1, r2, e, st);
    case 5: return derive_level<5>(count, m, salt, r1, r2, e, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_kem_K(int level, int64_t count, const uint8_t* m, const uint32_t* ok, const uint8_t* sigma,
                         const int32_t* key_idx, int64_t nkeys, const uint64_t* u, const uint64_t* v,
                         const uint8_t* salt, uint8_t* K, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  // one message per lane pair
  const unsigned kb = (unsigned)((2 * count + KEM_K2_THREADS - 1) / KEM_K2_THREADS);
  switch (level) {
    case 1: k_kem_K2<1><<<kb, KEM_K2_THREADS, 0, st>>>(count, m, ok, sigma, key_idx, nkeys, u, v, salt, K); break;
    case 3: k_kem_K2<3><<<kb, KEM_K2_THREADS, 0, st>>>(count, m, ok, sigma, key_idx, nkeys, u, v, salt, K); break;
    case 5: k_kem_K2<5><<<kb, KEM_K2_THREADS, 0, st>>>(count, m, ok, sigma, key_idx, nkeys, u, v, salt, K); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace hqc

// ---------------------------------------------------------------------------
// C ABI (include/hqc_gb300.h)
// ---------------------------------------------------------------------------
#include <cstdarg>
#include <cstdio>

#include "../../include/hqc_gb300.h"

namespace {

int kfail(int code, const char* fmt, ...) {
  char buf[400];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  hqc::set_last_error(buf);
  return code;
}

int kcuda(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return HQC_OK;
  return kfail(HQC_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

bool al(const void* p, size_t a) { return p && ((uintptr_t)p % a) == 0; }

size_t r16(size_t b) { return (b + 15) / 16 * 16; }

struct KemWs {
  uint8_t* m;
  uint32_t *r1, *r2, *e, *ok;
  size_t total;
};

KemWs kem_layout(const hqc_params_t& p, int64_t count, void* base) {
  KemWs w;
  uint8_t* b = static_cast<uint8_t*>(base);
  size_t o = 0;
  w.m = b + o;
  o += r16((size_t)count * p.k);
  w.r1 = reinterpret_cast<uint32_t*>(b + o);
  o += r16((size_t)count * p.wr * 4);
  w.r2 = reinterpret_cast<uint32_t*>(b + o);
  o += r16((size_t)count * p.wr * 4);
  w.e = reinterpret_cast<uint32_t*>(b + o);
  o += r16((size_t)count * p.we * 4);
  w.ok = reinterpret_cast<uint32_t*>(b + o);
  o += r16((size_t)count * 4);
  w.total = o;
  return w;
}

}  // namespace

extern "C" {

int hqc_shake256_batch(int64_t count, const uint8_t* msg, int32_t len, uint8_t* out, int32_t outlen, void* stream) {
  if (count < 0 || len < 0 || outlen < 0) return kfail(HQC_EINVAL, "count, len and outlen must be >= 0");
  if (count == 0 || outlen == 0) return HQC_OK;
  if (!out || (len > 0 && !msg)) return kfail(HQC_EINVAL, "NULL argument");
  return kcuda(hqc::launch_shake256(count, msg, len, out, outlen, (cudaStream_t)stream), "shake256 launch");
}

int hqc_kem_keygen(int level, int64_t nkeys, const uint8_t* seed_sk, const uint8_t* seed_pk, uint64_t* h_out,
                   uint32_t* x_out, uint32_t* y_out, uint64_t* s_out, void* stream) {
  hqc_params_t p;
  if (hqc_get_params(level, &p) != HQC_OK) return kfail(HQC_EINVAL, "level must be 1, 3 or 5");
  if (nkeys < 0) return kfail(HQC_EINVAL, "nkeys must be >= 0");
  if (nkeys == 0) return HQC_OK;
  if (!al(seed_sk, 8) || !al(seed_pk, 8)) return kfail(HQC_EINVAL, "seeds must be non-NULL 8-byte aligned");
  if (!al(h_out, 16) || !al(s_out, 16) || !al(x_out, 4) || !al(y_out, 4))
    return kfail(HQC_EINVAL, "h, s (16-byte) and x, y (4-byte) must be non-NULL aligned device pointers");
  cudaStream_t st = (cudaStream_t)stream;
  int rc = kcuda(hqc::launch_kem_seed_keys(level, nkeys, seed_sk, seed_pk, h_out, x_out, y_out, st), "seed keys");
  if (rc != HQC_OK) return rc;
  return kcuda(hqc::launch_keygen(level, nkeys, h_out, x_out, y_out, s_out, st), "keygen launch");
}

size_t hqc_kem_workspace_bytes(int level, int64_t count) {
  hqc_params_t p;
  if (hqc_get_params(level, &p) != HQC_OK || count <= 0) return 0;
  return kem_layout(p, count, nullptr).total;
}

int hqc_kem_encaps(int level, int64_t count, const uint64_t* h, const uint64_t* s, int64_t nkeys,
                   const int32_t* key_idx, const uint8_t* m, const uint8_t* salt, uint64_t* u_out, uint64_t* v_out,
                   uint8_t* K_out, void* workspace, size_t workspace_bytes, void* stream) {
  hqc_params_t p;
  if (hqc_get_params(level, &p) != HQC_OK) return kfail(HQC_EINVAL, "level must be 1, 3 or 5");
  if (count < 0 || nkeys <= 0) return kfail(HQC_EINVAL, "count >= 0 and nkeys >= 1");
  if (count == 0) return HQC_OK;
  if (!al(h, 16) || !al(s, 16) || !al(u_out, 16) || !al(v_out, 16))
    return kfail(HQC_EINVAL, "h, s, u_out, v_out must be non-NULL 16-byte aligned device pointers");
  if (!al(key_idx, 4) || !al(m, 8) || !al(salt, 8) || !al(K_out, 8))
    return kfail(HQC_EINVAL, "key_idx (4-byte), m, salt, K_out (8-byte) must be non-NULL aligned device pointers");
  if (!al(workspace, 16)) return kfail(HQC_EINVAL, "workspace must be a non-NULL 16-byte aligned device pointer");
  const KemWs w = kem_layout(p, count, workspace);
  if (workspace_bytes < w.total)
    return kfail(HQC_ENOMEM, "workspace has %zu bytes, needs %zu", workspace_bytes, w.total);
  cudaStream_t st = (cudaStream_t)stream;
  int rc = kcuda(hqc::launch_kem_derive(level, count, m, salt, w.r1, w.r2, w.e, st), "derive launch");
  if (rc == HQC_OK)
    rc = kcuda(hqc::launch_encrypt_valid(level, count, h, s, nkeys, key_idx, m, w.r1, w.r2, w.e, u_out, v_out, st),
               "encrypt launch");
  if (rc == HQC_OK)
    rc = kcuda(hqc::launch_kem_K(level, count, m, nullptr, nullptr, key_idx, nkeys, u_out, v_out, salt, K_out, st),
               "K launch");
  return rc;
}

int hqc_kem_decaps(int level, int64_t count, const hqc_keyset_t* keys, const uint64_t* h, const uint64_t* s,
                   const uint8_t* sigma, const int32_t* key_idx, const uint64_t* u, const uint64_t* v,
                   const uint8_t* salt, uint8_t* K_out, uint32_t* ok_out, void* workspace, size_t workspace_bytes,
                   void* stream) {
  hqc_params_t p;
  if (hqc_get_params(level, &p) != HQC_OK) return kfail(HQC_EINVAL, "level must be 1, 3 or 5");
  if (count < 0) return kfail(HQC_EINVAL, "count must be >= 0");
  if (count == 0) return HQC_OK;
  if (!keys || keys->level != level) return kfail(HQC_EINVAL, "keys missing or registered for another level");
  if (!al(h, 16) || !al(s, 16) || !al(u, 16) || !al(v, 16))
    return kfail(HQC_EINVAL, "h, s, u, v must be non-NULL 16-byte aligned device pointers");
  if (!al(key_idx, 4) || !al(sigma, 8) || !al(salt, 8) || !al(K_out, 8))
    return kfail(HQC_EINVAL, "key_idx (4-byte), sigma, salt, K_out (8-byte) must be non-NULL aligned device pointers");
  if (ok_out && !al(ok_out, 4)) return kfail(HQC_EINVAL, "ok_out must be 4-byte aligned");
  if (!al(workspace, 16)) return kfail(HQC_EINVAL, "workspace must be a non-NULL 16-byte aligned device pointer");
  const KemWs w = kem_layout(p, count, workspace);
  if (workspace_bytes < w.total)
    return kfail(HQC_ENOMEM, "workspace has %zu bytes, needs %zu", workspace_bytes, w.total);
  uint32_t* ok = ok_out ? ok_out : w.ok;
  cudaStream_t st = (cudaStream_t)stream;
  hqc::DecArgs a;
  a.count = count;
  a.u = u;
  a.v = v;
  a.y = keys->d_table;
  a.key_idx = key_idx;
  a.nkeys = keys->nkeys;
  a.m = w.m;
  int rc = kcuda(hqc::launch_fused(level, true, a, st, hqc::level_cfg(level)), "decrypt launch");
  if (rc == HQC_OK) rc = kcuda(hqc::launch_kem_derive(level, count, w.m, salt, w.r1, w.r2, w.e, st), "derive launch");
  if (rc != HQC_OK) return rc;
  rc = kcuda(hqc::launch_encrypt_compare(level, count, h, s, keys->nkeys, key_idx, w.m, w.r1, w.r2, w.e, u, v, ok, st),
             "re-encrypt launch");
  if (rc == HQC_OK)
    rc = kcuda(hqc::launch_kem_K(level, count, w.m, ok, sigma, key_idx, keys->nkeys, u, v, salt, K_out, st),
               "K launch");
  return rc;
}

}  // extern "C"

/*
 * hqc_gb300.h -- C ABI of the GB300 (sm_103a) batched HQC.PKE library.
 *
 * The operation is HQC.PKE.Decrypt (Algorithm 2 of OptHQC, arXiv
 * 2512.12904): for each ciphertext c = (u, v) and secret support y,
 *     m' = C.Decode(v - u*y)
 * where u*y is the quasi-cyclic product in GF(2)[x]/(x^n - 1) written as the
 * XOR of rotations of u (Eq. 1, Sec. III-B), the difference is truncated to
 * n1*n2 bits, C.Decode is duplicated RM(1,7) decoding per n2-bit block
 * followed by Reed-Solomon decoding over GF(2^8) (Sec. II-A, Sec. III-D).
 * The parameter sets are Table I.  (The paper prints u*s in Algorithm 2;
 * the operand that cancels the public h is the secret y, which is what this
 * library uses.)
 *
 * Conventions shared by every entry point
 *   - Bit i of a vector is bit (i % 64) of 64-bit word i / 64.
 *   - u rows have W_u_pitch 64-bit words (W_u = ceil(n/64) rounded up to
 *     even); bits >= n and the pad word are ignored.  v rows have W_v words
 *     (exactly n1*n2 bits).  m rows have k bytes.
 *   - RS codewords are (parity bytes || message bytes); m' is the last k
 *     bytes of the corrected codeword.
 *   - Data pointers are DEVICE pointers owned by the caller unless stated
 *     otherwise; u, v and arena pointers must be 16-byte aligned.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *     stream-ordered and asynchronous: argument errors are returned at once,
 *     results are ready when the stream reaches the call.
 *   - No entry point allocates device memory, except hqc_keys_register.
 *   - HQC.PKE.Decrypt has no failure output, so m_out is always written.
 *   - Every kernel has data-independent control flow, and no shared-memory
 *     access pattern depends on secret data: GF(2^8) lookups go through
 *     lane-replicated (decoder) or per-lane (encoder) tables, every lane of
 *     a product load reads at the same support entry's offset, and sparse
 *     vectors are added one entry per step by a single lane.
 *   - Return value: HQC_OK or a negative HQC_E* code; hqc_last_error()
 *     gives a message for the calling thread's last error.
 */
#ifndef HQC_GB300_H
#define HQC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HQC_OK 0
#define HQC_EINVAL (-1)     /* bad level, count, pointer, alignment or size */
#define HQC_ENOMEM (-2)     /* workspace too small / allocation failed */
#define HQC_ECUDA (-3)      /* CUDA launch or runtime error (see hqc_last_error) */
#define HQC_ETIMEOUT (-4)   /* a bounded wait gave up */
#define HQC_EBUSY (-5)      /* admission refused (serving) */
#define HQC_EINTERNAL (-6)  /* internal consistency check failed */

/* Table I plus derived sizes.  level in {1, 3, 5}. */
typedef struct hqc_params_s {
  int32_t level;
  int32_t n;          /* ring length */
  int32_t n1, k;      /* RS [n1, k, 2 delta + 1] over GF(2^8) */
  int32_t delta;
  int32_t n2, mult;   /* RM(1,7) duplicated mult times: n2 = 128 mult */
  int32_t w, wr, we;  /* weights of x, y; r1, r2; e */
  int32_t W_u;        /* ceil(n / 64) */
  int32_t W_u_pitch;  /* W_u rounded up to even */
  int32_t W_v;        /* n1 * n2 / 64 */
} hqc_params_t;

/* Fill *out for `level`.  Host only, needs no GPU.  HQC_EINVAL for an
 * unknown level or NULL out. */
int hqc_get_params(int level, hqc_params_t* out);

/* Message of the calling thread's last failed call ("" if none).  The
 * pointer stays valid until the thread's next call into the library. */
const char* hqc_last_error(void);

/* HQC.PKE.Decrypt of `count` ciphertexts with literal supports
 * (Algorithm 2): y is [count][w] uint32 positions of the secret y of each
 * ciphertext.  Entries >= n contribute nothing; repeated entries cancel
 * (the product is a XOR of rotations, Eq. 1).  u [count][W_u_pitch],
 * v [count][W_v], m_out [count][k].  One persistent fused kernel; with the
 * default launch shape, a batch of at most 512 runs the latency form
 * instead (one block of four warps per ciphertext, same results). */
int hqc_decrypt_batch(int level, int64_t count, const uint64_t* u, const uint64_t* v, const uint32_t* y,
                      uint8_t* m_out, void* stream);

/* Secret supports resident on the device, validated once. */
typedef struct hqc_keyset_s hqc_keyset_t;

/* Copy nkeys supports y_host [nkeys][w] (HOST memory) to the current
 * device.  Every entry must be < n and distinct within its row, else
 * HQC_EINVAL.  Allocates device memory; free with hqc_keys_free. */
int hqc_keys_register(int level, int64_t nkeys, const uint32_t* y_host, hqc_keyset_t** out);
int hqc_keys_free(hqc_keyset_t* keys);
/* Level and count of a keyset; the device pointer of its [nkeys][w] table. */
int hqc_keys_info(const hqc_keyset_t* keys, int* level, int64_t* nkeys, const uint32_t** device_table);

/* Decrypt with registered keys: ciphertext i uses key key_idx[i]
 * (device int32 [count]).  Same kernel as hqc_decrypt_batch with
 * validated supports.
 * Key indices: in this and every other entry point that takes key_idx
 * (the staged, no-alloc, plan and host forms, encryption and the KEM), an
 * item whose index lies outside [0, nkeys) is skipped: none of its outputs
 * (m row; u, v rows; K row; ok flag) is written.  The index says which key
 * an item uses, which is public, so skipping it leaks nothing secret.  To
 * learn whether a batch holds such items, call hqc_count_bad_key_idx.  The
 * host-buffer forms (hqc_decrypt_host_keyed, hqc_kem_decaps_host) copy
 * whole chunks back from device slots, so there a skipped item's host rows
 * are set to zero (K zero, ok 0), as hqc_decrypt_mixed_host does for
 * skipped items. */
int hqc_decrypt_batch_keyed(int level, int64_t count, const uint64_t* u, const uint64_t* v, const hqc_keyset_t* keys,
                            const int32_t* key_idx, uint8_t* m_out, void* stream);

/* Number of entries of key_idx (device int32 [count], count < 2^32) that
 * lie outside [0, nkeys), written to *out (device uint32; zeroed by this
 * call on the stream, then counted by one kernel).  The items these
 * entries name are the ones the keyed entry points skip.  The paper has no
 * counterpart: it is an argument check that runs on the device, since the
 * indices live there. */
int hqc_count_bad_key_idx(int64_t count, const int32_t* key_idx, int64_t nkeys, uint32_t* out, void* stream);

/* Plain one-kernel-per-stage form (product, RM decode, RS decode as three
 * launches with intermediates in global memory): the comparison baseline
 * of the fused kernel.  Give either y (literal) or keys + key_idx.
 * workspace: device memory of at least hqc_staged_workspace_bytes(level,
 * count) bytes, 16-byte aligned; its contents on return are unspecified. */
size_t hqc_staged_workspace_bytes(int level, int64_t count);
int hqc_decrypt_batch_staged(int level, int64_t count, const uint64_t* u, const uint64_t* v, const uint32_t* y,
                             const hqc_keyset_t* keys, const int32_t* key_idx, void* workspace,
                             size_t workspace_bytes, uint8_t* m_out, void* stream);

/* S5-S7 alone: decode the n1 duplicated RM(1,7) blocks of each of count
 * received words w [count][W_v] (device, 64-bit words, 16-byte aligned;
 * block j of word i is bits [j n2, (j + 1) n2) of row i) into r_out
 * [count][n1] bytes (device): byte = a* + 128 [F(a*) < 0] with F the
 * Walsh-Hadamard transform of the copy counts and a* = argmax |F|, ties
 * to the smaller a (Sec. II-A; the decoder inside every decryption form).
 * use_tensor_cores = 0 runs the register butterflies of the per-stage
 * form; 1 runs the same transform as one dense product on the tensor
 * cores (tcgen05, fp16 operands, fp32 accumulators in tensor memory, exact
 * for these small integers), a measured alternative.  Both give identical
 * bytes.  Asynchronous on stream; HQC_EINVAL on a bad level, count < 0 or a
 * NULL or misaligned pointer with count > 0. */
int hqc_rm_decode_batch(int level, int64_t count, const uint64_t* w, uint8_t* r_out, int use_tensor_cores,
                        void* stream);
/* Timed-out waits of the tensor-core RM form since the last call
 * (synchronises the current device; reads and clears a device counter).
 * Each wait for the tensor core is bounded: a timeout stops that block,
 * leaves its remaining bytes unwritten and is counted here.  0 in normal
 * operation. */
int hqc_rm_tc_timeouts(int* out);

/* Same per-stage decryption, for callers that cannot allocate device memory
 * at all (a framework that owns every device byte through its own
 * allocator, a latency-critical path where cudaMalloc could block or fail
 * under memory pressure, a service that reserves all of its memory at
 * load).  The paper has no counterpart to this entry point.
 *   - No allocation: the intermediates live in one array of
 *     HQC_NOALLOC_SCRATCH_BYTES compiled into the library, which every GPU
 *     that loads the library holds until the process exits.
 *   - Size limit: count may be at most (HQC_NOALLOC_SCRATCH_BYTES - 16) /
 *     (8 W_v + n1): 7443 (HQC-1), 3698 (HQC-3), 2301 (HQC-5) per call.  A
 *     larger count returns HQC_EINVAL (message in hqc_last_error) and
 *     launches nothing.
 *   - Device: the call works on the CURRENT device (cudaSetDevice); u, v,
 *     the keys, m_out and the stream must belong to it.
 *   - First call on a device: it looks up the array's device address with
 *     cudaGetSymbolAddress once (per device, that device current), so make
 *     that first call outside any stream capture.  The address is cached
 *     for the life of the process; do not call this entry point again
 *     after cudaDeviceReset in the same process (the cached address would
 *     point into the destroyed context).
 *   - Sharing: every call on a device uses the same array, and each call
 *     overwrites all of the part it reads before reading it (nothing needs
 *     to start at zero).  Calls whose work overlaps on the GPU -- two
 *     streams, or two host threads -- race on the array; order them on one
 *     stream or synchronize between them.
 * Arguments and errors are those of hqc_decrypt_batch_staged minus the
 * workspace. */
#define HQC_NOALLOC_SCRATCH_BYTES (16u << 20)
int hqc_decrypt_batch_staged_noalloc(int level, int64_t count, const uint64_t* u, const uint64_t* v,
                                     const uint32_t* y, const hqc_keyset_t* keys, const int32_t* key_idx,
                                     uint8_t* m_out, void* stream);

/* Decryption straight from host buffers, with uploads overlapped with the
 * kernels: the batch is cut into chunks of `chunk` ciphertexts that
 * alternate between two device slots in `workspace` (device memory of at
 * least hqc_host_workspace_bytes(level, chunk) bytes), uploaded on an
 * internal copy stream while the previous chunk is decrypted and its m
 * copied back on an internal compute stream (both created once per
 * device).  chunk <= 0 picks whole waves of the persistent grid, about
 * eight chunks per batch, as large as the workspace holds.  u_host, v_host,
 * key_idx_host and m_host are HOST memory and should be pinned for the
 * copies to overlap.  The call is ordered after
 * earlier work on `stream`, and `stream` waits for its completion; m_host is
 * valid once `stream` reaches that point. */
size_t hqc_host_workspace_bytes(int level, int64_t chunk);
int hqc_decrypt_host_keyed(int level, int64_t count, const uint64_t* u_host, const uint64_t* v_host,
                           const hqc_keyset_t* keys, const int32_t* key_idx_host, uint8_t* m_host, int64_t chunk,
                           void* workspace, size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------------
 * KEM (Sec. II-A: SHAKE-based sampling, domain-separated G and K, the HHK
 * transform with implicit rejection; Algorithms 1-3).  The paper names
 * these functions but not their inputs; this library's reading:
 *   theta   = SHAKE256(m || salt || 0x03)[0:32]          (G)
 *   r1 r2 e = 32-bit little-endian words of SHAKE256(theta || 0x01), in
 *             that order, each support through the sampler below
 *   K       = SHAKE256(x || U || V || salt || 0x04)[0:32], x = m, or sigma
 *             when decapsulation rejects; U = ceil(n/8) bytes of u with bits
 *             >= n cleared, V = n1 n2 / 8 bytes of v
 *   h       = first n bits of SHAKE256(seed_pk || 0x02); x then y from the
 *             words of SHAKE256(seed_sk || 0x01) through the sampler
 * Sampler on draws R_i: pos_i = i + floor(R_i (n - i) / 2^32), then for
 * i = w-2 down to 0, pos_i = i if it already occurs among pos_{i+1..w-1}.
 * salt: 16 bytes per ciphertext.  All buffers are device memory, rows
 * contiguous; m, salt, sigma, K, seeds 8-byte aligned; u, v, h, s 16-byte.
 * Not claimed bit-compatible with other HQC implementations. */

/* SHAKE256 (FIPS 202) of `count` rows of `len` bytes: msg [count][len] ->
 * out [count][outlen], one row per GPU thread. */
int hqc_shake256_batch(int64_t count, const uint8_t* msg, int32_t len, uint8_t* out, int32_t outlen, void* stream);

/* Key pairs from seeds (Algorithm 3): seed_sk, seed_pk [nkeys][32] ->
 * h_out, s_out [nkeys][W_u_pitch] (pad word zero), x_out, y_out [nkeys][w]
 * (register y_out with hqc_keys_register for decapsulation). */
int hqc_kem_keygen(int level, int64_t nkeys, const uint8_t* seed_sk, const uint8_t* seed_pk, uint64_t* h_out,
                   uint32_t* x_out, uint32_t* y_out, uint64_t* s_out, void* stream);

/* Device workspace that hqc_kem_encaps / hqc_kem_decaps need for `count`
 * items (0 for a bad level or count <= 0). */
size_t hqc_kem_workspace_bytes(int level, int64_t count);

/* Encapsulation: item i encrypts m[i] under key key_idx[i] of (h, s)
 * ([nkeys][W_u_pitch]) with the randomness drawn from G(m[i], salt[i]),
 * writes (u_out, v_out) and K_out [count][32].  Three kernels: derive,
 * encrypt, K.  HQC_ENOMEM if the workspace is short. */
int hqc_kem_encaps(int level, int64_t count, const uint64_t* h, const uint64_t* s, int64_t nkeys,
                   const int32_t* key_idx, const uint8_t* m, const uint8_t* salt, uint64_t* u_out, uint64_t* v_out,
                   uint8_t* K_out, void* workspace, size_t workspace_bytes, void* stream);

/* Decapsulation: decrypt with the registered y (keys), re-derive the
 * randomness, re-encrypt under (h, s) of the same key and compare with
 * (u, v) on the n and n1 n2 bits; K_out [count][32] = K(m', c) on a match,
 * K(sigma[key], c) otherwise (sigma [nkeys][k]), selected by mask.  ok_out
 * (optional, [count] uint32) receives 1 on a match.  Four kernels: fused
 * decrypt, derive, re-encrypt-and-compare, K.  An item whose key index is
 * outside [0, nkeys) is skipped: its K_out row and ok_out entry are not
 * written (as in encapsulation, where its u, v and K rows are not). */
int hqc_kem_decaps(int level, int64_t count, const hqc_keyset_t* keys, const uint64_t* h, const uint64_t* s,
                   const uint8_t* sigma, const int32_t* key_idx, const uint64_t* u, const uint64_t* v,
                   const uint8_t* salt, uint8_t* K_out, uint32_t* ok_out, void* workspace, size_t workspace_bytes,
                   void* stream);

/* Decapsulation from host buffers with uploads overlapped with the kernels,
 * as hqc_decrypt_host_keyed does for decryption: key_idx_host, u_host,
 * v_host, salt_host are HOST memory (pinned for overlap), K_host
 * [count][32] and ok_host ([count], may be NULL) receive the results; h,
 * s, sigma and keys are the device-resident key material of
 * hqc_kem_decaps.  workspace: device memory of at least
 * hqc_kem_host_workspace_bytes(level, chunk) bytes; chunk <= 0 lets the
 * library choose, bounded by the workspace. */
size_t hqc_kem_host_workspace_bytes(int level, int64_t chunk);
int hqc_kem_decaps_host(int level, int64_t count, const hqc_keyset_t* keys, const uint64_t* h, const uint64_t* s,
                        const uint8_t* sigma, const int32_t* key_idx_host, const uint64_t* u_host,
                        const uint64_t* v_host, const uint8_t* salt_host, uint8_t* K_host, uint32_t* ok_host,
                        int64_t chunk, void* workspace, size_t workspace_bytes, void* stream);

/* Every intermediate of Algorithm 2, per ciphertext (device arrays):
 *   t    [count][W_v]  u*y truncated to n1*n2 bits
 *   w    [count][W_v]  v + t
 *   r    [count][n1]   RM-decoded bytes
 *   S    [count][2 delta]      syndromes S_1..S_2delta
 *   lam  [count][2 delta + 1]  error locator Lambda_0..Lambda_2delta
 *   L    [count]               Berlekamp-Massey length
 *   errmask, errval, cw [count][n1]  Chien roots, Forney values, corrected word
 *   flag [count]  1 if L > delta or #roots != L (test aid, not an HQC output) */
typedef struct hqc_debug_dump_s {
  uint64_t* t;
  uint64_t* w;
  uint8_t* r;
  uint8_t* S;
  uint8_t* lam;
  int32_t* L;
  uint8_t* errmask;
  uint8_t* errval;
  uint8_t* cw;
  int32_t* flag;
} hqc_debug_dump_t;

/* Per-stage decrypt that also writes every intermediate.  dump points to
 * HOST memory holding device pointers; all ten must be non-NULL. */
int hqc_decrypt_debug(int level, int64_t count, const uint64_t* u, const uint64_t* v, const uint32_t* y,
                      const hqc_debug_dump_t* dump, uint8_t* m_out, void* stream);

/* The fused kernels' own intermediates: decrypt with literal supports
 * through form 0 (a block of four warps per ciphertext, k_decrypt_latency),
 * form 1 (a cluster of four blocks per ciphertext,
 * k_decrypt_latency_cluster) or form 2 (the per-turn code of the persistent
 * throughput kernels: k_decrypt_fused's solo warps with G words per turn,
 * HQC-1's Horner syndromes included, or k_decrypt_team's two-warp teams for
 * HQC-5), whatever the count, and write each ciphertext's RM bytes
 * (dump->r), syndromes (dump->S) and Lambda (dump->lam) as the warps that
 * ran RS hold them.  dump points to HOST
 * memory holding device pointers; r, S and lam must be non-NULL, the other
 * fields are ignored.  HQC_EINVAL on a bad form or pointer. */
int hqc_decrypt_debug_team(int level, int form, int64_t count, const uint64_t* u, const uint64_t* v, const uint32_t* y,
                           const hqc_debug_dump_t* dump, uint8_t* m_out, void* stream);

/* Mixed-level batch in one persistent launch.  items: device array of
 * `count` work items; u and v rows are read from `arena` (device, 64-bit
 * words) at the given word offsets (u_off even), m is written to
 * m_arena + m_off.  keys[0..2]: keysets for levels 1, 3, 5 (NULL if a level
 * is absent).  An item whose level, key or offsets fall outside these
 * arrays is skipped and its m bytes are left untouched.  workspace: at
 * least hqc_mixed_workspace_bytes() bytes of device memory (a work
 * counter, zeroed on the stream by this call).  With the default launch
 * shape, batches of at most 512 items run the latency form: a team of four
 * warps per item, one item per team, so the slowest item's chain is split
 * over 128 lanes. */
typedef struct hqc_item_s {
  int32_t level;
  int32_t key;
  int64_t u_off;
  int64_t v_off;
  int64_t m_off;
} hqc_item_t;

size_t hqc_mixed_workspace_bytes(void);
int hqc_decrypt_mixed(int64_t count, const hqc_item_t* items, const uint64_t* arena, int64_t arena_words,
                      const hqc_keyset_t* const keys[3], uint8_t* m_arena, int64_t m_bytes, void* workspace,
                      size_t workspace_bytes, void* stream);

/* Mixed-level decryption from host buffers with uploads overlapped with the
 * kernels.  items_host, arena_host (HOST memory, pinned for overlap) as for
 * hqc_decrypt_mixed, with the items in arena order: u_off and m_off
 * non-decreasing, so each chunk's rows and m bytes are one contiguous range
 * (HQC_EINVAL otherwise).  Per chunk (chunk <= 0: about four) the records
 * and the arena range go up, a one-block kernel groups the records by
 * level, one persistent kernel per level decrypts, and the chunk's m range
 * comes back to m_host; m bytes that no valid item writes are set to zero.
 * workspace: device memory of at least hqc_mixed_host_workspace_bytes(count,
 * items_host, chunk) bytes (0 on bad arguments). */
size_t hqc_mixed_host_workspace_bytes(int64_t count, const hqc_item_t* items_host, int64_t chunk);
int hqc_decrypt_mixed_host(int64_t count, const hqc_item_t* items_host, const uint64_t* arena_host,
                           int64_t arena_words, const hqc_keyset_t* const keys[3], uint8_t* m_host, int64_t m_bytes,
                           int64_t chunk, void* workspace, size_t workspace_bytes, void* stream);

/* Launch shape of the persistent kernels: warps per block and blocks per
 * SM (0 = the library's default).  level 1/3/5 sets the single-level
 * kernels, level 0 the mixed kernel.  Not thread-safe against concurrent
 * launches. */
typedef struct hqc_launch_cfg_s {
  int32_t warps_per_cta;
  int32_t ctas_per_sm;
} hqc_launch_cfg_t;

int hqc_set_launch_config(int level, const hqc_launch_cfg_t* cfg);
/* Resolved shape on the current device: warps per block, blocks per SM and
 * grid size of the persistent launch (keyed selects the kernel variant). */
int hqc_get_launch_shape(int level, int keyed, int32_t* warps, int32_t* ctas_per_sm, int32_t* grid);

/* Plans: one fixed batch (these exact pointers and count) captured in a
 * CUDA graph and replayed with hqc_plan_launch (one graph launch per
 * batch).  Creating a plan allocates small plan-owned device buffers and,
 * with autotune != 0, first times candidates on `stream` with the caller's
 * data (which writes m_out); launching allocates nothing.  The data behind
 * the pointers may change between launches, the pointers and count may
 * not.  Every candidate computes the same messages; only speed differs.
 *   keyed: the persistent kernel of hqc_decrypt_batch_keyed.  The tuner
 *          times every kernel variant -- the library's default choice,
 *          solo warps taking G = 1, 2 or 4 ciphertexts per turn (their RS
 *          stages side by side on 32 / G lanes; no G = 4 at HQC-5), two-warp
 *          teams sharing one doubled operand -- at every launch shape
 *          (warps per block x blocks per SM) and keeps the fastest.
 *   mixed: the items of hqc_decrypt_mixed.  The tuner compares the single
 *          mixed persistent kernel (form 1) with three level-split forms:
 *          the list is split by level once at creation, then one
 *          persistent kernel per level runs either side by side as
 *          parallel graph branches on a tuned share of the SMs each (form
 *          2), or one after another on the whole GPU (form 3); or one
 *          launch runs all three, its blocks taking a level by block range
 *          with that level's warp count and shared-memory layout (form 4).
 *          Forms 2-4 use per level the kernel variant that ran it fastest
 *          alone. */
typedef struct hqc_plan_s hqc_plan_t;
int hqc_plan_create_keyed(int level, int64_t count, const uint64_t* u, const uint64_t* v, const hqc_keyset_t* keys,
                          const int32_t* key_idx, uint8_t* m_out, int autotune, void* stream, hqc_plan_t** out);
int hqc_plan_create_mixed(int64_t count, const hqc_item_t* items, const uint64_t* arena, int64_t arena_words,
                          const hqc_keyset_t* const keys[3], uint8_t* m_arena, int64_t m_bytes, int autotune,
                          void* stream, hqc_plan_t** out);
/* Plans with a configuration the caller names instead of tuning (for
 * instance one that hqc_plan_describe reported for the same batch shape
 * earlier), so that start-up can skip the tuner:
 *   keyed: variant 0 the library's default, 1/2/3 solo warps with G =
 *          1/2/4 ciphertexts per turn (3 not at level 5), 4 two-warp teams;
 *          cfg the launch shape (NULL or zeros: the variant's default).
 *   mixed: form 1-4 as above; cfg the shape of form 1; variants3 the kernel
 *          variant of levels 1, 3, 5 for forms 2 and 3 (NULL: 0); grids3
 *          the blocks per level for forms 2 and 4 (each >= 1 for a level
 *          present).  Form 4's kernel fixes its variants (G = 2, G = 1,
 *          teams).
 * HQC_EINVAL for a variant, form or shape that does not exist; a shape
 * that does not fit the device fails at creation with HQC_ECUDA. */
int hqc_plan_create_keyed_fixed(int level, int64_t count, const uint64_t* u, const uint64_t* v,
                                const hqc_keyset_t* keys, const int32_t* key_idx, uint8_t* m_out, int variant,
                                const hqc_launch_cfg_t* cfg, void* stream, hqc_plan_t** out);
int hqc_plan_create_mixed_fixed(int64_t count, const hqc_item_t* items, const uint64_t* arena, int64_t arena_words,
                                const hqc_keyset_t* const keys[3], uint8_t* m_arena, int64_t m_bytes, int form,
                                const hqc_launch_cfg_t* cfg, const int32_t* variants3, const int32_t* grids3,
                                void* stream, hqc_plan_t** out);
int hqc_plan_launch(hqc_plan_t* plan, void* stream);
/* form: 0 keyed, 1 mixed single kernel, 2 mixed level-partitioned, 3 mixed
 * per-level sequential, 4 mixed one launch by block ranges; cfg: the
 * chosen shape (forms 0, 1); grids3: blocks per level 1/3/5 (forms 2, 4);
 * tuned_ms: the best time the tuner measured (0 without autotune). */
int hqc_plan_info(const hqc_plan_t* plan, int32_t* form, hqc_launch_cfg_t* cfg, int32_t* grids3, float* tuned_ms);
/* The plan's choice and every candidate the tuner timed, as one JSON
 * object written to buf (host memory, cap bytes, NUL-terminated):
 * {"form", "variant" (keyed) or "level_variants" (mixed), "warps_per_cta",
 *  "ctas_per_sm", "grids", "tuned_ms", "candidates": [{"form",
 *  "whole_batch", "levels", "variants", "warps", "ctas", "grids", "ms"},
 *  ...] fastest first}.  Mixed plans also list the per-level solo runs that
 * chose each level's variant (whole_batch false, levels: the one level
 * timed).  HQC_ENOMEM (and nothing written) if cap is too small. */
int hqc_plan_describe(const hqc_plan_t* plan, char* buf, size_t cap);
int hqc_plan_destroy(hqc_plan_t* plan);

/* Continuous-batching service loop over an open-loop request trace.
 *
 * Request i (i < count) arrives arrival_ns[i] nanoseconds after the call
 * starts (non-decreasing) and uses ring entry j = i % ring->period: level
 * ring->level[j], key ring->key[j] (an index into keys[level]), its u row
 * then v row at ring->words + ring->word_off[j] (PINNED host memory,
 * entries contiguous in ring order, word_off[period] = total words), and
 * its k result bytes at m_out + ring->m_off[j] (host; NULL to drop results;
 * a later request on the same entry overwrites them).
 * One host thread admits arrived requests into batches for `streams` CUDA
 * streams while a batch fits that stream's budget_bytes / streams (of
 * request bytes in flight) and max_batch requests.  Batches run
 * concurrently, and new arrivals are admitted whenever a stream frees up.
 * A batch of at most 512 requests is one launch of the latency form, a
 * larger one one persistent kernel per level present.  How the request
 * bytes reach the GPU (cfg->transfer):
 *   1  copy mode: one H2D copy of the batch's ring range into device
 *      memory, the kernels, one D2H copy of the m bytes;
 *   2  in place: the kernels read the batch's u and v rows straight from
 *      the host ring and write m into mapped pinned memory, so no copy
 *      engine is on the request path.  Needs a ring the device can address
 *      (mapped pinned memory, or any host memory on a device that uses the
 *      host's page tables, such as GB300 with its C2C link), 16-byte
 *      aligned, with even word offsets; HQC_EINVAL otherwise;
 *   0  in place when possible, else copy mode (stats->in_place says which).
 * On GB300 the copy engines' H2D rate was measured to collapse from ~192 to
 * ~8 GB/s for tens of milliseconds about twice a second, while SM loads
 * from the same memory hold ~182 GB/s, which is why 0 prefers in place.
 * word_off and m_off must start at 0 and never decrease (HQC_EINVAL
 * otherwise).
 * A request that arrives while max_queue requests wait is rejected.
 * Outputs per request: status[i] (HQC_STATUS_*) and latency_ns[i] =
 * completion time - arrival time (-1 unless DONE).  The call allocates the
 * budget at start and frees it before returning; it returns when every
 * request is answered.
 * A batch still incomplete stall_ms after its launch ends the call with
 * HQC_ETIMEOUT: the batches in flight are then waited for, again at most
 * stall_ms plus one second, and their buffers freed only if they finished
 * (a batch that never finishes keeps its device and pinned memory).
 * Requests not answered by then keep status QUEUED or RUNNING, and stats
 * counts what completed before the stall. */
#define HQC_STATUS_DONE 0
#define HQC_STATUS_QUEUED 1
#define HQC_STATUS_RUNNING 2
#define HQC_STATUS_REJECTED 3   /* queue full when it arrived */
#define HQC_STATUS_INVALID 4    /* bad level, absent keyset or key index out of range */
#define HQC_STATUS_TOO_LARGE 5  /* does not fit one stream's memory share */
typedef struct hqc_serve_cfg_s {
  int32_t streams;        /* batches in flight, 1..16 */
  int32_t max_batch;      /* requests per batch at most */
  int64_t budget_bytes;   /* device memory for request data, split over the streams */
  int64_t max_queue;      /* waiting requests at most */
  int32_t warps_per_cta;  /* launch shape of the per-level kernels (0 = default) */
  int32_t stall_ms;       /* per-batch completion limit in ms (0 = 10,000; < 0 is an error) */
  int32_t transfer;       /* 0 in place when possible, 1 copy engines, 2 in place (see above) */
} hqc_serve_cfg_t;
typedef struct hqc_serve_ring_s {
  int64_t period;
  const int32_t* level;     /* [period] */
  const int32_t* key;       /* [period] */
  const int64_t* word_off;  /* [period + 1] */
  const uint64_t* words;    /* pinned host */
  const int64_t* m_off;     /* [period + 1] */
} hqc_serve_ring_t;
typedef struct hqc_serve_stats_s {
  int64_t completed, rejected_queue, rejected_invalid, rejected_size, batches;
  double mean_batch;
  int64_t wall_ns;          /* start to last completion */
  int64_t items_per_slot;   /* batch capacity the budget allows */
  int64_t in_place;         /* 1 if the kernels read the ring in place, 0 if copied */
} hqc_serve_stats_t;
int hqc_serve_run(const hqc_serve_cfg_t* cfg, const hqc_keyset_t* const keys[3], const hqc_serve_ring_t* ring,
                  int64_t count, const int64_t* arrival_ns, int32_t* status, int64_t* latency_ns, uint8_t* m_out,
                  hqc_serve_stats_t* stats);

/* Key generation core of Algorithm 3: s = x + h*y per key.
 * h, s_out [nkeys][W_u_pitch]; x, y [nkeys][w] (device). */
int hqc_keygen_batch(int level, int64_t nkeys, const uint64_t* h, const uint32_t* x, const uint32_t* y,
                     uint64_t* s_out, void* stream);

/* HQC.PKE.Encrypt (Algorithm 1): u = r1 + h*r2, v = first n1*n2 bits of
 * C.Encode(m) + s*r2 + e.  h, s [nkeys][W_u_pitch]; key_idx [count] (an
 * item whose index is outside [0, nkeys) is skipped: its u and v rows are
 * not written); m [count][k]; r1, r2
 * [count][wr]; e [count][we]; u_out [count][W_u_pitch] (pad bits zero);
 * v_out [count][W_v]. */
int hqc_encrypt_batch(int level, int64_t count, const uint64_t* h, const uint64_t* s, int64_t nkeys,
                      const int32_t* key_idx, const uint8_t* m, const uint32_t* r1, const uint32_t* r2,
                      const uint32_t* e, uint64_t* u_out, uint64_t* v_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HQC_GB300_H */

// Internal launch interface between the C ABI (hqc_abi.cu) and the kernel
// translation units.  Not installed; the public interface is
// include/hqc_gb300.h.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

// A registered keyset (public handle hqc_keyset_t).
struct hqc_keyset_s {
  int level;
  int64_t nkeys;
  int device;
  uint32_t* d_table;  // [nkeys][w] support positions, each < n, distinct per row
};

namespace hqc {

// Launch shape of the persistent fused kernel: warps per block and blocks
// per SM (0 = the library's choice for the level).
struct LaunchCfg {
  int warps_per_cta = 0;
  int ctas_per_sm = 0;
};

struct DecArgs {
  int64_t count = 0;
  const uint64_t* u = nullptr;      // [count][W_u_pitch]
  const uint64_t* v = nullptr;      // [count][W_v]
  const uint32_t* y = nullptr;      // literal: [count][w]; keyed: [nkeys][w]
  const int32_t* key_idx = nullptr; // keyed: [count]
  int64_t nkeys = 0;
  uint8_t* m = nullptr;             // [count][k]
};

struct DebugArgs {
  uint64_t* t;        // [count][W_v]
  uint64_t* w;        // [count][W_v]
  uint8_t* r;         // [count][n1]
  uint8_t* S;         // [count][2 delta]
  uint8_t* lam;       // [count][2 delta + 1]
  int32_t* L;         // [count]
  uint8_t* errmask;   // [count][n1]
  uint8_t* errval;    // [count][n1]
  uint8_t* cw;        // [count][n1]
  int32_t* flag;      // [count]
};

// Mixed-level work item (see hqc_item_t in the public header).
struct MixedItem {
  int32_t level;
  int32_t key;
  int64_t u_off;
  int64_t v_off;
  int64_t m_off;
};

struct MixedArgs {
  int64_t count = 0;
  const MixedItem* items = nullptr;
  const uint64_t* arena = nullptr;  // u and v rows
  int64_t arena_words = 0;
  const uint32_t* keys[3] = {nullptr, nullptr, nullptr};  // levels 1, 3, 5: [nkeys][w]
  int64_t nkeys[3] = {0, 0, 0};
  uint8_t* m = nullptr;
  int64_t m_bytes = 0;
  uint32_t* counter = nullptr;      // dynamic scheduling counter (zeroed before launch)
};

int level_index(int level);  // 1 -> 0, 3 -> 1, 5 -> 2, else -1
void set_last_error(const char* msg);  // message returned by hqc_last_error() on this thread

cudaError_t launch_fused(int level, bool keyed, const DecArgs& a, cudaStream_t st, const LaunchCfg& cfg);
cudaError_t launch_staged(int level, bool keyed, const DecArgs& a, uint64_t* w_ws, uint8_t* r_ws, cudaStream_t st);
cudaError_t launch_debug(int level, const DecArgs& a, const DebugArgs& d, cudaStream_t st);
// The latency forms (form 0: a four-warp team per item, 1: a cluster of four
// blocks) with literal supports, dumping each item's r, S and lam to d.
cudaError_t launch_debug_team(int level, int form, const DecArgs& a, const DebugArgs& d, cudaStream_t st);
// S5-S7 alone on [count][W_v] words: the register butterflies (k_stage_rm)
// or the tensor-core product (hqc_rm_tc.cu); and the tensor-core form's
// count of timed-out waits since the last call (read and cleared).
cudaError_t launch_rm_decode(int level, int64_t count, const uint64_t* w, uint8_t* r, bool tensor_cores,
                             cudaStream_t st);
cudaError_t rm_tc_take_timeouts(int* out);
cudaError_t launch_mixed(const MixedArgs& a, cudaStream_t st, const LaunchCfg& cfg);
// Latency form of the mixed kernel: a team of warps per item, one item per
// team at a time, for batches of at most MIXED_LATENCY_MAX items.
constexpr int64_t MIXED_LATENCY_MAX = 512;
cudaError_t launch_mixed_latency(const MixedArgs& a, cudaStream_t st);
cudaError_t fused_occupancy(int level, bool keyed, const LaunchCfg& cfg, int* warps, int* ctas_per_sm, int* grid);
// Ciphertexts one full wave of the persistent fused grid decrypts at once.
cudaError_t fused_wave(int level, bool keyed, const LaunchCfg& cfg, int64_t* items);
// The launch shape hqc_set_launch_config chose for a level (1, 3, 5).
LaunchCfg level_cfg(int level);
// One level's items of a mixed list (a.items all of that level), at most
// `grid` blocks (0 = a full persistent grid).
cudaError_t launch_items(int level, const MixedArgs& a, int grid, cudaStream_t st, const LaunchCfg& cfg);
cudaError_t items_occupancy(int level, const LaunchCfg& cfg, int* warps, int* ctas_per_sm, int* grid);
cudaError_t mixed_occupancy(const LaunchCfg& cfg, int* warps, int* ctas_per_sm, int* grid);

// Kernel variants of the keyed and per-level persistent decryption that
// the plans' tuner times (hqc_tune.cu).  VAR_DEFAULT is the library's own
// choice (launch_fused / launch_items); the others fix the mapping of
// ciphertexts to warps: solo warps with G = 1, 2, 4 per turn, or two-warp
// teams.  HQC-5 has no G = 4 instance.
enum DecVariant : int { VAR_DEFAULT = 0, VAR_SOLO1 = 1, VAR_SOLO2 = 2, VAR_SOLO4 = 3, VAR_TEAM = 4, VAR_COUNT = 5 };
bool variant_exists(int level, int variant);
const char* variant_name(int variant);
cudaError_t launch_fused_variant(int level, int variant, const DecArgs& a, cudaStream_t st, const LaunchCfg& cfg);
cudaError_t launch_items_variant(int level, int variant, const MixedArgs& a, int grid, cudaStream_t st,
                                 const LaunchCfg& cfg);
cudaError_t items_variant_occupancy(int level, int variant, const LaunchCfg& cfg, int* warps, int* ctas_per_sm,
                                    int* grid);
// One launch over the three per-level lists of a partitioned mixed batch,
// grid[li] blocks for level li (0 for an empty list).
cudaError_t launch_mixed_ranges(const MixedArgs part[3], const int grid[3], cudaStream_t st);

cudaError_t launch_keygen(int level, int64_t nkeys, const uint64_t* h, const uint32_t* x, const uint32_t* y,
                          uint64_t* s, cudaStream_t st);
cudaError_t launch_encrypt(int level, int64_t count, const uint64_t* h, const uint64_t* s, int64_t nkeys,
                           const int32_t* key_idx, const uint8_t* m, const uint32_t* r1, const uint32_t* r2,
                           const uint32_t* e, uint64_t* u, uint64_t* v, cudaStream_t st);

cudaError_t launch_encrypt_compare(int level, int64_t count, const uint64_t* h, const uint64_t* s, int64_t nkeys,
                                   const int32_t* key_idx, const uint8_t* m, const uint32_t* r1, const uint32_t* r2,
                                   const uint32_t* e, const uint64_t* u_in, const uint64_t* v_in, uint32_t* ok,
                                   cudaStream_t st);
cudaError_t launch_encrypt_valid(int level, int64_t count, const uint64_t* h, const uint64_t* s, int64_t nkeys,
                                 const int32_t* key_idx, const uint8_t* m, const uint32_t* r1, const uint32_t* r2,
                                 const uint32_t* e, uint64_t* u, uint64_t* v, cudaStream_t st);
cudaError_t launch_shake256(int64_t count, const uint8_t* msg, int len, uint8_t* out, int outlen, cudaStream_t st);
cudaError_t launch_kem_seed_keys(int level, int64_t nkeys, const uint8_t* seed_sk, const uint8_t* seed_pk,
                                 uint64_t* h, uint32_t* x, uint32_t* y, cudaStream_t st);
cudaError_t launch_kem_derive(int level, int64_t count, const uint8_t* m, const uint8_t* salt, uint32_t* r1,
                              uint32_t* r2, uint32_t* e, cudaStream_t st);
cudaError_t launch_kem_K(int level, int64_t count, const uint8_t* m, const uint32_t* ok, const uint8_t* sigma,
                         const int32_t* key_idx, int64_t nkeys, const uint64_t* u, const uint64_t* v,
                         const uint8_t* salt, uint8_t* K, cudaStream_t st);

}  // namespace hqc

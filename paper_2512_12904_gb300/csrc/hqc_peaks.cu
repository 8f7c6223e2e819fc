// Microbenchmarks for the on-chip roofline denominators of the decryption
// kernels: shared-memory read bandwidth (conflict-free 32-bit loads, the
// access the rotate-XOR product makes) and 32-bit integer funnel-shift/XOR
// throughput.  Separate library (libhqc_peaks.so); bench.py calls it once
// before timing.
#include <cuda_runtime.h>

#include <cstdint>

namespace {

constexpr int PEAK_THREADS = 1024;
constexpr int SMEM_WORDS = 8192;  // 32 KB

__global__ void __launch_bounds__(PEAK_THREADS) k_smem_read(int iters, uint32_t* out) {
  __shared__ uint32_t buf[SMEM_WORDS];
  for (int i = threadIdx.x; i < SMEM_WORDS; i += blockDim.x) buf[i] = i * 2654435761u;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0;
  // 16 independent conflict-free warp-wide loads per iteration, addresses
  // move every iteration so nothing is hoisted.  base is a multiple of 512
  // in [0, SMEM_WORDS - 512], so base + lane + 15 * 32 < SMEM_WORDS.
  int base = (warp * 512) & (SMEM_WORDS - 512);
  for (int it = 0; it < iters; it++) {
    const uint32_t* p = buf + base + lane;
#pragma unroll
    for (int k = 0; k < 16; k += 4) {
      acc0 ^= p[(k + 0) * 32];
      acc1 ^= p[(k + 1) * 32];
      acc2 ^= p[(k + 2) * 32];
      acc3 ^= p[(k + 3) * 32];
    }
    base = (base + 512) & (SMEM_WORDS - 512);
  }
  const uint32_t r = acc0 ^ acc1 ^ acc2 ^ acc3;
  if (r == 0x12345678u) out[blockIdx.x] = r;  // keeps the loads alive
}

__global__ void __launch_bounds__(PEAK_THREADS) k_int_ops(int iters, uint32_t seed, uint32_t* out) {
  uint32_t a0 = seed ^ threadIdx.x, a1 = a0 * 3u, a2 = a0 * 5u, a3 = a0 * 7u;
  uint32_t b0 = a0 + 1u, b1 = a1 + 1u, b2 = a2 + 1u, b3 = a3 + 1u;
  const uint32_t s = seed & 31u;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int k = 0; k < 8; k++) {
      // 2 ops per chain per step: one funnel shift, one XOR (8 chains)
      a0 ^= __funnelshift_r(b0, a1, s);
      a1 ^= __funnelshift_r(b1, a2, s);
      a2 ^= __funnelshift_r(b2, a3, s);
      a3 ^= __funnelshift_r(b3, a0, s);
      b0 ^= __funnelshift_r(a0, b1, s);
      b1 ^= __funnelshift_r(a1, b2, s);
      b2 ^= __funnelshift_r(a2, b3, s);
      b3 ^= __funnelshift_r(a3, b0, s);
    }
  }
  const uint32_t r = a0 ^ a1 ^ a2 ^ a3 ^ b0 ^ b1 ^ b2 ^ b3;
  if (r == 0x12345678u) out[blockIdx.x] = r;
}

// Integer issue ceiling across two pipes: half of the operations are
// funnel shifts and XORs (integer ALU pipe), half are 32-bit multiply-adds
// with a runtime odd multiplier (IMAD, fused multiply-add pipe).  A kernel
// that moves part of its integer work to multiply-adds (as the decryption
// kernels do for butterflies and table addresses) is bounded by this rate,
// not by the ALU pipe alone.
__global__ void __launch_bounds__(PEAK_THREADS) k_int_mix(int iters, uint32_t seed, uint32_t* out) {
  uint32_t a0 = seed ^ threadIdx.x, a1 = a0 * 3u, b0 = a0 + 1u, b1 = a1 + 1u;
  uint32_t c0 = a0 * 5u, c1 = a0 * 7u, c2 = a0 * 11u, c3 = a0 * 13u;
  const uint32_t s = seed & 31u, M = seed | 1u;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int k = 0; k < 8; k++) {
      // 4 ALU ops (2 funnel shifts, 2 XORs) and 4 multiply-adds per step
      a0 ^= __funnelshift_r(b0, a1, s);
      b1 ^= __funnelshift_r(a1, b0, s);
      c0 = c0 * M + c1;
      c1 = c1 * M + c2;
      c2 = c2 * M + c3;
      c3 = c3 * M + c0;
      a1 ^= __funnelshift_r(b1, a0, s);
      b0 ^= __funnelshift_r(a0, b1, s);
      c0 = c0 * M + c2;
      c1 = c1 * M + c3;
      c2 = c2 * M + c0;
      c3 = c3 * M + c1;
    }
  }
  const uint32_t r = a0 ^ a1 ^ b0 ^ b1 ^ c0 ^ c1 ^ c2 ^ c3;
  if (r == 0x12345678u) out[blockIdx.x] = r;
}

template <class F>
float time_ms(F launch, int reps) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  launch();  // warm-up
  cudaEventRecord(e0);
  for (int i = 0; i < reps; i++) launch();
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms / reps;
}

}  // namespace

extern "C" {

// Shared-memory read bandwidth in bytes/s over all SMs; 0 on error.
double hqc_peak_smem_read_bytes_per_s(void) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint32_t* out = nullptr;
  if (cudaMalloc(&out, 4096 * sizeof(uint32_t)) != cudaSuccess) return 0;
  const int iters = 20000, grid = sms * 2;
  const float ms = time_ms([&] { k_smem_read<<<grid, PEAK_THREADS>>>(iters, out); }, 5);
  cudaFree(out);
  if (cudaGetLastError() != cudaSuccess || ms <= 0) return 0;
  const double bytes = (double)grid * PEAK_THREADS * iters * 16 * 4;
  return bytes / (ms * 1e-3);
}

// 32-bit integer operations per second (funnel shift + XOR mix); 0 on error.
double hqc_peak_int_ops_per_s(void) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint32_t* out = nullptr;
  if (cudaMalloc(&out, 4096 * sizeof(uint32_t)) != cudaSuccess) return 0;
  const int iters = 4000, grid = sms * 2;
  const float ms = time_ms([&] { k_int_ops<<<grid, PEAK_THREADS>>>(iters, 0x9E3779B9u, out); }, 5);
  cudaFree(out);
  if (cudaGetLastError() != cudaSuccess || ms <= 0) return 0;
  const double ops = (double)grid * PEAK_THREADS * iters * 8 * 8 * 2;
  return ops / (ms * 1e-3);
}

// 32-bit integer operations per second when half are ALU-pipe funnel
// shifts/XORs and half multiply-adds on the FMA pipe; 0 on error.
double hqc_peak_int_issue_ops_per_s(void) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint32_t* out = nullptr;
  if (cudaMalloc(&out, 4096 * sizeof(uint32_t)) != cudaSuccess) return 0;
  const int iters = 4000, grid = sms * 2;
  const float ms = time_ms([&] { k_int_mix<<<grid, PEAK_THREADS>>>(iters, 0x9E3779B9u, out); }, 5);
  cudaFree(out);
  if (cudaGetLastError() != cudaSuccess || ms <= 0) return 0;
  const double ops = (double)grid * PEAK_THREADS * iters * 8 * 16;
  return ops / (ms * 1e-3);
}

}  // extern "C"

// Rate microbenchmarks behind the compute-side roofline of the doc-tiled
// main pass (bench.py --microbench builds and runs this file):
//   - red.shared.add.{s32,f32,u64}, 2 CTAs x 512 threads per SM (the tile
//     kernel's shape), lanes to 32 distinct banks and lanes to random cells of
//     a 64 KB block (the sparse tail's pattern);
//   - FP32 FMAs, 16 independent chains per thread (the dense head's bound);
//   - red.global.add.f32 to random cells of eight 4 MB rows (the plain
//     term-parallel scatter's bound, served by the L2).
// Each prints its rate per SM and clock; the clock is the device's maximum.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("err %s line %d\n", cudaGetErrorString(e), __LINE__); return 1; } } while (0)

constexpr int kThreads = 512;
constexpr int kIters = 4096;

__device__ __forceinline__ uint32_t hash32(uint32_t x) { x ^= x >> 16; x *= 0x7feb352dU; x ^= x >> 15; x *= 0x846ca68bU; x ^= x >> 16; return x; }

// MODE 0: s32 lane-distinct banks; 1: s32 random in 16K cells; 2: f32 distinct; 3: f32 random; 4: u64 distinct; 5: u64 random (8K cells)
template <int MODE>
__global__ void __launch_bounds__(kThreads, 2) red_shared(uint32_t* out) {
  extern __shared__ __align__(16) uint8_t sm[];
  uint32_t* a = reinterpret_cast<uint32_t*>(sm);
  for (int i = threadIdx.x; i < 16384; i += blockDim.x) a[i] = 0;
  __syncthreads();
  const uint32_t base = (uint32_t)__cvta_generic_to_shared(a);
  uint32_t h = hash32(threadIdx.x * 7919u + blockIdx.x);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int it = 0; it < kIters; ++it) {
    uint32_t cell;
    if (MODE == 0 || MODE == 2) cell = (uint32_t)((warp * 997 + it * 32) & (16384 - 32)) + lane;
    else if (MODE == 4) cell = (uint32_t)((warp * 997 + it * 32) & (8192 - 32)) + lane;
    else if (MODE == 5) { h = hash32(h + it); cell = h & 8191; }
    else { h = hash32(h + it); cell = h & 16383; }
    if (MODE == 0 || MODE == 1) asm volatile("red.shared.add.s32 [%0], %1;" :: "r"(base + cell * 4), "r"(1) : "memory");
    else if (MODE == 2 || MODE == 3) asm volatile("red.shared.add.f32 [%0], %1;" :: "r"(base + cell * 4), "f"(1.0f) : "memory");
    else asm volatile("red.shared.add.u64 [%0], %1;" :: "r"(base + cell * 8), "l"(1ll) : "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) out[blockIdx.x] = a[5];
}

__global__ void __launch_bounds__(kThreads, 2) ffma_peak(float* out, float a, float b) {
  float x[16];
  for (int i = 0; i < 16; ++i) x[i] = threadIdx.x * 0.001f + i;
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = fmaf(x[i], a, b);
  }
  float s = 0; for (int i = 0; i < 16; ++i) s += x[i];
  if (s == 123.0f) out[0] = s;
}

// L2 reductions: each warp adds into random cells of one 4 MB row per query-like slab
__global__ void red_global(float* rows, int64_t cells, int iters) {
  uint32_t h = hash32(blockIdx.x * 1024 + threadIdx.x);
  const int64_t slab = (int64_t)(blockIdx.x % 8) * (1 << 20);
  for (int it = 0; it < iters; ++it) {
    h = hash32(h + it);
    atomicAdd(rows + slab + (h & ((1 << 20) - 1)), 1.0f);
  }
}

int main() {
  uint32_t* out; CK(cudaMalloc(&out, 1 << 20));
  int sms; CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
  int clk; CK(cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0));
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  const int grid = sms * 2;
  auto run = [&](auto kern, const char* name, int smem, double ops_per_thread) -> int {
    if (smem) CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    for (int w = 0; w < 2; ++w) kern<<<grid, kThreads, smem>>>(out);
    CK(cudaDeviceSynchronize());
    cudaEventRecord(e0);
    for (int r = 0; r < 5; ++r) kern<<<grid, kThreads, smem>>>(out);
    cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    float ms; cudaEventElapsedTime(&ms, e0, e1); ms /= 5;
    const double ops = ops_per_thread * grid * kThreads;
    const double per_s = ops / (ms * 1e-3);
    printf("%-34s %8.3f ms  %10.3f G lanes/s  %6.2f lanes/clk/SM (at %d MHz)\n", name, ms, per_s / 1e9,
           per_s / sms / (clk * 1e3), clk / 1000);
    return 0;
  };
  if (run(red_shared<0>, "red.shared.add.s32 distinct banks", 65536, kIters)) return 1;
  if (run(red_shared<1>, "red.shared.add.s32 random cells", 65536, kIters)) return 1;
  if (run(red_shared<2>, "red.shared.add.f32 distinct banks", 65536, kIters)) return 1;
  if (run(red_shared<3>, "red.shared.add.f32 random cells", 65536, kIters)) return 1;
  if (run(red_shared<4>, "red.shared.add.u64 distinct", 65536, kIters)) return 1;
  if (run(red_shared<5>, "red.shared.add.u64 random cells", 65536, kIters)) return 1;
  {
    float* f = reinterpret_cast<float*>(out);
    for (int w = 0; w < 2; ++w) ffma_peak<<<grid, kThreads>>>(f, 1.0001f, 0.5f);
    CK(cudaDeviceSynchronize());
    cudaEventRecord(e0);
    for (int r = 0; r < 5; ++r) ffma_peak<<<grid, kThreads>>>(f, 1.0001f, 0.5f);
    cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    float ms; cudaEventElapsedTime(&ms, e0, e1); ms /= 5;
    const double flops = 2.0 * 16 * kIters * (double)grid * kThreads;
    printf("%-34s %8.3f ms  %10.3f TFLOP/s  %6.2f FMA lanes/clk/SM\n", "ffma (16 chains per thread)", ms,
           flops / (ms * 1e-3) / 1e12, flops / 2 / (ms * 1e-3) / sms / (clk * 1e3));
  }
  {
    float* rows; CK(cudaMalloc(&rows, sizeof(float) * 8 * (1 << 20)));
    CK(cudaMemset(rows, 0, sizeof(float) * 8 * (1 << 20)));
    const int g = sms * 8, t = 256, iters = 256;
    for (int w = 0; w < 2; ++w) red_global<<<g, t>>>(rows, 8 << 20, iters);
    CK(cudaDeviceSynchronize());
    cudaEventRecord(e0);
    for (int r = 0; r < 5; ++r) red_global<<<g, t>>>(rows, 8 << 20, iters);
    cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    float ms; cudaEventElapsedTime(&ms, e0, e1); ms /= 5;
    const double ops = (double)g * t * iters;
    printf("%-34s %8.3f ms  %10.3f G reductions/s (random cells of 8 rows x 4 MB)\n", "red.global.add.f32 (L2)", ms,
           ops / (ms * 1e-3) / 1e9);
  }
  return 0;
}

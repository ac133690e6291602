// Throughput of shared-memory operations on random slots of a 64 KB table,
// the operations the per-row hash tables of the walk are made of.  Not part
// of the library: `bench.py --mode atomics` compiles and runs it.
//
// Every thread performs `iters` operations on pseudo-random slots (a linear
// congruential sequence per thread, so addresses never depend on results);
// the result is reported as operations per SM clock cycle.
#include <cstdint>
#include <cstdio>

#include <cuda_runtime.h>

enum Op { kCas64, kCas32, kRed32, kAdd32, kAdd64, kLoad64, kLoad32 };

template <int OP>
__global__ void k_ops(int iters, int tlog, unsigned long long *cycles,
                      unsigned long long *sink) {
  extern __shared__ unsigned long long tab64[];
  uint32_t *tab32 = reinterpret_cast<uint32_t *>(tab64);
  const int T = 1 << tlog;
  for (int i = threadIdx.x; i < T; i += blockDim.x) tab64[i] = 0;
  __syncthreads();
  uint32_t x = (threadIdx.x + 1) * 2654435761u ^ (blockIdx.x * 40503u);
  unsigned long long acc = 0;
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
    x = x * 1664525u + 1013904223u;
    const uint32_t h64 = x >> (32 - tlog);  // < T
    const uint32_t h32 = x >> (31 - tlog);  // < 2 T (32-bit view)
    if (OP == kCas64) acc += atomicCAS(&tab64[h64], 0ull, (unsigned long long)x);
    if (OP == kCas32) acc += atomicCAS(&tab32[h32], 0u, x);
    if (OP == kRed32) atomicAdd(&tab32[h32], 1u);
    if (OP == kAdd32) acc += atomicAdd(&tab32[h32], 1u);
    if (OP == kAdd64) acc += atomicAdd(&tab64[h64], 1ull);
    if (OP == kLoad64) acc += *(volatile unsigned long long *)&tab64[h64];
    if (OP == kLoad32) acc += *(volatile uint32_t *)&tab32[h32];
  }
  __syncthreads();
  const long long t1 = clock64();
  if (threadIdx.x == 0) cycles[blockIdx.x] = (unsigned long long)(t1 - t0);
  if (acc == 0x123456789ull) sink[0] = acc;  // keeps the loads
}

template <int OP>
void run(const char *name, int nt, int per_sm, int sms) {
  const int tlog = 13, iters = 2048, grid = sms * per_sm;
  unsigned long long *cyc, *sink;
  cudaMalloc(&cyc, grid * sizeof(unsigned long long));
  cudaMalloc(&sink, sizeof(unsigned long long));
  const size_t smem = (size_t)8 << tlog;
  cudaFuncSetAttribute(k_ops<OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_ops<OP><<<grid, nt, smem>>>(iters, tlog, cyc, sink);  // warm-up
  k_ops<OP><<<grid, nt, smem>>>(iters, tlog, cyc, sink);
  const cudaError_t e = cudaDeviceSynchronize();
  static unsigned long long h[8192];
  cudaMemcpy(h, cyc, grid * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
  double avg = 0;
  for (int i = 0; i < grid; ++i) avg += (double)h[i];
  avg /= grid;
  std::printf("{\"op\": \"%s\", \"threads\": %d, \"ctas_per_sm\": %d, \"ops_per_cycle_per_sm\": %.2f%s}\n",
              name, nt, per_sm, (double)nt * per_sm * iters / avg,
              e == cudaSuccess ? "" : ", \"error\": true");
  cudaFree(cyc);
  cudaFree(sink);
}

int main() {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  run<kCas64>("cas64", 512, 2, sms);
  run<kCas32>("cas32", 512, 2, sms);
  run<kRed32>("add32 (no result)", 512, 2, sms);
  run<kAdd32>("add32", 512, 2, sms);
  run<kAdd64>("add64", 512, 2, sms);
  run<kLoad64>("load64", 512, 2, sms);
  run<kLoad32>("load32", 512, 2, sms);
  return 0;
}

// alu_peak.cu -- test program (tests/test_gpu_alu_peak.py): measures the
// integer-pipe peaks the annealer's roofline uses:
// per-SM throughput of 32-bit multiply-add (mad.lo), 32x32->64 multiply
// (mul.wide), three-input logic (lop3) and whole Philox4x32-10 blocks.
// One CTA of 1024 threads per SM; each CTA counts its own SM cycles with
// clock64, so ops/clk/SM does not depend on the clock the GPU runs at.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
#include <vector>
#include <algorithm>

__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0; k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
  }
  return make_uint4(c0, c1, c2, c3);
}

template <int MODE>
__global__ void __launch_bounds__(1024, 1) bench(uint32_t* out, long long* cyc, int iters, uint32_t seed) {
  uint32_t a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = threadIdx.x * 8 + j + seed;
  __syncthreads();
  long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
    if (MODE == 0) {         // 8 independent mad.lo chains, 8 ops
#pragma unroll
      for (int j = 0; j < 8; ++j) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[j]) : "r"(seed|1u), "r"(j));
    } else if (MODE == 1) {  // 8 mad.wide chains (lo of result fed back, hi xored in)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        uint64_t w; asm volatile("mul.wide.u32 %0, %1, %2;" : "=l"(w) : "r"(a[j]), "r"(0xD2511F53u));
        a[j] = (uint32_t)w ^ (uint32_t)(w >> 32);
      }
    } else if (MODE == 2) {  // lop3 chains
#pragma unroll
      for (int j = 0; j < 8; ++j) asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[j]) : "r"(seed), "r"(j));
    } else {                 // philox calls, 2 independent per iteration
      uint4 u = philox(a[0], it, a[1], 0u, seed, 7u);
      uint4 v = philox(a[2], it, a[3], 0u, seed, 9u);
      a[0] ^= u.x ^ u.y; a[1] ^= u.z ^ u.w; a[2] ^= v.x ^ v.y; a[3] ^= v.z ^ v.w;
    }
  }
  long long t1 = clock64();
  __syncthreads();
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s ^= a[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

template <int MODE>
void run(const char* name, int sms, double ops_per_iter_thread) {
  uint32_t* out; long long* cyc;
  cudaMalloc(&out, sizeof(uint32_t) * sms * 1024);
  cudaMalloc(&cyc, sizeof(long long) * sms);
  int iters = MODE == 3 ? 2000 : 20000;
  bench<MODE><<<sms, 1024>>>(out, cyc, 100, 1);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  cudaEventRecord(e0);
  bench<MODE><<<sms, 1024>>>(out, cyc, iters, 1);
  cudaEventRecord(e1);
  cudaError_t err = cudaDeviceSynchronize();
  if (err != cudaSuccess) { printf("%s: error %s\n", name, cudaGetErrorString(err)); return; }
  float ms; cudaEventElapsedTime(&ms, e0, e1);
  std::vector<long long> c(sms);
  cudaMemcpy(c.data(), cyc, sizeof(long long) * sms, cudaMemcpyDeviceToHost);
  std::sort(c.begin(), c.end());
  double cycles = (double)c[sms / 2];
  double ops_per_sm = ops_per_iter_thread * iters * 1024.0;
  printf("%-10s %8.2f ops/clk/SM  %8.3f Tops/s  (%.3f ms, median %.0f cycles, implied clock %.0f MHz)\n",
         name, ops_per_sm / cycles, ops_per_sm * sms / (ms * 1e-3) / 1e12, ms, cycles, cycles / (ms * 1e3));
  cudaFree(out); cudaFree(cyc);
}

int main() {
  int sms; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  printf("SMs %d\n", sms);
  run<0>("mad.lo", sms, 8);
  run<1>("mul.wide", sms, 8);
  run<2>("lop3", sms, 8);
  run<3>("philox", sms, 2);   // reported as Philox calls
  return 0;
}

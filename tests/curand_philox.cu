// Test helper: the first m outputs of cuRAND's device Philox4_32_10 generator
// after curand_init(seed, subsequence, 0), printed as hex words, so a test can
// compare the library's Philox4x32-10 blocks with the CUDA library's.
#include <cstdio>
#include <cstdlib>
#include <curand_kernel.h>

__global__ void draw(unsigned long long seed, unsigned long long subsequence, int m, uint4* out) {
  curandStatePhilox4_32_10_t st;
  curand_init(seed, subsequence, 0, &st);
  for (int i = 0; i < m; ++i) out[i] = curand4(&st);
}

int main(int argc, char** argv) {
  if (argc != 4) return 2;
  const unsigned long long seed = strtoull(argv[1], nullptr, 0);
  const unsigned long long sub = strtoull(argv[2], nullptr, 0);
  const int m = atoi(argv[3]);
  if (m <= 0 || m > 1024) return 2;
  uint4* d = nullptr;
  if (cudaMalloc(&d, sizeof(uint4) * m) != cudaSuccess) return 1;
  draw<<<1, 1>>>(seed, sub, m, d);
  uint4 h[1024];
  if (cudaMemcpy(h, d, sizeof(uint4) * m, cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
  cudaFree(d);
  for (int i = 0; i < m; ++i) printf("%08x %08x %08x %08x\n", h[i].x, h[i].y, h[i].z, h[i].w);
  return 0;
}

// cut.cu -- exact Max-Cut objective of given configurations (Eq. 1).
//
// cut(s) = sum over the 2n torus edges of w_ij [s_i != s_j], which equals
// 1/2 sum_{i<j} w_ij (1 - s_i s_j) for s in {-1,+1}.  One CTA per
// configuration; each site contributes its right and down edge.  Integer
// sums, so the result does not depend on the reduction order.
#include "internal.h"

namespace ising {
namespace {

__global__ void __launch_bounds__(256) cut_kernel(const uint8_t* __restrict__ eflags,
                                                  const int8_t* __restrict__ spins, int32_t X,
                                                  int32_t Y, int32_t n, int32_t* __restrict__ out) {
  __shared__ int32_t warp_sums[8];
  const int8_t* s = spins + static_cast<size_t>(blockIdx.x) * n;
  int32_t acc = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int y = i / X;
    const int x = i - y * X;
    const bool si = s[i] > 0;
    const int jr = y * X + (x + 1 == X ? 0 : x + 1);
    const int jd = (y + 1 == Y ? 0 : y + 1) * X + x;
    const uint8_t f = eflags[i];
    if (si != (s[jr] > 0)) acc += (f & 1u) ? -1 : 1;
    if (si != (s[jd] > 0)) acc += (f & 2u) ? -1 : 1;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
  if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t t = 0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t += warp_sums[w];
    out[blockIdx.x] = t;
  }
}

}  // namespace

cudaError_t launch_cut(const ising_problem* p, const int8_t* spins, int32_t k, int32_t* out,
                       cudaStream_t stream) {
  if (k <= 0) return cudaSuccess;
  cut_kernel<<<k, 256, 0, stream>>>(p->d_eflags, spins, p->X, p->Y, p->n, out);
  return cudaGetLastError();
}

}  // namespace ising

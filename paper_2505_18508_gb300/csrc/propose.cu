// propose.cu -- proposals from the network's logits, each judged by its exact
// integer energy change (Eq. 2 with J = -w: H = sum w_ij s_i s_j).
//
// Flipping a set B of spins reverses the sign of exactly the terms on B's
// boundary, so dE_B = -2 sum_{i in B, j ~ i, j not in B} w_ij s_i s_j; the
// proposal is taken iff dE_B <= 0.
//
// * Tiles: B = the sites with logit > 0 inside one square tile of side `tile`
//   (the last tile of a row or column may be smaller).  Tiles whose
//   (tx + ty) is even are decided first, then the odd ones; with 1 or an even
//   number of tiles along each side, tiles of one parity share no edge, so all
//   of them are decided at once, one warp per tile.
// * Whole lattice (tile = 0): B = all sites with logit > 0, one CTA per trial.
#include "../../include/ising.h"
#include "internal.h"

namespace ising {
namespace {

__device__ __forceinline__ int wrap(int v, int m) { return v < 0 ? v + m : (v >= m ? v - m : v); }

__global__ void __launch_bounds__(128) propose_tiles_kernel(int8_t* __restrict__ spins,
                                                            const float* __restrict__ logits,
                                                            const uint8_t* __restrict__ eflags, int X, int Y, int tile,
                                                            int ntx, int nty, int phase,
                                                            int32_t* __restrict__ accepted) {
  const int lane = threadIdx.x & 31;
  const int tidx = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (tidx >= ntx * nty) return;
  const int ty = tidx / ntx, tx = tidx - ty * ntx;
  if (((tx + ty) & 1) != phase) return;
  const int b = blockIdx.y;
  const int n = X * Y;
  int8_t* s = spins + static_cast<size_t>(b) * n;
  const float* z = logits + static_cast<size_t>(b) * n;
  const int x0 = tx * tile, y0 = ty * tile;
  const int x1 = min(X, x0 + tile), y1 = min(Y, y0 + tile);
  const int w = x1 - x0, cnt = w * (y1 - y0);
  int dE = 0;
  bool any = false;
  for (int k = lane; k < cnt; k += 32) {
    const int y = y0 + k / w, x = x0 + k % w;
    const int i = y * X + x;
    if (!(z[i] > 0.f)) continue;
    any = true;
    const int si = s[i] > 0 ? 1 : -1;
    const int xl = wrap(x - 1, X), xr = wrap(x + 1, X), yu = wrap(y - 1, Y), yd = wrap(y + 1, Y);
    const int nbr[4] = {y * X + xr, y * X + xl, yd * X + x, yu * X + x};
    const int wgt[4] = {(eflags[i] & 1u) ? -1 : 1, (eflags[y * X + xl] & 1u) ? -1 : 1, (eflags[i] & 2u) ? -1 : 1,
                        (eflags[yu * X + x] & 2u) ? -1 : 1};
    const int nx[4] = {xr, xl, x, x};
    const int ny[4] = {y, y, yd, yu};
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      const int j = nbr[d];
      const bool inside = nx[d] >= x0 && nx[d] < x1 && ny[d] >= y0 && ny[d] < y1 && z[j] > 0.f;
      if (!inside) dE += -2 * wgt[d] * si * (s[j] > 0 ? 1 : -1);
    }
  }
  for (int o = 16; o > 0; o >>= 1) dE += __shfl_xor_sync(0xFFFFFFFFu, dE, o);
  any = __any_sync(0xFFFFFFFFu, any);
  if (!any || dE > 0) return;
  for (int k = lane; k < cnt; k += 32) {
    const int y = y0 + k / w, x = x0 + k % w;
    const int i = y * X + x;
    if (z[i] > 0.f) s[i] = s[i] > 0 ? int8_t(-1) : int8_t(1);
  }
  if (lane == 0 && accepted) atomicAdd(accepted + b, 1);
}

__global__ void __launch_bounds__(1024) propose_global_kernel(int8_t* __restrict__ spins,
                                                              const float* __restrict__ logits,
                                                              const uint8_t* __restrict__ eflags, int X, int Y,
                                                              int32_t* __restrict__ accepted) {
  __shared__ int red[32];
  __shared__ int s_any, s_take;
  const int b = blockIdx.x;
  const int n = X * Y;
  int8_t* s = spins + static_cast<size_t>(b) * n;
  const float* z = logits + static_cast<size_t>(b) * n;
  if (threadIdx.x == 0) s_any = 0;
  __syncthreads();
  int dE = 0;
  bool any = false;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    if (!(z[i] > 0.f)) continue;
    any = true;
    const int y = i / X, x = i - y * X;
    const int si = s[i] > 0 ? 1 : -1;
    const int xl = wrap(x - 1, X), xr = wrap(x + 1, X), yu = wrap(y - 1, Y), yd = wrap(y + 1, Y);
    const int nbr[4] = {y * X + xr, y * X + xl, yd * X + x, yu * X + x};
    const int wgt[4] = {(eflags[i] & 1u) ? -1 : 1, (eflags[y * X + xl] & 1u) ? -1 : 1, (eflags[i] & 2u) ? -1 : 1,
                        (eflags[yu * X + x] & 2u) ? -1 : 1};
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      const int j = nbr[d];
      if (!(z[j] > 0.f)) dE += -2 * wgt[d] * si * (s[j] > 0 ? 1 : -1);
    }
  }
  for (int o = 16; o > 0; o >>= 1) dE += __shfl_xor_sync(0xFFFFFFFFu, dE, o);
  if (__any_sync(0xFFFFFFFFu, any) && (threadIdx.x & 31) == 0) s_any = 1;
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dE;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t += red[w];
    s_take = s_any && t <= 0;
    if (accepted) accepted[b] = s_take;
  }
  __syncthreads();
  if (!s_take) return;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    if (z[i] > 0.f) s[i] = s[i] > 0 ? int8_t(-1) : int8_t(1);
}

// y = [s != r'] with r' = r or -r, whichever is closer to s (a tie keeps site 0)
__global__ void __launch_bounds__(1024) flip_targets_kernel(const int8_t* __restrict__ spins,
                                                            const int8_t* __restrict__ ref, int n,
                                                            uint8_t* __restrict__ targets) {
  __shared__ int red[32];
  __shared__ int s_flip;
  const int b = blockIdx.x;
  const int8_t* s = spins + static_cast<size_t>(b) * n;
  const int8_t* r = ref + static_cast<size_t>(b) * n;
  int d = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) d += (s[i] > 0) != (r[i] > 0);
  for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xFFFFFFFFu, d, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t += red[w];
    s_flip = (2 * t > n) || (2 * t == n && ((s[0] > 0) != (r[0] > 0)));
  }
  __syncthreads();
  const int f = s_flip;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    targets[static_cast<size_t>(b) * n + i] = static_cast<uint8_t>(((s[i] > 0) != (r[i] > 0)) ^ f);
}

}  // namespace
}  // namespace ising

extern "C" int ising_flip_targets(const int8_t* spins, const int8_t* ref, int32_t B, int32_t n, uint8_t* targets,
                                  void* cuda_stream) {
  if (B < 0 || n <= 0 || (B > 0 && (!spins || !ref || !targets))) return ISING_ERR_ARG;
  if (B == 0) return ISING_OK;
  ising::flip_targets_kernel<<<B, 1024, 0, static_cast<cudaStream_t>(cuda_stream)>>>(spins, ref, n, targets);
  return cudaGetLastError() == cudaSuccess ? ISING_OK : ISING_ERR_CUDA;
}

extern "C" int ising_propose(const ising_problem* p, int8_t* spins, int32_t B, const float* logits, int32_t tile,
                             int32_t* accepted, void* cuda_stream) {
  if (!p || B < 0 || tile < 0 || (B > 0 && (!spins || !logits))) return ISING_ERR_ARG;
  if (p->graph) return ISING_ERR_UNSUPPORTED;   // tiles and boundaries of the torus
  if (B == 0) return ISING_OK;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (tile == 0) {
    ising::propose_global_kernel<<<B, 1024, 0, st>>>(spins, logits, p->d_eflags, p->X, p->Y, accepted);
    return cudaGetLastError() == cudaSuccess ? ISING_OK : ISING_ERR_CUDA;
  }
  const int ntx = (p->X + tile - 1) / tile, nty = (p->Y + tile - 1) / tile;
  if ((ntx != 1 && (ntx & 1)) || (nty != 1 && (nty & 1))) return ISING_ERR_ARG;
  if (B > 65535) return ISING_ERR_UNSUPPORTED;
  if (accepted && cudaMemsetAsync(accepted, 0, sizeof(int32_t) * B, st) != cudaSuccess) return ISING_ERR_CUDA;
  const dim3 grid((ntx * nty + 3) / 4, B);
  for (int phase = 0; phase < 2; ++phase)
    ising::propose_tiles_kernel<<<grid, 128, 0, st>>>(spins, logits, p->d_eflags, p->X, p->Y, tile, ntx, nty, phase,
                                                      accepted);
  return cudaGetLastError() == cudaSuccess ? ISING_OK : ISING_ERR_CUDA;
}

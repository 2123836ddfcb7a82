// anneal.cu -- checkerboard Metropolis sweeps with multi-spin coding.
//
// One CTA holds one row strip of one trial group in shared memory; the C
// strips of a group form a thread-block cluster and exchange boundary rows
// through distributed shared memory after every half-sweep.
//
// Method (Zick 2025, Section III: independent trials of sweeps, read out at
// the end of each trial; Eq. 1 and Eq. 2 with J = -w, h = 0).  The sweep is a
// Metropolis sweep over the two checkerboard colours.  The torus has even
// sides, so it is bipartite: all sites of one colour are updated at once, which
// equals visiting them one by one.
//
// Layout (per trial group of G <= 32 trials, bit b of a word = trial t0 + b):
//   spin word  sp[c][lr][h]   colour plane c, local row lr (0 and rows+1 are
//                              halo rows), h = x / 2; the site of colour c in
//                              global row y sits at x = 2h + ((y + c) & 1).
//   bit = 1 <=> spin +1.
// With e_j = NOT(s_i XOR s_j XOR neg_ij) marking a +1 energy term w_ij s_i s_j,
// the count m = e_L + e_R + e_U + e_D gives dE = 8 - 4m.  m >= 2: flip;
// m = 1: flip iff u < T4; m = 0: flip iff u < T8.  The counts are bit-sliced
// over the 32 trials of a word; the draws u come from Philox4x32-10 at
// counter (i, k, t / 4, 0), word t mod 4.
//
// Half-sweep c writes only colour-c words and reads only colour-(1-c) words,
// so the boundary-row push into a neighbour's halo (colour c) never races
// with that neighbour's reads (colour 1-c) in the same half-sweep; one
// cluster barrier per half-sweep orders everything.
#include "device_common.cuh"
#include "internal.h"

namespace ising {
namespace {

__device__ __forceinline__ int strip_rows(int Y, int C, int r) { return Y / C + (r < Y % C ? 1 : 0); }
__device__ __forceinline__ int strip_y0(int Y, int C, int r) { return r * (Y / C) + min(r, Y % C); }

template <bool kCluster>
__device__ __forceinline__ void block_or_cluster_sync() {
  if constexpr (kCluster) cluster_barrier();
  else __syncthreads();
}

template <bool kCluster>
__global__ void __launch_bounds__(1024, 1) anneal_strip_kernel(const AnnealArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int C = a.C;
  const int r = kCluster ? static_cast<int>(cluster_ctarank()) : 0;
  const int g = blockIdx.y;
  const int rows = strip_rows(a.Y, C, r);
  const int y0 = strip_y0(a.Y, C, r);
  const int H = a.H;
  const int L = a.Rmax + 2;
  uint32_t* sp = reinterpret_cast<uint32_t*>(smem);
  unsigned char* fl = smem + static_cast<size_t>(2) * L * H * 4;
  int32_t* part = reinterpret_cast<int32_t*>(fl + ((static_cast<size_t>(2) * a.Rmax * H + 15) & ~size_t(15)));

  const int t0 = g * a.G;
  const int live = min(a.G, a.T - t0);
  const int nq = (live + 3) >> 2;
  const uint32_t q0 = static_cast<uint32_t>(t0) >> 2;
  const int tid = threadIdx.x, nt = blockDim.x;

  if (tid < 32) part[tid] = 0;

  // weights of the own rows
  for (int idx = tid; idx < 2 * rows * H; idx += nt) {
    const int c = idx / (rows * H);
    const int rem = idx - c * rows * H;
    const int lr0 = rem / H;
    const int h = rem - lr0 * H;
    fl[(c * a.Rmax + lr0) * H + h] = a.flags[(static_cast<size_t>(c) * a.Y + y0 + lr0) * H + h];
  }
  // starting spins of the own rows and of both halo rows (counter-based, so a
  // halo row is initialised here to the same value its owner computes)
  for (int idx = tid; idx < 2 * (rows + 2) * H; idx += nt) {
    const int c = idx / ((rows + 2) * H);
    const int rem = idx - c * (rows + 2) * H;
    const int lr = rem / H;
    const int h = rem - lr * H;
    int y = y0 - 1 + lr;
    if (y < 0) y += a.Y;
    if (y >= a.Y) y -= a.Y;
    const uint32_t i = static_cast<uint32_t>(y * a.X + 2 * h + ((y + c) & 1));
    uint32_t w = 0;
    if (a.init) {
      for (int b = 0; b < live; ++b)
        w |= static_cast<uint32_t>(a.init[static_cast<size_t>(t0 + b) * a.n + i] > 0) << b;
    } else {
      for (int j = 0; j < nq; ++j) {
        const uint4 u = philox4x32_10(i, 0xFFFFFFFFu, q0 + j, 0u, a.key0, a.key1);
        w |= ((u.x >> 31) | ((u.y >> 31) << 1) | ((u.z >> 31) << 2) | ((u.w >> 31) << 3)) << (4 * j);
      }
    }
    sp[(c * L + lr) * H + h] = w;
  }
  block_or_cluster_sync<kCluster>();

  const int r_up = (r + C - 1) % C, r_dn = (r + 1) % C;
  const int rows_up = strip_rows(a.Y, C, r_up);
  const int items = rows * H;
  const int dq = nt / H, dr = nt - (nt / H) * H;
  const int lr_start = 1 + tid / H, h_start = tid - (tid / H) * H;

  for (int kk = 0; kk < a.S; ++kk) {
    const uint32_t k = a.k0 + static_cast<uint32_t>(kk);
    const uint32_t T4 = __ldg(a.thr + 2 * kk);
    const uint32_t T8 = __ldg(a.thr + 2 * kk + 1);
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
      uint32_t* self = sp + static_cast<size_t>(c) * L * H;
      const uint32_t* nb = sp + static_cast<size_t>(1 - c) * L * H;
      const unsigned char* fc = fl + static_cast<size_t>(c) * a.Rmax * H;
      int lr = lr_start, h = h_start;
      for (int it = tid; it < items; it += nt) {
        const int y = y0 + lr - 1;
        const int par = (y + c) & 1;
        const uint32_t i = static_cast<uint32_t>(y * a.X + 2 * h + par);
        const int row = lr * H;
        const uint32_t s = self[row + h];
        const uint32_t nu = nb[row - H + h];
        const uint32_t nd = nb[row + H + h];
        const int hl = par ? h : (h == 0 ? H - 1 : h - 1);
        const int hr = par ? (h == H - 1 ? 0 : h + 1) : h;
        const uint32_t nl = nb[row + hl];
        const uint32_t nr = nb[row + hr];
        const uint32_t f = fc[(lr - 1) * H + h];
        const uint32_t mL = 0u - (f & 1u), mR = 0u - ((f >> 1) & 1u);
        const uint32_t mU = 0u - ((f >> 2) & 1u), mD = 0u - ((f >> 3) & 1u);
        const uint32_t eL = ~(s ^ nl ^ mL), eR = ~(s ^ nr ^ mR);
        const uint32_t eU = ~(s ^ nu ^ mU), eD = ~(s ^ nd ^ mD);
        const uint32_t any = eL | eR | eU | eD;
        const uint32_t eq1 = ((eL ^ eR) ^ (eU ^ eD)) & ~((eL & eR) | (eU & eD));
        const uint32_t eq0 = ~any;
        const uint32_t ge2 = any & ~eq1;
        uint32_t acc4 = 0, acc8 = 0;
        for (int j = nq - 1; j >= 0; --j) {
          const uint4 u = philox4x32_10(i, k, q0 + j, 0u, a.key0, a.key1);
          acc4 = (acc4 << 4) | static_cast<uint32_t>(u.x < T4) | (static_cast<uint32_t>(u.y < T4) << 1) |
                 (static_cast<uint32_t>(u.z < T4) << 2) | (static_cast<uint32_t>(u.w < T4) << 3);
          acc8 = (acc8 << 4) | static_cast<uint32_t>(u.x < T8) | (static_cast<uint32_t>(u.y < T8) << 1) |
                 (static_cast<uint32_t>(u.z < T8) << 2) | (static_cast<uint32_t>(u.w < T8) << 3);
        }
        const uint32_t ns = s ^ (ge2 | (eq1 & acc4) | (eq0 & acc8));
        self[row + h] = ns;
        if (lr == 1) {          // first own row -> bottom halo of the strip above
          if constexpr (kCluster) st_cluster_u32(smem_addr(self + (rows_up + 1) * H + h), r_up, ns);
          else self[(rows + 1) * H + h] = ns;
        }
        if (lr == rows) {       // last own row -> top halo of the strip below
          if constexpr (kCluster) st_cluster_u32(smem_addr(self + h), r_dn, ns);
          else self[h] = ns;
        }
        h += dr;
        lr += dq;
        if (h >= H) { h -= H; ++lr; }
      }
      block_or_cluster_sync<kCluster>();
    }
  }

  // ---- read-out: spins of the own rows
  if (a.out_spins) {
    const int span = rows * a.X;
    const size_t gbase = static_cast<size_t>(y0) * a.X;
    for (int idx = tid; idx < live * span; idx += nt) {
      const int b = idx / span;
      const int rem = idx - b * span;
      const int yl = rem / a.X;
      const int x = rem - yl * a.X;
      const int c = (x + y0 + yl) & 1;
      const uint32_t w = sp[(c * L + yl + 1) * H + (x >> 1)];
      a.out_spins[static_cast<size_t>(t0 + b) * a.n + gbase + rem] = ((w >> b) & 1u) ? int8_t(1) : int8_t(-1);
    }
  }
  // ---- exact cut: sum over own right/down edges of w [s_i != s_j], counted
  // per trial as sum(v) - #neg with v = d for w = +1 and NOT d for w = -1
  if (a.out_cuts) {
    const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
    uint32_t acc = 0;
    const int total = 2 * rows * H;
    for (int base = warp * 32; base < total; base += nwarps * 32) {
      const int idx = base + lane;
      uint32_t vr = 0, vd = 0;
      if (idx < total) {
        const int c = idx / (rows * H);
        const int rem = idx - c * rows * H;
        const int lr = 1 + rem / H;
        const int h = rem - (lr - 1) * H;
        const int par = (y0 + lr - 1 + c) & 1;
        const uint32_t s = sp[(c * L + lr) * H + h];
        const uint32_t* nb = sp + static_cast<size_t>(1 - c) * L * H;
        const int hr = par ? (h == H - 1 ? 0 : h + 1) : h;
        const uint32_t sr = nb[lr * H + hr];
        const uint32_t sd = nb[(lr + 1) * H + h];
        const uint32_t f = fl[(c * a.Rmax + lr - 1) * H + h];
        vr = (s ^ sr) ^ (0u - ((f >> 1) & 1u));
        vd = (s ^ sd) ^ (0u - ((f >> 3) & 1u));
      }
#pragma unroll 4
      for (int b = 0; b < 32; ++b) {
        const uint32_t cnt = __popc(__ballot_sync(0xFFFFFFFFu, (vr >> b) & 1u)) +
                             __popc(__ballot_sync(0xFFFFFFFFu, (vd >> b) & 1u));
        if (lane == b) acc += cnt;
      }
    }
    if constexpr (kCluster) red_add_cluster_u32(smem_addr(part + lane), 0u, acc);
    else atomicAdd(reinterpret_cast<unsigned int*>(part + lane), acc);
  }
  block_or_cluster_sync<kCluster>();
  if (a.out_cuts && r == 0 && tid < live) a.out_cuts[t0 + tid] = part[tid] - a.neg_edges;
}

}  // namespace

size_t anneal_smem_bytes(int32_t H, int32_t Rmax) {
  const size_t L = static_cast<size_t>(Rmax) + 2;
  size_t b = 2 * L * H * 4;
  b += (2 * static_cast<size_t>(Rmax) * H + 15) & ~size_t(15);
  b += 32 * 4;
  return b;
}

cudaError_t launch_anneal(const AnnealArgs& a, int threads, cudaStream_t stream) {
  const size_t smem = anneal_smem_bytes(a.H, a.Rmax);
  const int groups = (a.T + a.G - 1) / a.G;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.C, groups, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  cudaError_t e;
  if (a.C > 1) {
    e = cudaFuncSetAttribute(anneal_strip_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    if (a.C > 8) {
      e = cudaFuncSetAttribute(anneal_strip_kernel<true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = a.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, anneal_strip_kernel<true>, a);
  }
  e = cudaFuncSetAttribute(anneal_strip_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  return cudaLaunchKernelEx(&cfg, anneal_strip_kernel<false>, a);
}

}  // namespace ising

// anneal.cu -- the strip kernel of ising_anneal: one CTA per (row strip,
// trial group); the C strips of a group form a thread-block cluster and trade
// boundary rows through distributed shared memory (see anneal_core.cuh).
#include "anneal_core.cuh"

namespace ising {
namespace {

template <bool kCluster, bool kU16>
__global__ void __launch_bounds__(1024, 1) anneal_strip_kernel(const __grid_constant__ AnnealArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  GroupJob job;
  job.flags = a.flags;
  job.thr = a.thr + static_cast<size_t>(blockIdx.y) * a.thr_group_stride;
  job.init = a.init;
  job.out_spins = a.out_spins;
  job.out_cuts = a.out_cuts;
  job.X = a.X; job.Y = a.Y; job.H = a.H; job.n = a.n;
  job.T = a.T; job.G = a.G; job.S = a.S;
  job.k0 = a.k0;
  job.key0 = a.key0; job.key1 = a.key1;
  job.rk = a.rk;
  job.C = a.C; job.Rmax = a.Rmax;
  job.neg_edges = a.neg_edges;
  const int r = kCluster ? static_cast<int>(cluster_ctarank()) : 0;
  anneal_group<kCluster, kU16>(job, blockIdx.y, r, smem);
}

}  // namespace

size_t anneal_smem_bytes(int32_t H, int32_t Rmax) { return core_smem_bytes(H, Rmax); }

template <bool kU16>
cudaError_t launch_strip(const AnnealArgs& a, int threads, cudaStream_t stream) {
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
    e = cudaFuncSetAttribute(anneal_strip_kernel<true, kU16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    if (a.C > 8) {
      e = cudaFuncSetAttribute(anneal_strip_kernel<true, kU16>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = a.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, anneal_strip_kernel<true, kU16>, a);
  }
  e = cudaFuncSetAttribute(anneal_strip_kernel<false, kU16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  return cudaLaunchKernelEx(&cfg, anneal_strip_kernel<false, kU16>, a);
}

cudaError_t launch_anneal(const AnnealArgs& a, int threads, cudaStream_t stream) {
  return a.u16 ? launch_strip<true>(a, threads, stream) : launch_strip<false>(a, threads, stream);
}

}  // namespace ising

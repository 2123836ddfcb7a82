// batched.cu -- one persistent launch over many instances of uneven size,
// trial count and sweep count (the campaigns of Section III run as a batch).
//
// The grid holds a fixed number of CTAs per SM.  Each CTA takes the next work
// unit (instance, trial group) from an atomic counter over a list sorted
// longest-first on the host, anneals it whole in shared memory (the strip
// body of anneal_core.cuh with a single strip), writes its spins and cuts,
// and takes the next unit.  Results equal ising_anneal on each instance,
// including a resumed run (starting spins and the global index of the first
// sweep).
#include "anneal_core.cuh"

namespace ising {
namespace {

__global__ void __launch_bounds__(1024, 1) batched_kernel(const BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_unit;
  __shared__ uint32_t s_rk[20];
  for (;;) {
    if (threadIdx.x == 0) s_unit = static_cast<int>(atomicAdd(a.counter, 1u));
    __syncthreads();
    const int u = s_unit;
    __syncthreads();
    if (u >= a.n_units) break;
    const BatchUnit un = a.units[u];
    const BatchInst in = a.inst[un.inst];
    if (threadIdx.x < 20) {
      const uint32_t r = threadIdx.x >> 1;
      s_rk[threadIdx.x] = (threadIdx.x & 1) ? in.key1 + r * kPhiloxW1 : in.key0 + r * kPhiloxW0;
    }
    __syncthreads();
    GroupJob job;
    job.flags = in.flags;
    job.thr = in.thr;
    job.init = in.init;
    job.out_spins = in.out_spins;
    job.out_cuts = in.out_cuts;
    job.X = in.X; job.Y = in.Y; job.H = in.H; job.n = in.n;
    job.T = in.T; job.G = in.G; job.S = in.S;
    job.k0 = in.k0;
    job.key0 = in.key0; job.key1 = in.key1;
    job.rk = s_rk;
    job.C = 1; job.Rmax = in.Y;
    job.neg_edges = in.neg_edges;
    if (in.u16) anneal_group<false, true>(job, un.group, 0, smem);
    else anneal_group<false, false>(job, un.group, 0, smem);
  }
}

}  // namespace

size_t batched_smem_bytes(int32_t H, int32_t Y) { return core_smem_bytes(H, Y); }

size_t batched_static_smem() { return static_smem_of(reinterpret_cast<const void*>(batched_kernel)); }

cudaError_t batched_prepare(size_t smem) {
  return cudaFuncSetAttribute(batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
}

cudaError_t launch_batched(const BatchArgs& a, int grid, int threads, size_t smem, cudaStream_t stream) {
  if (a.n_units <= 0 || grid <= 0) return cudaSuccess;
  batched_kernel<<<grid, threads, smem, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace ising

// pt.cu -- replica exchange (parallel tempering) on the torus: R temperatures
// x C chains, rounds of L sweeps at constant temperature followed by swaps
// between neighbouring temperatures.  The paper's update rule is unpublished
// (Section III); this is a variant of the library built on its Metropolis
// sweep.
//
// Slot t = r C + c holds chain c's replica at temperature r and keeps the
// random stream of trial index t.  C is a multiple of 32, so every 32-trial
// group sits at one temperature: the strip kernel anneals all slots at once
// with one threshold table per group.  After round q the pairs (r, r+1), r =
// q mod 2, q mod 2 + 2, ..., exchange chain c's configurations iff
// d = E_r - E_{r+1} <= 0 or u < T_r(d), where E = W - 2 cut (Eq. 1, 2), u is
// word 0 of Philox4x32-10 at counter (c, q, r, 0xFFFFFFFD) and
// T_r(d) = min(floor(exp(-(beta_{r+1} - beta_r) d) 2^32), 2^32 - 1), taken
// from a table the host builds with libm exp (indexed by d / 2, since d is
// even).
#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/ising.h"
#include "device_common.cuh"
#include "internal.h"

namespace {

// one CTA per (chain, pair): thread 0 decides, every thread swaps the rows
__global__ void pt_swap_kernel(int8_t* __restrict__ spins, int32_t* __restrict__ cuts,
                               const uint32_t* __restrict__ swap_thr, int32_t half_range, int32_t C, int32_t n,
                               int32_t parity, uint32_t round, uint32_t key0, uint32_t key1,
                               int32_t* __restrict__ swaps) {
  __shared__ int take;
  const int c = blockIdx.x;
  const int r = parity + 2 * static_cast<int>(blockIdx.y);
  const int a = r * C + c, b = (r + 1) * C + c;
  if (threadIdx.x == 0) {
    // d = E_a - E_b = 2 (cut_b - cut_a)
    const int32_t h = cuts[b] - cuts[a];
    bool t = h <= 0;
    if (!t) {
      const uint4 u = ising::philox4x32_10(static_cast<uint32_t>(c), round, static_cast<uint32_t>(r), 0xFFFFFFFDu,
                                           key0, key1);
      const uint32_t T = h <= half_range ? swap_thr[static_cast<size_t>(r) * half_range + (h - 1)] : 0u;
      t = u.x < T;
    }
    take = t;
    if (t) {
      const int32_t ca = cuts[a];
      cuts[a] = cuts[b];
      cuts[b] = ca;
      if (swaps) atomicAdd(swaps, 1);
    }
  }
  __syncthreads();
  if (!take) return;
  uint32_t* ra = reinterpret_cast<uint32_t*>(spins + static_cast<size_t>(a) * n);
  uint32_t* rb = reinterpret_cast<uint32_t*>(spins + static_cast<size_t>(b) * n);
  for (int i = threadIdx.x; i < n / 4; i += blockDim.x) {
    const uint32_t x = ra[i];
    ra[i] = rb[i];
    rb[i] = x;
  }
}

int map_err(cudaError_t e) {
  if (e == cudaSuccess) return ISING_OK;
  if (e == cudaErrorMemoryAllocation) return ISING_ERR_OOM;
  return ISING_ERR_CUDA;
}

}  // namespace

extern "C" int ising_anneal_pt(ising_problem* p, int32_t temps, const double* betas, int32_t chains, int32_t rounds,
                               int32_t sweeps_per_round, uint64_t seed, int8_t* out_spins, int32_t* out_cuts,
                               int32_t* out_swaps, void* cuda_stream) {
  if (!p || temps < 1 || !betas || chains < 32 || chains % 32 || rounds < 0 || sweeps_per_round < 0 ||
      !out_spins || !out_cuts)
    return ISING_ERR_ARG;
  if (p->graph || p->draw_bits != 32) return ISING_ERR_UNSUPPORTED;
  if (const int crc = ising::refuse_capture(static_cast<cudaStream_t>(cuda_stream))) return crc;
  for (int32_t r = 0; r < temps; ++r)
    if (!(betas[r] > 0.0) || !std::isfinite(betas[r])) return ISING_ERR_ARG;
  if (static_cast<int64_t>(temps) * chains > (int64_t(1) << 30)) return ISING_ERR_UNSUPPORTED;
  const int32_t T = temps * chains, L = sweeps_per_round, n = p->n;
  const int32_t groups = T / 32, half_range = 2 * n;   // |cut_b - cut_a| <= |E| <= 2n edges
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

  // host tables: per-group Metropolis thresholds (L sweeps at the group's beta)
  // and per-pair swap thresholds T_r(2h), h = 1 .. 2n
  std::vector<uint32_t> thr, sthr;
  try {
    thr.resize(static_cast<size_t>(groups) * 2 * (L > 0 ? L : 1));
    for (int32_t g = 0; g < groups; ++g) {
      const double beta = betas[g * 32 / chains];
      for (int32_t k = 0; k < (L > 0 ? L : 1); ++k) {
        thr[(static_cast<size_t>(g) * (L > 0 ? L : 1) + k) * 2 + 0] = ising::accept_threshold(beta * 4.0, 32);
        thr[(static_cast<size_t>(g) * (L > 0 ? L : 1) + k) * 2 + 1] = ising::accept_threshold(beta * 8.0, 32);
      }
    }
    sthr.resize(static_cast<size_t>(temps > 1 ? temps - 1 : 1) * half_range);
    for (int32_t r = 0; r + 1 < temps; ++r) {
      const double db = betas[r + 1] - betas[r];
      for (int32_t h = 1; h <= half_range; ++h)
        sthr[static_cast<size_t>(r) * half_range + (h - 1)] = ising::accept_threshold(db * (2.0 * h), 32);
    }
  } catch (const std::bad_alloc&) {
    return ISING_ERR_OOM;
  }

  // launch shape of the strip kernel with 32-trial groups
  ising::StripShape sh;
  const int src = ising::strip_shape(p, T, 32, &sh);
  if (src != ISING_OK) return src;
  const int Cs = sh.C, Rmax = sh.Rmax, threads = sh.threads;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess || sms <= 0) sms = 152;

  // device scratch: thresholds, swap tables, the other spin buffer
  const size_t b_thr = ((thr.size() * 4 + 255) / 256) * 256, b_sthr = ((sthr.size() * 4 + 255) / 256) * 256;
  const size_t b_spin = ((static_cast<size_t>(T) * n + 255) / 256) * 256;
  unsigned char* d = nullptr;
  cudaError_t e = ising::dev_malloc_async(reinterpret_cast<void**>(&d), b_thr + b_sthr + b_spin, st);
  if (e != cudaSuccess) return map_err(e);
  uint32_t* d_thr = reinterpret_cast<uint32_t*>(d);
  uint32_t* d_sthr = reinterpret_cast<uint32_t*>(d + b_thr);
  int8_t* other = reinterpret_cast<int8_t*>(d + b_thr + b_sthr);
  e = cudaMemcpyAsync(d_thr, thr.data(), thr.size() * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_sthr, sthr.data(), sthr.size() * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && out_swaps) e = cudaMemsetAsync(out_swaps, 0, sizeof(int32_t), st);

  // the persistent flow kernel (per-group threshold tables) when it takes
  // the problem, as ising_anneal would choose it; else the strip kernel
  FlowRun* fr = nullptr;
  if (e == cudaSuccess && p->cfg_kernel != 1 && p->cfg_strips == 0 && (p->cfg_group == 0 || p->cfg_group == 32) &&
      n >= 2048 && static_cast<long long>(groups) * p->Y >= 4LL * sms) {
    const int rc = ising::flow_run_create(p, T, 0, &fr, st);
    if (rc != ISING_OK && rc != ISING_ERR_UNSUPPORTED) {
      cudaFreeAsync(d, st);
      return rc;
    }
  }
  const int32_t stride = 2 * (L > 0 ? L : 1);

  ising::AnnealArgs a{};
  a.flags = p->d_flags;
  a.thr = d_thr;
  a.thr_group_stride = 2 * (L > 0 ? L : 1);
  a.X = p->X; a.Y = p->Y; a.H = p->H; a.n = n;
  a.T = T;
  a.G = 32;
  a.key0 = static_cast<uint32_t>(seed & 0xFFFFFFFFull);
  a.key1 = static_cast<uint32_t>(seed >> 32);
  for (uint32_t r = 0; r < 10; ++r) {
    a.rk[2 * r] = a.key0 + r * 0x9E3779B9u;
    a.rk[2 * r + 1] = a.key1 + r * 0xBB67AE85u;
  }
  a.C = Cs;
  a.Rmax = Rmax;
  a.neg_edges = p->neg_edges;
  a.out_cuts = out_cuts;
  // the start (no sweeps) into the buffer that makes the last round write
  // out_spins: every round moves the state to the other buffer
  const int8_t* cur = nullptr;
  if (e == cudaSuccess) {
    a.init = nullptr;
    a.out_spins = (rounds % 2 == 0) ? out_spins : other;
    a.S = 0;
    a.k0 = 0;
    if (fr) {
      const int rc = ising::flow_run_launch(fr, d_thr, stride, 0, 0, seed, nullptr, a.out_spins, out_cuts, st);
      e = rc == ISING_OK ? cudaSuccess : cudaErrorUnknown;
    } else {
      e = ising::launch_anneal(a, threads, st);
    }
    cur = a.out_spins;
  }
  for (int32_t q = 0; q < rounds && e == cudaSuccess; ++q) {
    int8_t* nxt = (cur == out_spins) ? other : out_spins;
    a.init = cur;
    a.out_spins = nxt;
    a.S = L;
    a.k0 = static_cast<uint32_t>(q) * static_cast<uint32_t>(L);
    if (fr) {
      const int rc = ising::flow_run_launch(fr, d_thr, stride, L, a.k0, seed, cur, nxt, out_cuts, st);
      e = rc == ISING_OK ? cudaSuccess : cudaErrorUnknown;
    } else {
      e = ising::launch_anneal(a, threads, st);
    }
    const int par = q & 1;
    const int npairs = temps - 1 > par ? (temps - 1 - par + 1) / 2 : 0;
    if (e == cudaSuccess && npairs > 0) {
      pt_swap_kernel<<<dim3(chains, npairs), 256, 0, st>>>(nxt, out_cuts, d_sthr, half_range, chains, n, par,
                                                            static_cast<uint32_t>(q), a.key0, a.key1, out_swaps);
      e = cudaGetLastError();
    }
    cur = nxt;
  }
  if (!fr && e == cudaSuccess) p->last_kernel = 1;
  ising::flow_run_destroy(fr, st);
  const cudaError_t e2 = cudaFreeAsync(d, st);
  if (e == cudaSuccess) e = e2;
  return map_err(e);
}

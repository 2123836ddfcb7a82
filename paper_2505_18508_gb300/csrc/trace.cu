// trace.cu -- read-out along the trajectory: the cut of every trial after
// every `trace_every` sweeps (and after the last), and the best of those cuts
// per trial with the first configuration that reached it.
//
// The paper reads each trial out at its end (Section III); its Fig. 1 plots
// cut against sweeps.  This entry point runs the anneal in chunks of
// trace_every sweeps through ising_anneal (resuming from the previous chunk's
// spins at the right global sweep, so the trajectory is the one a single call
// would take), lets each chunk's fused cut land in its trace row, and folds
// the row into the running best with one small kernel per chunk.
#include <cstdint>

#include "../../include/ising.h"
#include "internal.h"

namespace {

// One CTA per trial: keep the chunk's cut when it beats the best so far (or
// when it is the first point) and copy that trial's spins with it.
__global__ void best_update_kernel(const int32_t* __restrict__ cuts, const int8_t* __restrict__ spins,
                                   int32_t* __restrict__ best, int8_t* __restrict__ best_spins, int32_t n,
                                   int32_t first) {
  __shared__ int take;
  const int t = blockIdx.x;
  if (threadIdx.x == 0) {
    const int32_t c = cuts[t];
    take = first || c > best[t];
    if (take) best[t] = c;
  }
  __syncthreads();
  if (!take || !best_spins) return;
  // n is a multiple of 4 (both sides even), so rows are whole 32-bit words
  const uint32_t* src = reinterpret_cast<const uint32_t*>(spins + static_cast<size_t>(t) * n);
  uint32_t* dst = reinterpret_cast<uint32_t*>(best_spins + static_cast<size_t>(t) * n);
  for (int i = threadIdx.x; i < n / 4; i += blockDim.x) dst[i] = src[i];
}

int map_err(cudaError_t e) {
  if (e == cudaSuccess) return ISING_OK;
  if (e == cudaErrorMemoryAllocation) return ISING_ERR_OOM;
  return ISING_ERR_CUDA;
}

}  // namespace

extern "C" int ising_anneal_trace(ising_problem* p, int32_t trials, const double* betas, int32_t S, uint64_t seed,
                                  uint32_t sweep_offset, const int8_t* init_spins, int8_t* out_spins,
                                  int32_t* out_cuts, int32_t trace_every, int32_t* out_trace, int32_t* out_best,
                                  int8_t* out_best_spins, void* cuda_stream) {
  if (!p || trials < 0 || S < 0 || (S > 0 && !betas) || trace_every <= 0 || !out_spins) return ISING_ERR_ARG;
  if (init_spins && init_spins == out_spins) return ISING_ERR_ARG;   // the chunks read one buffer, write another
  if (reinterpret_cast<uintptr_t>(out_spins) % 4 || reinterpret_cast<uintptr_t>(out_best_spins) % 4)
    return ISING_ERR_ARG;
  for (int32_t k = 0; k < S; ++k)
    if (!(betas[k] > 0.0)) return ISING_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (const int crc = ising::refuse_capture(st)) return crc;
  if (trials == 0) return ISING_OK;
  const size_t spin_bytes = static_cast<size_t>(trials) * p->n;
  const int32_t points = (S + trace_every - 1) / trace_every;

  // scratch: the other spin buffer of the ping-pong, and a cut row when the
  // caller keeps no trace
  unsigned char* scratch = nullptr;
  const size_t cut_bytes =
      (out_trace && points > 0) ? 0 : ((static_cast<size_t>(trials) * 4 + 255) & ~size_t(255));
  const size_t sbytes = (points > 1 ? ((spin_bytes + 255) & ~size_t(255)) : 0) + cut_bytes;
  if (sbytes) {
    const cudaError_t e = ising::dev_malloc_async(reinterpret_cast<void**>(&scratch), sbytes, st);
    if (e != cudaSuccess) return map_err(e);
  }
  int8_t* other = points > 1 ? reinterpret_cast<int8_t*>(scratch) : nullptr;
  int32_t* cut_row = cut_bytes ? reinterpret_cast<int32_t*>(scratch + (sbytes - cut_bytes)) : nullptr;

  int rc = ISING_OK;
  if (points == 0) {
    // no sweeps: the starting configuration is the only point
    int32_t* c = out_cuts ? out_cuts : cut_row;
    rc = ising_anneal(p, trials, betas, 0, seed, sweep_offset, init_spins, out_spins, c, cuda_stream);
    if (rc == ISING_OK && out_best) {
      best_update_kernel<<<trials, 256, 0, st>>>(c, out_spins, out_best, out_best_spins, p->n, 1);
      rc = map_err(cudaGetLastError());
    }
  }
  const int8_t* prev = init_spins;
  for (int32_t q = 0; q < points && rc == ISING_OK; ++q) {
    const int32_t j0 = q * trace_every;
    const int32_t len = (S - j0) < trace_every ? (S - j0) : trace_every;
    // the last chunk writes the caller's buffer; earlier ones alternate
    int8_t* dst = ((points - 1 - q) % 2 == 0) ? out_spins : other;
    int32_t* row = out_trace ? out_trace + static_cast<size_t>(q) * trials : cut_row;
    rc = ising_anneal(p, trials, betas + j0, len, seed, sweep_offset + static_cast<uint32_t>(j0), prev, dst, row,
                      cuda_stream);
    if (rc != ISING_OK) break;
    if (out_best) {
      best_update_kernel<<<trials, 256, 0, st>>>(row, dst, out_best, out_best_spins, p->n, q == 0 ? 1 : 0);
      rc = map_err(cudaGetLastError());
    }
    if (rc == ISING_OK && q == points - 1 && out_cuts) {
      rc = map_err(cudaMemcpyAsync(out_cuts, row, static_cast<size_t>(trials) * 4, cudaMemcpyDeviceToDevice, st));
    }
    prev = dst;
  }
  if (scratch) {
    const cudaError_t e = cudaFreeAsync(scratch, st);
    if (rc == ISING_OK) rc = map_err(e);
  }
  return rc;
}

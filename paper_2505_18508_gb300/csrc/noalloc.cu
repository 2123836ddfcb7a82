// noalloc.cu -- ising_anneal_noalloc: the annealer without any device
// allocation inside the call.
//
// Who needs this: callers that cannot call cudaMalloc (or cudaMallocAsync)
// during their run, for instance a host application whose framework has
// already reserved the device memory it is allowed to use, or a control loop
// that must not enter the CUDA allocator once it is running.  ising_anneal
// allocates its per-sweep threshold table in stream order on every call; this
// entry point instead keeps that table in one fixed array that lives in the
// library's device image, so the call itself allocates nothing.
//
// The fixed array holds kNoAllocMaxSweeps sweeps (256 KiB).  Every GPU that
// loads this library holds it until the process exits.  All calls on a
// device share it and it keeps the last call's contents; two calls whose work
// overlaps on the GPU (different streams, no ordering between them) race on
// it, so order such calls on one stream or with events.
#include <mutex>

#include "../../include/ising.h"
#include "internal.h"

namespace {

constexpr int32_t kNoAllocMaxSweeps = 32768;
constexpr int kMaxDevices = 64;

// (T4_k, T8_k) for every sweep of the current call; written by the fill
// kernels queued ahead of the annealing launch, read by that launch.
static __device__ __align__(256) uint32_t g_noalloc_thresholds[2 * kNoAllocMaxSweeps];

std::mutex g_setup_mutex;
uint32_t* g_table_of_device[kMaxDevices] = {};

// Device address of the fixed table on the current device; looked up once per
// device (the host-side name of a __device__ array is not a device address).
int table_address(int device, uint32_t** out) {
  if (device < 0 || device >= kMaxDevices) return ISING_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_table_of_device[device]) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_thresholds);
    if (e != cudaSuccess || ptr == nullptr) return ISING_ERR_CUDA;
    g_table_of_device[device] = static_cast<uint32_t*>(ptr);
  }
  *out = g_table_of_device[device];
  return ISING_OK;
}

// Copies one slice of the threshold table into the fixed array.  The words
// travel inside the kernel's parameters, which the launch copies when it is
// queued, so no host buffer has to outlive the call and no pageable
// host-to-device copy is involved.
constexpr int kFillWords = 2048;   // 1,024 sweeps (8 KiB of parameters) per launch
struct FillSlice {
  uint32_t w[kFillWords];
};
__global__ void fill_table_kernel(uint32_t* __restrict__ dst, const FillSlice slice, int32_t words) {
  for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = slice.w[i];
}

int map_err(cudaError_t e) {
  if (e == cudaSuccess) return ISING_OK;
  if (e == cudaErrorMemoryAllocation) return ISING_ERR_OOM;
  return ISING_ERR_CUDA;
}

}  // namespace

extern "C" int ising_anneal_noalloc(ising_problem* p, int32_t trials, const double* betas, int32_t S,
                                    uint64_t seed, uint32_t sweep_offset, const int8_t* init_spins,
                                    int8_t* out_spins, int32_t* out_cuts, void* cuda_stream) {
  if (!p || trials < 0 || S < 0 || (S > 0 && !betas)) return ISING_ERR_ARG;
  if (p->graph) return ISING_ERR_UNSUPPORTED;
  if (p->draw_bits == 16 && p->cfg_group % 8) return ISING_ERR_ARG;
  if (S > kNoAllocMaxSweeps) return ISING_ERR_UNSUPPORTED;
  for (int32_t k = 0; k < S; ++k)
    if (!(betas[k] > 0.0)) return ISING_ERR_ARG;
  if (trials == 0) return ISING_OK;
  int device = -1;
  if (cudaGetDevice(&device) != cudaSuccess) return ISING_ERR_CUDA;
  if (device != p->device) return ISING_ERR_ARG;
  uint32_t* table = nullptr;
  int rc = table_address(device, &table);
  if (rc != ISING_OK) return rc;

  // the launch shape ising_anneal gives the strip kernel
  ising::StripShape sh;
  rc = ising::strip_shape(p, trials, 0, &sh);
  if (rc != ISING_OK) return rc;

  // thresholds into the fixed table, one slice per fill launch
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  FillSlice slice;
  for (int32_t k0 = 0; k0 < S; k0 += kFillWords / 2) {
    const int32_t m = S - k0 < kFillWords / 2 ? S - k0 : kFillWords / 2;
    rc = ising::threshold_table(betas + k0, m, p->draw_bits, slice.w);
    if (rc != ISING_OK) return rc;
    fill_table_kernel<<<1, 256, 0, st>>>(table + 2 * static_cast<size_t>(k0), slice, 2 * m);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return map_err(e);
  }

  ising::AnnealArgs a{};
  a.flags = p->d_flags;
  a.thr = table;
  a.init = init_spins;
  a.out_spins = out_spins;
  a.out_cuts = out_cuts;
  a.X = p->X; a.Y = p->Y; a.H = p->H; a.n = p->n;
  a.T = trials;
  a.G = sh.G;
  a.S = S;
  a.k0 = sweep_offset;
  a.key0 = static_cast<uint32_t>(seed & 0xFFFFFFFFull);
  a.key1 = static_cast<uint32_t>(seed >> 32);
  for (uint32_t r = 0; r < 10; ++r) {
    a.rk[2 * r] = a.key0 + r * 0x9E3779B9u;
    a.rk[2 * r + 1] = a.key1 + r * 0xBB67AE85u;
  }
  a.C = sh.C;
  a.Rmax = sh.Rmax;
  a.neg_edges = p->neg_edges;
  a.u16 = p->draw_bits == 16 ? 1 : 0;
  const cudaError_t e = ising::launch_anneal(a, sh.threads, st);
  if (e != cudaSuccess) return map_err(e);
  ising::record_strip_launch(p, trials, S, sh);
  return ISING_OK;
}

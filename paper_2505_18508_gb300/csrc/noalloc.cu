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
#include <cmath>
#include <mutex>

#include "../../include/ising.h"
#include "internal.h"

namespace {

constexpr int32_t kNoAllocMaxSweeps = 32768;
constexpr int kMaxDevices = 64;

// (T4_k, T8_k) for every sweep of the current call; written by the host
// through its device address before each launch, read by the kernel.
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

// floor(exp(-beta dE) 2^32), clamped to 2^32 - 1, for dE = 4 and 8 (the same
// acceptance thresholds as ising_anneal); in the 16-bit draw mode
// floor(exp(-beta dE) 2^16), clamped to 2^16 - 1, shifted left by 16 bits
int threshold_pair(double beta, int bits, uint32_t* t4, uint32_t* t8) {
  if (!(beta > 0.0)) return ISING_ERR_ARG;
  const double scale = bits == 16 ? 65536.0 : 4294967296.0;
  const double v4 = std::floor(std::exp(-(beta * 4.0)) * scale);
  const double v8 = std::floor(std::exp(-(beta * 8.0)) * scale);
  const uint32_t top = bits == 16 ? 0xFFFFu : 0xFFFFFFFFu;
  const uint32_t a4 = v4 >= scale - 1.0 ? top : static_cast<uint32_t>(v4);
  const uint32_t a8 = v8 >= scale - 1.0 ? top : static_cast<uint32_t>(v8);
  *t4 = bits == 16 ? a4 << 16 : a4;
  *t8 = bits == 16 ? a8 << 16 : a8;
  return ISING_OK;
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

  // launch shape: the handle's fixed shape, else one trial group of 32 per
  // cluster of strips as wide as fits one CTA per SM (same rule as ising_anneal)
  int sms = 0, smem_max = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0) sms = 152;
  if (cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess ||
      smem_max <= 0)
    smem_max = 227 * 1024;
  const int unit = p->draw_bits == 16 ? 8 : 4;   // trials per Philox block
  int G = p->cfg_group ? p->cfg_group : (trials >= 32 ? 32 : ((trials + unit - 1) / unit) * unit);
  const int groups = (trials + G - 1) / G;
  int C = p->cfg_strips;
  if (C == 0) {
    C = 1;
    while (C < 8 && groups * (C * 2) <= sms && p->Y / (C * 2) >= 2) C *= 2;
    while (C < 16 && ising::anneal_smem_bytes(p->H, (p->Y + C - 1) / C) > static_cast<size_t>(smem_max) &&
           C * 2 <= p->Y)
      C *= 2;
  }
  if (C > p->Y || groups > 65535) return ISING_ERR_UNSUPPORTED;
  const int Rmax = (p->Y + C - 1) / C;
  if (ising::anneal_smem_bytes(p->H, Rmax) > static_cast<size_t>(smem_max)) return ISING_ERR_UNSUPPORTED;
  int threads = p->cfg_threads;
  if (threads == 0) {
    const int items = Rmax * p->H;
    threads = 1024;
    if (items <= 768) {
      threads = ((items + 31) / 32) * 32;
      if (threads < 64) threads = 64;
    } else {
      double best = -1.0;
      for (int t = 768; t <= 1024; t += 32) {
        const int it = (items + t - 1) / t;
        const double eff = static_cast<double>(items) / (static_cast<double>(it) * t);
        if (eff > best + 1e-9 || (std::fabs(eff - best) <= 1e-9 && t > threads)) {
          best = eff;
          threads = t;
        }
      }
    }
  }

  // thresholds into the fixed table, through a small host buffer on the stack
  // (pageable host-to-device copies are staged before cudaMemcpyAsync returns,
  // so the buffer can be refilled right away)
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  constexpr int32_t kChunk = 512;
  uint32_t buf[2 * kChunk];
  for (int32_t k0 = 0; k0 < S; k0 += kChunk) {
    const int32_t m = S - k0 < kChunk ? S - k0 : kChunk;
    for (int32_t j = 0; j < m; ++j) {
      rc = threshold_pair(betas[k0 + j], p->draw_bits, &buf[2 * j], &buf[2 * j + 1]);
      if (rc != ISING_OK) return rc;
    }
    const cudaError_t e = cudaMemcpyAsync(table + 2 * static_cast<size_t>(k0), buf, sizeof(uint32_t) * 2 * m,
                                          cudaMemcpyHostToDevice, st);
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
  a.G = G;
  a.S = S;
  a.k0 = sweep_offset;
  a.key0 = static_cast<uint32_t>(seed & 0xFFFFFFFFull);
  a.key1 = static_cast<uint32_t>(seed >> 32);
  for (uint32_t r = 0; r < 10; ++r) {
    a.rk[2 * r] = a.key0 + r * 0x9E3779B9u;
    a.rk[2 * r + 1] = a.key1 + r * 0xBB67AE85u;
  }
  a.C = C;
  a.Rmax = Rmax;
  a.neg_edges = p->neg_edges;
  a.u16 = p->draw_bits == 16 ? 1 : 0;
  return map_err(ising::launch_anneal(a, threads, st));
}

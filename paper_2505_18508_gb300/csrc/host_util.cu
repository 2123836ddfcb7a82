// host_util.cu -- host-side services of the library: device allocation with
// a test hook that makes allocations fail (fault injection on the host, never
// on the GPU), the log level, hex import/export of configurations, and the
// decision-stream generator as an entry point.
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "../../include/ising.h"
#include "device_common.cuh"
#include "internal.h"

namespace {

std::mutex g_alloc_mutex;
int g_alloc_failures = 0;   // the next this many allocations fail

bool take_failure() {
  std::lock_guard<std::mutex> lock(g_alloc_mutex);
  if (g_alloc_failures > 0) {
    --g_alloc_failures;
    return true;
  }
  return false;
}

__global__ void philox_kernel(const uint4* __restrict__ ctr, uint32_t k0, uint32_t k1, int32_t k,
                              uint4* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < k) {
    const uint4 c = ctr[t];
    out[t] = ising::philox4x32_10(c.x, c.y, c.z, c.w, k0, k1);
  }
}

int hex_value(char c) {
  if (c >= '0' && c <= '9') return c - '0';
  if (c >= 'a' && c <= 'f') return c - 'a' + 10;
  if (c >= 'A' && c <= 'F') return c - 'A' + 10;
  return -1;
}

}  // namespace

namespace ising {

cudaError_t dev_malloc(void** p, size_t bytes) {
  if (take_failure()) return cudaErrorMemoryAllocation;
  return cudaMalloc(p, bytes);
}

// The library's stream-ordered allocations come from a pool of its own per
// device that keeps the memory it has held (release threshold: all of it).
// The default pool returns freed memory at every synchronisation, and mapping
// it again made the first call after one several milliseconds slower.
static cudaError_t library_pool(cudaMemPool_t* pool) {
  static std::mutex m;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaDeviceGetDefaultMemPool(pool, dev);
  std::lock_guard<std::mutex> lock(m);
  if (!pools[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t created = nullptr;
    e = cudaMemPoolCreate(&created, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = ~0ull;
    e = cudaMemPoolSetAttribute(created, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(created);
      return e;
    }
    pools[dev] = created;
  }
  *pool = pools[dev];
  return cudaSuccess;
}

cudaError_t dev_malloc_async(void** p, size_t bytes, cudaStream_t st) {
  if (take_failure()) return cudaErrorMemoryAllocation;
  cudaMemPool_t pool = nullptr;
  const cudaError_t e = library_pool(&pool);
  if (e != cudaSuccess) return e;
  return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

size_t static_smem_of(const void* kernel) {
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) {
    (void)cudaGetLastError();   // leave no error for the next launch check to find
    return 1024;
  }
  return fa.sharedSizeBytes;
}

int refuse_capture(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const cudaError_t e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    // the legacy stream while another stream captures in global mode
    return e == cudaErrorStreamCaptureImplicit ? ISING_ERR_UNSUPPORTED : ISING_ERR_CUDA;
  }
  return cs == cudaStreamCaptureStatusNone ? ISING_OK : ISING_ERR_UNSUPPORTED;
}

int log_level() {
  static const int level = [] {
    const char* v = std::getenv("ISING_LOG");
    return v ? std::atoi(v) : 0;
  }();
  return level;
}

}  // namespace ising

extern "C" {

int ising_debug_fail_allocs(int32_t count) {
  if (count < 0) return ISING_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_alloc_mutex);
  g_alloc_failures = count;
  return ISING_OK;
}

int ising_philox(const uint32_t* ctr, uint64_t seed, int32_t k, uint32_t* out, void* cuda_stream) {
  if (k < 0 || (k > 0 && (!ctr || !out))) return ISING_ERR_ARG;
  if (k == 0) return ISING_OK;
  if (reinterpret_cast<uintptr_t>(ctr) % 16 || reinterpret_cast<uintptr_t>(out) % 16) return ISING_ERR_ARG;
  philox_kernel<<<(k + 255) / 256, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
      reinterpret_cast<const uint4*>(ctr), static_cast<uint32_t>(seed & 0xFFFFFFFFull),
      static_cast<uint32_t>(seed >> 32), k, reinterpret_cast<uint4*>(out));
  return cudaGetLastError() == cudaSuccess ? ISING_OK : ISING_ERR_CUDA;
}

int ising_spins_to_hex(const int8_t* spins, int32_t n, char* out, int64_t cap) {
  if (n < 0 || (n > 0 && !spins) || !out) return ISING_ERR_ARG;
  const int64_t digits = (static_cast<int64_t>(n) + 3) / 4;
  if (cap < digits + 1) return ISING_ERR_ARG;
  static const char kHex[] = "0123456789ABCDEF";
  for (int64_t d = 0; d < digits; ++d) {
    int v = 0;
    for (int b = 0; b < 4; ++b) {
      const int64_t i = 4 * d + b;
      v = (v << 1) | (i < n && spins[i] > 0 ? 1 : 0);
    }
    out[d] = kHex[v];
  }
  out[digits] = '\0';
  return ISING_OK;
}

int ising_hex_to_spins(const char* hex, int32_t n, int8_t* out) {
  if (!hex || n < 0 || (n > 0 && !out)) return ISING_ERR_ARG;
  const int64_t digits = (static_cast<int64_t>(n) + 3) / 4;
  int64_t d = 0;
  for (const char* c = hex; *c; ++c) {
    if (*c == ' ' || *c == '\n' || *c == '\r' || *c == '\t') continue;
    const int v = hex_value(*c);
    if (v < 0 || d >= digits) return ISING_ERR_ARG;
    for (int b = 0; b < 4; ++b) {
      const int64_t i = 4 * d + b;
      const int bit = (v >> (3 - b)) & 1;
      if (i < n) out[i] = bit ? 1 : -1;
      else if (bit) return ISING_ERR_ARG;   // padding bits must be 0
    }
    ++d;
  }
  return d == digits ? ISING_OK : ISING_ERR_ARG;
}

}  // extern "C"

// abi.cu -- the C ABI declared in include/ising.h: argument checks, instance
// packing, per-sweep thresholds and the choice of launch shape.
//
// Everything here is host code; the kernels live in anneal.cu, cut.cu and
// batched.cu.  No C++ exception leaves an extern "C" function.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/ising.h"
#include "internal.h"

namespace {

int map_cuda(cudaError_t e) {
  if (e == cudaSuccess) return ISING_OK;
  if (e == cudaErrorMemoryAllocation) return ISING_ERR_OOM;
  return ISING_ERR_CUDA;
}

// T_d = min(floor(exp(-beta d) 2^32), 2^32 - 1) for d = 4 and 8: the
// Metropolis acceptance probability min(1, exp(-beta dE)) of an uphill move,
// as an integer threshold for a uniform 32-bit draw (accept iff u < T).
int make_thresholds(const double* betas, int32_t S, std::vector<uint32_t>& out) {
  out.assign(static_cast<size_t>(2) * (S > 0 ? S : 0), 0u);
  for (int32_t k = 0; k < S; ++k) {
    const double beta = betas[k];
    if (!(beta > 0.0)) return ISING_ERR_ARG;
    for (int d = 0; d < 2; ++d) {
      const double dE = d == 0 ? 4.0 : 8.0;
      const double v = std::floor(std::exp(-(beta * dE)) * 4294967296.0);
      out[2 * static_cast<size_t>(k) + d] = v >= 4294967295.0 ? 0xFFFFFFFFu : static_cast<uint32_t>(v);
    }
  }
  return ISING_OK;
}

int num_sms_of(int device) {
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || v <= 0) v = 148;
  return v;
}

int max_smem_of(int device) {
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess || v <= 0)
    v = 227 * 1024;
  return v;
}

struct Shape {
  int G, C, threads, Rmax;
};

// threads per CTA: the multiple of 32 in [lo, hi] that leaves the fewest idle
// item slots over the half-sweep (ties -> more threads)
int pick_threads(int items, int lo, int hi) {
  int best = hi;
  double best_eff = -1.0;
  for (int t = lo; t <= hi; t += 32) {
    const int iters = (items + t - 1) / t;
    const double eff = static_cast<double>(items) / (static_cast<double>(iters) * t);
    if (eff > best_eff + 1e-9 || (std::fabs(eff - best_eff) <= 1e-9 && t > best)) {
      best_eff = eff;
      best = t;
    }
  }
  return best;
}

int choose_shape(const ising_problem* p, int32_t T, Shape* out) {
  const int sms = num_sms_of(p->device);
  const int smem_max = max_smem_of(p->device);
  int G = p->cfg_group;
  if (G == 0) G = T >= 32 ? 32 : ((T + 3) / 4) * 4;
  if (G < 4) G = 4;
  const int groups = (T + G - 1) / G;
  int C = p->cfg_strips;
  if (C == 0) {
    C = 1;
    while (C < 8 && groups * C < sms && p->Y / (C * 2) >= 2) C *= 2;
    while (C < 16 && ising::anneal_smem_bytes(p->H, (p->Y + C - 1) / C) > static_cast<size_t>(smem_max) &&
           (C * 2) <= p->Y)
      C *= 2;
  }
  if (C > p->Y) return ISING_ERR_UNSUPPORTED;
  const int Rmax = (p->Y + C - 1) / C;
  if (ising::anneal_smem_bytes(p->H, Rmax) > static_cast<size_t>(smem_max)) return ISING_ERR_UNSUPPORTED;
  if (groups > 65535) return ISING_ERR_UNSUPPORTED;
  int threads = p->cfg_threads;
  if (threads == 0) threads = pick_threads(Rmax * p->H, 128, C == 1 ? 1024 : 512);
  out->G = G;
  out->C = C;
  out->threads = threads;
  out->Rmax = Rmax;
  return ISING_OK;
}

}  // namespace

extern "C" {

const char* ising_strerror(int code) {
  switch (code) {
    case ISING_OK: return "ok";
    case ISING_ERR_ARG: return "invalid argument";
    case ISING_ERR_NOT_TORUS: return "CSR is not a symmetric 4-neighbour torus of the given shape";
    case ISING_ERR_ODD_DIM: return "torus width and height must be even";
    case ISING_ERR_H_UNSUPPORTED: return "non-zero local fields h are not supported";
    case ISING_ERR_OOM: return "out of memory";
    case ISING_ERR_CUDA: return "CUDA error";
    case ISING_ERR_TIMEOUT: return "bounded device wait timed out";
    case ISING_ERR_UNSUPPORTED: return "valid input outside what this build supports";
    default: return "unknown status code";
  }
}

int ising_create(int32_t n, const int64_t* row_ptr, const int32_t* col_idx, const int8_t* J,
                 const int8_t* h, int32_t X, int32_t Y, ising_problem** out) {
  if (!row_ptr || !col_idx || !J || !out) return ISING_ERR_ARG;
  if (X < 4 || Y < 4) return ISING_ERR_ARG;
  if ((X & 1) || (Y & 1)) return ISING_ERR_ODD_DIM;
  if (static_cast<int64_t>(X) * Y != n || n > (1 << 28)) return ISING_ERR_ARG;
  if (row_ptr[0] != 0) return ISING_ERR_NOT_TORUS;
  for (int32_t i = 0; i < n; ++i)
    if (row_ptr[i + 1] - row_ptr[i] != 4) return ISING_ERR_NOT_TORUS;
  if (h) {
    for (int32_t i = 0; i < n; ++i)
      if (h[i] != 0) return ISING_ERR_H_UNSUPPORTED;
  }
  // J of each site towards left, right, up, down
  std::vector<int8_t> jl, jr, ju, jd;
  try {
    jl.resize(n); jr.resize(n); ju.resize(n); jd.resize(n);
  } catch (const std::bad_alloc&) {
    return ISING_ERR_OOM;
  }
  for (int32_t y = 0; y < Y; ++y) {
    for (int32_t x = 0; x < X; ++x) {
      const int32_t i = y * X + x;
      const int32_t want[4] = {y * X + (x + X - 1) % X, y * X + (x + 1) % X, ((y + Y - 1) % Y) * X + x,
                               ((y + 1) % Y) * X + x};
      bool seen[4] = {false, false, false, false};
      int8_t val[4] = {0, 0, 0, 0};
      for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
        const int8_t v = J[e];
        if (v != 1 && v != -1) return ISING_ERR_ARG;
        int which = -1;
        for (int d = 0; d < 4; ++d)
          if (col_idx[e] == want[d]) which = d;
        if (which < 0 || seen[which]) return ISING_ERR_NOT_TORUS;
        seen[which] = true;
        val[which] = v;
      }
      jl[i] = val[0]; jr[i] = val[1]; ju[i] = val[2]; jd[i] = val[3];
    }
  }
  // symmetry J_ij = J_ji
  for (int32_t y = 0; y < Y; ++y)
    for (int32_t x = 0; x < X; ++x) {
      const int32_t i = y * X + x;
      if (jr[i] != jl[y * X + (x + 1) % X]) return ISING_ERR_NOT_TORUS;
      if (jd[i] != ju[((y + 1) % Y) * X + x]) return ISING_ERR_NOT_TORUS;
    }
  // pack: w = -J, flag bit set where w = -1, i.e. J = +1
  const int32_t H = X / 2;
  std::vector<uint8_t> flags(n), eflags(n);
  int32_t neg = 0;
  for (int32_t y = 0; y < Y; ++y)
    for (int32_t x = 0; x < X; ++x) {
      const int32_t i = y * X + x;
      const int c = (x + y) & 1;
      const uint8_t f = static_cast<uint8_t>((jl[i] == 1 ? 1 : 0) | (jr[i] == 1 ? 2 : 0) | (ju[i] == 1 ? 4 : 0) |
                                             (jd[i] == 1 ? 8 : 0));
      flags[(static_cast<size_t>(c) * Y + y) * H + (x >> 1)] = f;
      eflags[i] = static_cast<uint8_t>((jr[i] == 1 ? 1 : 0) | (jd[i] == 1 ? 2 : 0));
      neg += (jr[i] == 1) + (jd[i] == 1);
    }
  ising_problem* p = new (std::nothrow) ising_problem();
  if (!p) return ISING_ERR_OOM;
  p->X = X; p->Y = Y; p->n = n; p->H = H;
  p->neg_edges = neg;
  p->weight_sum = 2 * n - 2 * neg;
  if (cudaGetDevice(&p->device) != cudaSuccess) { delete p; return ISING_ERR_CUDA; }
  cudaError_t e = cudaMalloc(&p->d_flags, n);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_eflags, n);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_flags, flags.data(), n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_eflags, eflags.data(), n, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(p->d_flags);
    cudaFree(p->d_eflags);
    delete p;
    return map_cuda(e);
  }
  *out = p;
  return ISING_OK;
}

void ising_destroy(ising_problem* p) {
  if (!p) return;
  cudaFree(p->d_flags);
  cudaFree(p->d_eflags);
  delete p;
}

int ising_set_launch(ising_problem* p, int32_t group_trials, int32_t strips, int32_t threads) {
  if (!p) return ISING_ERR_ARG;
  if (group_trials != 0 && (group_trials < 4 || group_trials > 32 || group_trials % 4)) return ISING_ERR_ARG;
  if (strips != 0 && (strips < 1 || strips > 16 || strips > p->Y)) return ISING_ERR_ARG;
  if (threads != 0 && (threads < 64 || threads > 1024 || threads % 32)) return ISING_ERR_ARG;
  p->cfg_group = group_trials;
  p->cfg_strips = strips;
  p->cfg_threads = threads;
  return ISING_OK;
}

int ising_last_launch(const ising_problem* p, int32_t* group_trials, int32_t* strips, int32_t* threads,
                      int32_t* grid_ctas) {
  if (!p) return ISING_ERR_ARG;
  if (group_trials) *group_trials = p->last_group;
  if (strips) *strips = p->last_strips;
  if (threads) *threads = p->last_threads;
  if (grid_ctas) *grid_ctas = p->last_grid;
  return ISING_OK;
}

int ising_problem_info(const ising_problem* p, int32_t* X, int32_t* Y, int32_t* weight_sum) {
  if (!p) return ISING_ERR_ARG;
  if (X) *X = p->X;
  if (Y) *Y = p->Y;
  if (weight_sum) *weight_sum = p->weight_sum;
  return ISING_OK;
}

int ising_anneal(ising_problem* p, int32_t trials, const double* betas, int32_t S, uint64_t seed,
                 uint32_t sweep_offset, const int8_t* init_spins, int8_t* out_spins, int32_t* out_cuts,
                 void* cuda_stream) {
  if (!p || trials < 0 || S < 0 || (S > 0 && !betas)) return ISING_ERR_ARG;
  std::vector<uint32_t> thr;
  try {
    const int rc = make_thresholds(betas, S, thr);
    if (rc != ISING_OK) return rc;
  } catch (const std::bad_alloc&) {
    return ISING_ERR_OOM;
  }
  if (trials == 0) return ISING_OK;
  Shape sh;
  const int rc = choose_shape(p, trials, &sh);
  if (rc != ISING_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  uint32_t* d_thr = nullptr;
  const size_t thr_bytes = thr.size() * sizeof(uint32_t);
  if (thr_bytes) {
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&d_thr), thr_bytes, st);
    if (e != cudaSuccess) return map_cuda(e);
    e = cudaMemcpyAsync(d_thr, thr.data(), thr_bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) { cudaFreeAsync(d_thr, st); return map_cuda(e); }
  }
  ising::AnnealArgs a;
  a.flags = p->d_flags;
  a.thr = d_thr;
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
  a.C = sh.C;
  a.Rmax = sh.Rmax;
  a.neg_edges = p->neg_edges;
  cudaError_t e = ising::launch_anneal(a, sh.threads, st);
  if (d_thr) {
    const cudaError_t e2 = cudaFreeAsync(d_thr, st);
    if (e == cudaSuccess) e = e2;
  }
  if (e != cudaSuccess) return map_cuda(e);
  p->last_group = sh.G;
  p->last_strips = sh.C;
  p->last_threads = sh.threads;
  p->last_grid = sh.C * ((trials + sh.G - 1) / sh.G);
  return ISING_OK;
}

int ising_cut(const ising_problem* p, const int8_t* spins, int32_t k, int32_t* out_cuts, void* cuda_stream) {
  if (!p || k < 0 || (k > 0 && (!spins || !out_cuts))) return ISING_ERR_ARG;
  return map_cuda(ising::launch_cut(p, spins, k, out_cuts, static_cast<cudaStream_t>(cuda_stream)));
}

int ising_anneal_batched(ising_problem* const*, int32_t, const int32_t*, const int32_t*, const double* const*,
                         const uint64_t*, int8_t* const*, int32_t* const*, void*) {
  return ISING_ERR_UNSUPPORTED;
}
int ising_batch_create(ising_problem* const*, int32_t, const int32_t*, const int32_t*, const double* const*,
                       const uint64_t*, int8_t* const*, int32_t* const*, int32_t, int32_t, void*, ising_batch**) {
  return ISING_ERR_UNSUPPORTED;
}
int ising_batch_launch(ising_batch*, void*) { return ISING_ERR_UNSUPPORTED; }
void ising_batch_destroy(ising_batch*) {}

}  // extern "C"

// clusters.cu -- connected-component moves on the torus, judged by their
// exact integer energy change (Eq. 2 with J = -w: H = sum w_ij s_i s_j).
//
// For a set of sites M, its connected components under 4-neighbour adjacency
// (with the periodic wrap) are never adjacent to one another, so flipping
// component C changes the energy by its own boundary terms only:
// dE_C = -2 sum_{i in C, j ~ i, j not in M} w_ij s_i s_j, and any set of
// components can be flipped together with the sum of their changes.
//
// * Proposals (the learned stage's block flips): M = the sites whose logit is
//   > 0; every component with dE_C <= 0 is flipped.
// * Droplet targets (its training labels): M = the sites where s differs from
//   the gauge-aligned better state r' (r or -r, whichever is closer to s; a
//   tie keeps site 0); y_i = 1 iff i lies in a component with dE_C < 0, an
//   exact energy-lowering move from s towards r'.
// * Partner moves: the same components with r = another configuration of the
//   same problem (partner (t + shift) mod B), every component with dE_C < 0
//   flipped; all configurations read their partners' states before any move
//   (input and output buffers differ).
//
// One CTA per configuration, everything in shared memory: the spins, a label
// per site (the smallest site index of its component once converged) and a
// dE accumulator per label.  Labels converge by repeated minimum propagation
// over the neighbours plus one pointer jump per pass; every pass that changes
// nothing ends the loop, and a pass can only lower labels, so at most n
// passes run.
#include <climits>

#include "../../include/ising.h"
#include "internal.h"

namespace ising {
namespace {

constexpr int kClusterThreads = 1024;
constexpr int kMaxClusterProblems = 16;

struct ClusterArgs {
  int8_t* spins;                  // [B][n] (proposals: updated in place; partner moves: read only)
  int8_t* out;                    // [B][n] new states (partner moves)
  int32_t shift;                  // partner offset within a problem's configurations (partner moves)
  const float* logits;            // [B][n] (proposals) or null
  const int8_t* ref;              // [B][n] (targets) or null
  uint8_t* targets;               // [B][n] (targets) or null
  int32_t* accepted;              // [B] components flipped (proposals) or null
  int32_t accumulate;             // 1: add to accepted instead of writing it
  const uint8_t* eflags[kMaxClusterProblems];   // per problem: bit 0 right edge w = -1, bit 1 down edge
  int32_t per_problem;            // configurations per problem: image b uses eflags[b / per_problem]
  int32_t X, Y;
  int32_t use_list;               // 1: the masked sites are listed in shared memory at byte offset list_off
  uint32_t list_off;
};

__device__ __forceinline__ int wrapc(int v, int m) { return v < 0 ? v + m : (v >= m ? v - m : v); }

// kMode: 0 = proposals from logits, 1 = droplet targets, 2 = partner moves
template <int kMode>
__global__ void __launch_bounds__(kClusterThreads) cluster_kernel(const ClusterArgs a) {
  constexpr bool kTargets = kMode != 0;   // the mask is the disagreement with a reference
  extern __shared__ __align__(16) unsigned char smem[];
  const int X = a.X, Y = a.Y, n = X * Y;
  int32_t* lab = reinterpret_cast<int32_t*>(smem);            // [n]
  int32_t* dE = lab + n;                                        // [n]
  int8_t* sv = reinterpret_cast<int8_t*>(dE + n);               // [n]
  __shared__ int red[32];
  __shared__ int s_flag;
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31;
  const uint8_t* ef = a.eflags[b / a.per_problem];
  int8_t* s = a.spins + static_cast<size_t>(b) * n;

  // gauge of the reference (targets and partner moves): r' = -r when more than half of the
  // sites differ, or exactly half and site 0 differs
  const int8_t* r = nullptr;
  if constexpr (kMode == 1) r = a.ref + static_cast<size_t>(b) * n;
  if constexpr (kMode == 2) {
    const int q = b / a.per_problem, t = b - q * a.per_problem;
    r = a.spins + (static_cast<size_t>(q) * a.per_problem + (t + a.shift) % a.per_problem) * n;
  }
  int flip_ref = 0;
  if constexpr (kTargets) {
    int d = 0;
    for (int i = tid; i < n; i += kClusterThreads) d += (s[i] > 0) != (r[i] > 0);
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xFFFFFFFFu, d, o);
    if (lane == 0) red[tid >> 5] = d;
    __syncthreads();
    if (tid == 0) {
      int t = 0;
      for (int w = 0; w < kClusterThreads / 32; ++w) t += red[w];
      s_flag = (2 * t > n) || (2 * t == n && ((s[0] > 0) != (r[0] > 0)));
    }
    __syncthreads();
    flip_ref = s_flag;
  }
  for (int i = tid; i < n; i += kClusterThreads) {
    const int8_t si = s[i] > 0 ? int8_t(1) : int8_t(-1);
    bool in;
    if constexpr (kTargets) {
      in = (((s[i] > 0) != (r[i] > 0)) ? 1 : 0) ^ flip_ref;
    } else {
      in = a.logits[static_cast<size_t>(b) * n + i] > 0.f;
    }
    sv[i] = si;
    lab[i] = in ? i : INT_MAX;
    dE[i] = 0;
  }
  __syncthreads();

  // ---- the masked sites as a list (when it fits in shared memory): the
  // label passes and the energy sums then visit only them
  const bool use_list = a.use_list != 0;
  uint16_t* list = reinterpret_cast<uint16_t*>(smem + a.list_off);
  __shared__ int s_cnt;
  int nlist = n;
  if (use_list) {
    if (tid == 0) s_cnt = 0;
    __syncthreads();
    for (int i0 = 0; i0 < n; i0 += kClusterThreads) {   // the same count of iterations in every thread
      const int i = i0 + tid;
      const bool m = i < n && lab[i] != INT_MAX;
      const unsigned bal = __ballot_sync(0xFFFFFFFFu, m);
      int base = 0;
      if (lane == 0 && bal != 0u) base = atomicAdd(&s_cnt, __popc(bal));
      base = __shfl_sync(0xFFFFFFFFu, base, 0);
      if (m) list[base + __popc(bal & ((1u << lane) - 1u))] = static_cast<uint16_t>(i);
    }
    __syncthreads();
    nlist = s_cnt;
  }
  // row of a listed site without a division: floor(i * ceil(2^32 / X) / 2^32)
  // is exact for i, X < 2^16
  const uint32_t mX = X > 1 ? 0xFFFFFFFFu / static_cast<uint32_t>(X) + 1u : 0u;
  auto row_of = [&](int i) { return X > 1 ? static_cast<int>(__umulhi(static_cast<uint32_t>(i), mX)) : i; };

  // one relaxation of masked site i at (y, x): the minimum over its masked
  // neighbours and one pointer jump; true if its label fell
  auto relax = [&](int i, int y, int x) {
    const int l = lab[i];
    int mn = l;
    const int j0 = y * X + wrapc(x + 1, X), j1 = y * X + wrapc(x - 1, X);
    const int j2 = wrapc(y + 1, Y) * X + x, j3 = wrapc(y - 1, Y) * X + x;
    mn = min(mn, lab[j0]);
    mn = min(mn, lab[j1]);
    mn = min(mn, lab[j2]);
    mn = min(mn, lab[j3]);
    mn = min(mn, lab[mn]);
    if (mn < l) {
      atomicMin(&lab[i], mn);
      atomicMin(&lab[l], mn);   // lower the old label's site too: joins the trees faster
      return true;
    }
    return false;
  };
  // the boundary terms of masked site i at (y, x)
  auto boundary = [&](int i, int y, int x) {
    const int xl = wrapc(x - 1, X), xr = wrapc(x + 1, X), yu = wrapc(y - 1, Y), yd = wrapc(y + 1, Y);
    const int j[4] = {y * X + xr, y * X + xl, yd * X + x, yu * X + x};
    const int w[4] = {(ef[i] & 1u) ? -1 : 1, (ef[y * X + xl] & 1u) ? -1 : 1, (ef[i] & 2u) ? -1 : 1,
                      (ef[yu * X + x] & 2u) ? -1 : 1};
    int c = 0;
#pragma unroll
    for (int d = 0; d < 4; ++d)
      if (lab[j[d]] == INT_MAX) c += -2 * w[d] * sv[i] * sv[j[d]];
    return c;
  };

  // ---- labels: minimum over the masked neighbours, then one pointer jump
  // (without the list: site i = tid + m * kClusterThreads at row y, column x,
  // advanced without a division)
  const int dq = kClusterThreads / X, dr = kClusterThreads - dq * X;
  const int y_first = tid / X, x_first = tid - y_first * X;
  for (int pass = 0; pass <= n; ++pass) {
    if (tid == 0) s_flag = 0;
    __syncthreads();
    int changed = 0;
    if (use_list) {
      for (int q = tid; q < nlist; q += kClusterThreads) {
        const int i = list[q];
        const int y = row_of(i);
        if (relax(i, y, i - y * X)) changed = 1;
      }
    } else {
      int y = y_first, x = x_first;
      for (int i = tid; i < n; i += kClusterThreads, y += dq, x += dr) {
        if (x >= X) {
          x -= X;
          ++y;
        }
        if (lab[i] == INT_MAX) continue;
        if (relax(i, y, x)) changed = 1;
      }
    }
    if (changed) s_flag = 1;
    __syncthreads();
    const int again = s_flag;
    __syncthreads();
    if (!again) break;
  }

  // ---- dE per component: boundary terms, summed per label within a warp first
  const int span = (nlist + kClusterThreads - 1) / kClusterThreads * kClusterThreads;
  int y = y_first, x = x_first;
  for (int q = tid; q < span; q += kClusterThreads, y += dq, x += dr) {
    if (x >= X) {
      x -= X;
      ++y;
    }
    int l = INT_MAX, c = 0;
    if (q < nlist) {
      if (use_list) {
        const int i = list[q];
        const int yi = row_of(i);
        l = lab[i];
        c = boundary(i, yi, i - yi * X);
      } else {
        l = lab[q];
        if (l != INT_MAX) c = boundary(q, y, x);
      }
    }
    // only lanes with a boundary term take part (most warps have none)
    if (__ballot_sync(0xFFFFFFFFu, c != 0) == 0u) continue;
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, l);
    const int sum = __reduce_add_sync(peers, c);
    if (l != INT_MAX && lane == __ffs(peers) - 1 && sum != 0) atomicAdd(&dE[l], sum);
  }
  __syncthreads();

  // ---- apply
  int cnt = 0;
  for (int i = tid; i < n; i += kClusterThreads) {
    const int l = lab[i];
    if constexpr (kMode == 1) {
      a.targets[static_cast<size_t>(b) * n + i] = static_cast<uint8_t>(l != INT_MAX && dE[l] < 0);
    } else if constexpr (kMode == 2) {
      const bool f = l != INT_MAX && dE[l] < 0;
      a.out[static_cast<size_t>(b) * n + i] = f ? static_cast<int8_t>(-sv[i]) : sv[i];
      cnt += f && l == i;
    } else {
      if (l != INT_MAX && dE[l] <= 0) {
        s[i] = static_cast<int8_t>(-sv[i]);
        cnt += l == i;   // one count per flipped component, at its label site
      }
    }
  }
  if constexpr (kMode != 1) {
    if (a.accepted) {
      for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
      __syncthreads();
      if (lane == 0) red[tid >> 5] = cnt;
      __syncthreads();
      if (tid == 0) {
        int t = 0;
        for (int w = 0; w < kClusterThreads / 32; ++w) t += red[w];
        a.accepted[b] = a.accumulate ? a.accepted[b] + t : t;
      }
    }
  }
}

size_t cluster_smem(int n) { return static_cast<size_t>(n) * 9; }
// with the list of masked sites (16-bit indices) after the other arrays
size_t cluster_list_off(int n) { return (cluster_smem(n) + 15) & ~static_cast<size_t>(15); }
size_t cluster_smem_list(int n) { return cluster_list_off(n) + static_cast<size_t>(n) * 2; }

// the dynamic shared memory a launch of `kernel` may ask for: the per-block
// opt-in limit less the kernel's own static arrays
int cluster_dyn_max(const void* kernel, int* out) {
  int dev = 0, smem_max = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return ISING_ERR_CUDA;
  *out = smem_max - static_cast<int>(static_smem_of(kernel));
  return ISING_OK;
}

template <int kMode>
int cluster_check(const ising_problem* const* probs, int32_t m, int32_t B, ClusterArgs* a) {
  if (!probs || m < 1 || m > kMaxClusterProblems || B < 0) return ISING_ERR_ARG;
  for (int q = 0; q < m; ++q) {
    if (!probs[q]) return ISING_ERR_ARG;
    if (probs[q]->graph) return ISING_ERR_UNSUPPORTED;
    if (probs[q]->X != probs[0]->X || probs[q]->Y != probs[0]->Y) return ISING_ERR_ARG;
  }
  int dyn_max = 0;
  const int rc = cluster_dyn_max(reinterpret_cast<const void*>(cluster_kernel<kMode>), &dyn_max);
  if (rc != ISING_OK) return rc;
  if (dyn_max < 0 || cluster_smem(probs[0]->n) > static_cast<size_t>(dyn_max)) return ISING_ERR_UNSUPPORTED;
  for (int q = 0; q < m; ++q) a->eflags[q] = probs[q]->d_eflags;
  a->per_problem = B > 0 ? B : 1;
  a->X = probs[0]->X;
  a->Y = probs[0]->Y;
  return ISING_OK;
}

template <int kMode>
int launch_clusters(ClusterArgs a, int32_t images, cudaStream_t st) {
  const int n = a.X * a.Y;
  int dyn_max = 0;
  const int rc = cluster_dyn_max(reinterpret_cast<const void*>(cluster_kernel<kMode>), &dyn_max);
  if (rc != ISING_OK) return rc;
  a.use_list = n < 65536 && dyn_max >= 0 && cluster_smem_list(n) <= static_cast<size_t>(dyn_max) ? 1 : 0;
  a.list_off = static_cast<uint32_t>(cluster_list_off(n));
  const size_t sm = a.use_list ? cluster_smem_list(n) : cluster_smem(n);
  if (cudaFuncSetAttribute(cluster_kernel<kMode>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(sm)) != cudaSuccess)
    return ISING_ERR_CUDA;
  cluster_kernel<kMode><<<images, kClusterThreads, sm, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? ISING_OK : ISING_ERR_CUDA;
}

}  // namespace
}  // namespace ising

namespace ising {

int propose_clusters_launch(const ising_problem* const* probs, int32_t m, int8_t* spins, int32_t B,
                            const float* logits, int32_t* accepted, int accumulate, cudaStream_t st) {
  ClusterArgs a{};
  const int rc = cluster_check<0>(probs, m, B, &a);
  if (rc != ISING_OK) return rc;
  if (B > 0 && (!spins || !logits)) return ISING_ERR_ARG;
  if (B == 0) return ISING_OK;
  if (static_cast<long long>(m) * B > 0x7FFFFFFFLL) return ISING_ERR_UNSUPPORTED;
  a.spins = spins;
  a.logits = logits;
  a.accepted = accepted;
  a.accumulate = accumulate;
  return launch_clusters<0>(a, m * B, st);
}

int transcribe_launch(const ising_problem* const* probs, int32_t m, const int8_t* spins, int8_t* out, int32_t B,
                      int32_t shift, int32_t* accepted, int accumulate, cudaStream_t st) {
  ClusterArgs a{};
  const int rc = cluster_check<2>(probs, m, B, &a);
  if (rc != ISING_OK) return rc;
  if (shift < 0 || (B > 0 && (!spins || !out || spins == out))) return ISING_ERR_ARG;
  if (B == 0) return ISING_OK;
  if (static_cast<long long>(m) * B > 0x7FFFFFFFLL) return ISING_ERR_UNSUPPORTED;
  a.spins = const_cast<int8_t*>(spins);   // read only in this mode
  a.out = out;
  a.shift = shift % B;
  a.accepted = accepted;
  a.accumulate = accumulate;
  return launch_clusters<2>(a, m * B, st);
}

}  // namespace ising

extern "C" int ising_propose_clusters(const ising_problem* const* probs, int32_t m, int8_t* spins, int32_t B,
                                      const float* logits, int32_t* accepted, void* cuda_stream) {
  return ising::propose_clusters_launch(probs, m, spins, B, logits, accepted, 0,
                                        static_cast<cudaStream_t>(cuda_stream));
}

extern "C" int ising_droplet_targets(const ising_problem* p, const int8_t* spins, const int8_t* ref, int32_t B,
                                     uint8_t* targets, void* cuda_stream) {
  ising::ClusterArgs a{};
  const int rc = ising::cluster_check<1>(&p, 1, B, &a);
  if (rc != ISING_OK) return rc;
  if (B > 0 && (!spins || !ref || !targets)) return ISING_ERR_ARG;
  if (B == 0) return ISING_OK;
  a.spins = const_cast<int8_t*>(spins);   // read only in this mode
  a.ref = ref;
  a.targets = targets;
  return ising::launch_clusters<1>(a, B, static_cast<cudaStream_t>(cuda_stream));
}

extern "C" int ising_transcribe(const ising_problem* const* probs, int32_t m, const int8_t* spins, int8_t* out,
                                int32_t B, int32_t shift, int32_t* accepted, void* cuda_stream) {
  return ising::transcribe_launch(probs, m, spins, out, B, shift, accepted, 0, static_cast<cudaStream_t>(cuda_stream));
}

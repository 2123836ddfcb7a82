// graph.cu -- the annealer on general sparse graphs: any symmetric CSR with
// integer couplings J (|J| <= 127) and integer fields h, i.e. Eq. 2 in full,
// H = -sum_{i<j} J_ij s_i s_j - sum_i h_i s_i (Section II frames the problem
// as general Ising / Max-Cut).
//
// Sweep: the classes of a first-fit colouring (host, index order) in order;
// sites of one class are never adjacent, so a class updates at once, exactly
// as the sequential visit.  Decision stream and start spins as on the torus:
// Philox4x32-10 at counter (i, k, t/4, 0), word t mod 4; start +1 iff bit 31
// of the block at (i, 0xFFFFFFFF, t/4, 0).  A torus given as a graph takes
// the checkerboard colouring and the same trajectory as the torus kernels.
//
// Energy change, bit-sliced over the 32 trials of a word: each neighbour j
// (and the field, as a neighbour fixed at +1) is a term J_e s_i s_j of weight
// |J_e|; with a = the weight of the terms that are positive and
// D = sum |J_e| + |h_i|, flipping i costs dE = 2 (2a - D).  a is counted in
// kP bit planes (weights added at their binary digits).  Trials with
// 2a <= D flip; the others flip iff their draw is below T(dE), read from a
// per-sweep table indexed by dE / 2 = 2a - D.
//
// Layout: one trial group (32 trials) per thread-block cluster of C CTAs.
// Every CTA holds the group's whole spin vector (one word per site) in
// shared memory, updates its share of each colour class and stores every new
// word into all C copies (distributed shared memory); a cluster barrier
// separates the classes.
#include "anneal_core.cuh"

namespace ising {
namespace {

constexpr int kGraphThreads = 512;

// add weight w (1..127) times the mask x into the bit-sliced counter pl
template <int kP>
__device__ __forceinline__ void add_weighted(uint32_t (&pl)[kP], uint32_t x, uint32_t w) {
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    if (q < kP && ((w >> q) & 1u)) {
      uint32_t carry = x;
#pragma unroll
      for (int p = 0; p < kP; ++p) {
        if (p >= q) {
          const uint32_t t = pl[p] & carry;
          pl[p] ^= carry;
          carry = t;
        }
      }
    }
  }
}

// lanes whose counter value is >= the constant A
template <int kP>
__device__ __forceinline__ uint32_t ge_const(const uint32_t (&pl)[kP], uint32_t A) {
  uint32_t gt = 0u, eq = 0xFFFFFFFFu;
#pragma unroll
  for (int p = kP - 1; p >= 0; --p) {
    if ((A >> p) & 1u) {
      eq &= pl[p];
    } else {
      gt |= eq & pl[p];
      eq &= ~pl[p];
    }
  }
  return gt | eq;
}

template <int kP>
__device__ __forceinline__ uint32_t lane_value(const uint32_t (&pl)[kP], int t) {
  uint32_t v = 0;
#pragma unroll
  for (int p = 0; p < kP; ++p) v |= ((pl[p] >> t) & 1u) << p;
  return v;
}

// counter values of trials 8g .. 8g+7, one byte each (trials 8g .. 8g+3 in
// .x, 8g+4 .. 8g+7 in .y): byte p of an 8 x 8 bit matrix holds plane p's bits
// of the eight trials; transposing it (three delta swaps, Hacker's Delight
// 7-3) leaves trial j's value in byte j
template <int kP>
__device__ __forceinline__ uint2 group_values(const uint32_t (&pl)[kP], int g) {
  const uint32_t sel = static_cast<uint32_t>(g) | (static_cast<uint32_t>(g + 4) << 4);
  auto plane = [&](int p) { return p < kP ? pl[p < kP ? p : 0] : 0u; };
  const uint32_t lo = __byte_perm(__byte_perm(plane(0), plane(1), sel), __byte_perm(plane(2), plane(3), sel), 0x5410);
  const uint32_t hi = kP > 4 ? __byte_perm(__byte_perm(plane(4), plane(5), sel), __byte_perm(plane(6), plane(7), sel),
                                           0x5410)
                             : 0u;
  uint64_t x = (static_cast<uint64_t>(hi) << 32) | lo;
  uint64_t t = (x ^ (x >> 7)) & 0x00AA00AA00AA00AAull;
  x = x ^ t ^ (t << 7);
  t = (x ^ (x >> 14)) & 0x0000CCCC0000CCCCull;
  x = x ^ t ^ (t << 14);
  t = (x ^ (x >> 28)) & 0x00000000F0F0F0F0ull;
  x = x ^ t ^ (t << 28);
  return make_uint2(static_cast<uint32_t>(x), static_cast<uint32_t>(x >> 32));
}

// the decisions of the uphill trials of quad jq (bits of m4): trial t's
// value v = a from its byte of vq, dE / 2 = 2v - D indexes the threshold row
__device__ __forceinline__ uint32_t quad_accepts(const uint4 u, uint32_t m4, uint32_t vq, uint32_t D,
                                                 const uint32_t* thr, int jq) {
  const uint32_t uu[4] = {u.x, u.y, u.z, u.w};
  uint32_t acc = 0u;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    if ((m4 >> m) & 1u) {
      const uint32_t q = 2u * ((vq >> (8 * m)) & 0xFFu) - D;   // dE / 2, 1 .. D
      if (uu[m] < thr[q]) acc |= 1u << (4 * jq + m);
    }
  }
  return acc;
}

template <int kP>
__device__ __forceinline__ uint32_t graph_update(const GraphArgs& a, const uint32_t* sp, const uint32_t* thr,
                                                 const uint4* heads, uint32_t i, int nq) {
  const uint32_t b = sp[i];
  const int4 ri = __ldg(a.rowinfo + i);        // {first entry, degree, h, D}
  uint32_t pl[kP];
#pragma unroll
  for (int p = 0; p < kP; ++p) pl[p] = 0u;
  for (int e = 0; e < ri.y; ++e) {
    const uint32_t v = __ldg(a.nb + ri.x + e);
    const uint32_t j = v & 0xFFFFFFu;
    const uint32_t neg = 0u - ((v >> 24) & 1u);
    add_weighted<kP>(pl, ~(b ^ sp[j]) ^ neg, (v >> 25) + 1u);
  }
  if (ri.z != 0) add_weighted<kP>(pl, ri.z > 0 ? b : ~b, static_cast<uint32_t>(ri.z > 0 ? ri.z : -ri.z));
  const uint32_t D = static_cast<uint32_t>(ri.w);
  const uint32_t up = ge_const<kP>(pl, D / 2 + 1);   // 2a > D: uphill
  uint32_t flip = ~up;
  if (up) {
    // Philox4x32-10 at (i, k, q0 + jq, 0): the site's products of rounds 1-2
    // here, the (sweep, block) part from the per-sweep heads
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo(kPhiloxM0, i, hi0, lo0);
    mulhilo(kPhiloxM1, hi0 ^ a.rk[1], hi1, lo1);
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      if (2 * g >= nq) break;
      if (!((up >> (8 * g)) & 0xFFu)) continue;
      const uint2 v = group_values<kP>(pl, g);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int jq = 2 * g + h;
        const uint32_t m4 = (up >> (4 * jq)) & 0xFu;
        if (jq >= nq || !m4) continue;
        const uint4 hd = heads[jq];
        const uint4 u = philox_rounds_3_to_10(hi1 ^ hd.x, lo1, hd.y ^ lo0, hd.z, a.rk);
        flip |= quad_accepts(u, m4, h ? v.y : v.x, D, thr, jq);
      }
    }
  }
  return b ^ flip;
}

// graph_update split over a team of kTPW consecutive lanes: lane r of the
// team counts the neighbours e = r, r + kTPW, ... into its own bit-sliced
// counter, the team adds the counters up (butterfly over xor shuffles; every
// partial sum is at most the total, so kP planes hold it), and lane r draws
// the decision blocks jq = r, r + kTPW, ...; the accepted trials are OR-ed
// back together.  The decisions are those of graph_update.  Every lane of
// the warp must call it (inactive teams with active = false).
template <int kP, int kTPW>
__device__ __forceinline__ uint32_t graph_update_team(const GraphArgs& a, const uint32_t* sp, const uint32_t* thr,
                                                      const uint4* heads, uint32_t i, int nq, int r, bool active) {
  uint32_t b = 0u;
  int4 ri = make_int4(0, 0, 0, 0);
  if (active) {
    b = sp[i];
    ri = __ldg(a.rowinfo + i);
  }
  uint32_t pl[kP];
#pragma unroll
  for (int p = 0; p < kP; ++p) pl[p] = 0u;
  for (int e = r; e < ri.y; e += kTPW) {
    const uint32_t v = __ldg(a.nb + ri.x + e);
    const uint32_t j = v & 0xFFFFFFu;
    const uint32_t neg = 0u - ((v >> 24) & 1u);
    add_weighted<kP>(pl, ~(b ^ sp[j]) ^ neg, (v >> 25) + 1u);
  }
  if (r == 0 && ri.z != 0) add_weighted<kP>(pl, ri.z > 0 ? b : ~b, static_cast<uint32_t>(ri.z > 0 ? ri.z : -ri.z));
#pragma unroll
  for (int off = 1; off < kTPW; off <<= 1) {
    uint32_t carry = 0u;
#pragma unroll
    for (int p = 0; p < kP; ++p) {
      const uint32_t o = __shfl_xor_sync(0xFFFFFFFFu, pl[p], off);
      const uint32_t x = pl[p] ^ o;               // full adder, bit-sliced
      const uint32_t c_out = (pl[p] & o) | (carry & x);
      pl[p] = x ^ carry;
      carry = c_out;
    }
  }
  const uint32_t D = static_cast<uint32_t>(ri.w);
  const uint32_t up = ge_const<kP>(pl, D / 2 + 1);   // 2a > D: uphill
  uint32_t acc = 0u;
  uint32_t hi0 = 0u, lo0 = 0u, hi1 = 0u, lo1 = 0u;
  if (up) {
    mulhilo(kPhiloxM0, i, hi0, lo0);
    mulhilo(kPhiloxM1, hi0 ^ a.rk[1], hi1, lo1);
  }
#pragma unroll
  for (int s = 0; s < 8 / kTPW; ++s) {
    const int jq = r + s * kTPW;
    const uint32_t m4 = (up >> (4 * jq)) & 0xFu;
    if (jq >= nq || !m4) continue;
    const uint2 v = group_values<kP>(pl, jq >> 1);
    const uint4 hd = heads[jq];
    const uint4 u = philox_rounds_3_to_10(hi1 ^ hd.x, lo1, hd.y ^ lo0, hd.z, a.rk);
    acc |= quad_accepts(u, m4, (jq & 1) ? v.y : v.x, D, thr, jq);
  }
#pragma unroll
  for (int off = 1; off < kTPW; off <<= 1) acc |= __shfl_xor_sync(0xFFFFFFFFu, acc, off);
  return b ^ (~up | acc);
}

template <bool kCluster, int kP, int kTPW>
__global__ void __launch_bounds__(kGraphThreads, 1) graph_anneal_kernel(const __grid_constant__ GraphArgs a) {
  extern __shared__ __align__(16) uint32_t gsm[];
  uint32_t* sp = gsm;                       // [n] spin words of the group
  uint32_t* thr = gsm + a.n_pad;            // [Dmax + 1]: thr[q] = T(dE = 2q) of the current sweep
  uint32_t* part = thr + a.thr_pad;         // [32] cut partial sums (mod 2^32)
  uint4* heads = reinterpret_cast<uint4*>(part + 32);   // [8] Philox heads of the current sweep
  const int C = kCluster ? a.C : 1;
  const uint32_t rank = kCluster ? cluster_ctarank() : 0u;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int g = blockIdx.y;
  const int t0 = g * 32;
  const int live = min(32, a.T - t0);
  const int nq = (live + 3) >> 2;
  const uint32_t q0 = static_cast<uint32_t>(t0) >> 2;
  const int n = a.n;

  if (tid < 32) part[tid] = 0u;
  for (int i = tid; i < n; i += nt) {
    uint32_t w = 0;
    if (a.init) {
      for (int b = 0; b < live; ++b) w |= static_cast<uint32_t>(a.init[static_cast<size_t>(t0 + b) * n + i] > 0) << b;
    } else {
      for (int jq = 0; jq < nq; ++jq) {
        const uint4 u = philox4x32_10(static_cast<uint32_t>(i), 0xFFFFFFFFu, q0 + jq, 0u, a.key0, a.key1);
        w |= ((u.x >> 31) | ((u.y >> 31) << 1) | ((u.z >> 31) << 2) | ((u.w >> 31) << 3)) << (4 * jq);
      }
    }
    sp[i] = w;
  }
  if constexpr (kCluster) cluster_barrier();
  else __syncthreads();

  for (int kk = 0; kk < a.S; ++kk) {
    const uint32_t k = a.k0 + static_cast<uint32_t>(kk);
    for (int q = tid; q < a.Dmax; q += nt) thr[q + 1] = __ldg(a.thr + static_cast<size_t>(kk) * a.Dmax + q);
    if (tid < nq) heads[tid] = philox_head_sweep_quad(k, q0 + tid, a.key0, a.key1);
    __syncthreads();
    for (int c = 0; c < a.ncol; ++c) {
      const int beg = __ldg(a.colour_off + c), len = __ldg(a.colour_off + c + 1) - beg;
      const int my0 = beg + static_cast<int>((static_cast<long long>(len) * rank) / C);
      const int my1 = beg + static_cast<int>((static_cast<long long>(len) * (rank + 1)) / C);
      if constexpr (kTPW == 1) {
        for (int idx = my0 + tid; idx < my1; idx += nt) {
          const uint32_t i = static_cast<uint32_t>(__ldg(a.sites + idx));
          const uint32_t w = graph_update<kP>(a, sp, thr, heads, i, nq);
          sp[i] = w;
          if constexpr (kCluster) {
            const uint32_t addr = smem_addr(sp + i);
            for (int r = 0; r < C; ++r)
              if (r != static_cast<int>(rank)) st_cluster_u32(addr, static_cast<uint32_t>(r), w);
          }
        }
      } else {
        // teams of kTPW lanes per site word; the loop is warp-uniform so that
        // every lane takes part in the team shuffles
        constexpr int kWpw = 32 / kTPW;   // site words per warp and pass
        const int lane = tid & 31, r = lane % kTPW;
        for (int base = (tid >> 5) * kWpw; base < my1 - my0; base += (nt >> 5) * kWpw) {
          const int wi = base + lane / kTPW;
          const bool act = wi < my1 - my0;
          const uint32_t i = act ? static_cast<uint32_t>(__ldg(a.sites + my0 + wi)) : 0u;
          const uint32_t w = graph_update_team<kP, kTPW>(a, sp, thr, heads, i, nq, r, act);
          if (act) {
            if (r == 0) sp[i] = w;
            if constexpr (kCluster) {
              const uint32_t addr = smem_addr(sp + i);
              for (int rr = r; rr < C; rr += kTPW)
                if (rr != static_cast<int>(rank)) st_cluster_u32(addr, static_cast<uint32_t>(rr), w);
            }
          }
        }
      }
      if constexpr (kCluster) cluster_barrier();
      else __syncthreads();
    }
  }

  // ---- read-out: spins of this CTA's share of the sites, and the Eq. 1 cut
  // (w = -J) of the edges whose lower end is in that share
  const int s0 = static_cast<int>((static_cast<long long>(n) * rank) / C);
  const int s1 = static_cast<int>((static_cast<long long>(n) * (rank + 1)) / C);
  const uint32_t live_mask = live == 32 ? 0xFFFFFFFFu : ((1u << live) - 1u);
  for (int i = s0 + tid; i < s1; i += nt) {
    const uint32_t w = sp[i];
    if (a.out_spins)
      for (int b = 0; b < live; ++b) a.out_spins[static_cast<size_t>(t0 + b) * n + i] = ((w >> b) & 1u) ? 1 : -1;
    if (a.out_cuts) {
      const int4 ri = __ldg(a.rowinfo + i);
      for (int e = 0; e < ri.y; ++e) {
        const uint32_t v = __ldg(a.nb + ri.x + e);
        const uint32_t j = v & 0xFFFFFFu;
        if (j <= static_cast<uint32_t>(i)) continue;
        const int32_t wt = ((v >> 24) & 1u) ? static_cast<int32_t>((v >> 25) + 1u)     // J < 0: w = |J|
                                            : -static_cast<int32_t>((v >> 25) + 1u);   // J > 0: w = -|J|
        uint32_t x = (w ^ sp[j]) & live_mask;
        while (x) {
          const int t = __ffs(x) - 1;
          atomicAdd(part + t, static_cast<uint32_t>(wt));
          x &= x - 1u;
        }
      }
    }
  }
  if (a.out_cuts) {
    __syncthreads();
    if constexpr (kCluster) {
      if (rank != 0 && tid < 32) red_add_cluster_u32(smem_addr(part + tid), 0u, part[tid]);
      cluster_barrier();
    }
    if (rank == 0 && tid < live) a.out_cuts[t0 + tid] = static_cast<int32_t>(part[tid]);
  }
  if constexpr (kCluster) cluster_barrier();   // no CTA leaves while a peer may still write to it
}

// Eq. 1 cut and Eq. 2 energy (with fields) of int8 configurations: one CTA
// per configuration.
__global__ void graph_measure_kernel(const GraphArgs a, const int8_t* __restrict__ spins, int32_t* __restrict__ cuts,
                                     long long* __restrict__ energies) {
  __shared__ long long red_c[32], red_e[32];
  const int8_t* s = spins + static_cast<size_t>(blockIdx.x) * a.n;
  long long cut = 0, en = 0;
  for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
    const int si = s[i] > 0 ? 1 : -1;
    const int4 ri = __ldg(a.rowinfo + i);
    for (int e = 0; e < ri.y; ++e) {
      const uint32_t v = __ldg(a.nb + ri.x + e);
      const int j = static_cast<int>(v & 0xFFFFFFu);
      if (j <= i) continue;
      const int Jv = ((v >> 24) & 1u) ? -static_cast<int>((v >> 25) + 1u) : static_cast<int>((v >> 25) + 1u);
      const int sj = s[j] > 0 ? 1 : -1;
      en -= static_cast<long long>(Jv) * si * sj;
      if (si != sj) cut -= Jv;
    }
    en -= static_cast<long long>(ri.z) * si;
  }
  for (int o = 16; o > 0; o >>= 1) {
    cut += __shfl_xor_sync(0xFFFFFFFFu, cut, o);
    en += __shfl_xor_sync(0xFFFFFFFFu, en, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red_c[threadIdx.x >> 5] = cut;
    red_e[threadIdx.x >> 5] = en;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long tc = 0, te = 0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) {
      tc += red_c[w];
      te += red_e[w];
    }
    if (cuts) cuts[blockIdx.x] = static_cast<int32_t>(tc);
    if (energies) energies[blockIdx.x] = te;
  }
}

template <int kP, int kTPW>
cudaError_t launch_graph_pt(const GraphArgs& a, cudaStream_t st) {
  const size_t smem = graph_smem_bytes(a.n, a.Dmax);
  const int groups = (a.T + 31) / 32;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.C, groups, 1);
  cfg.blockDim = dim3(kGraphThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  cudaError_t e;
  if (a.C > 1) {
    e = cudaFuncSetAttribute(graph_anneal_kernel<true, kP, kTPW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = a.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, graph_anneal_kernel<true, kP, kTPW>, a);
  }
  e = cudaFuncSetAttribute(graph_anneal_kernel<false, kP, kTPW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  return cudaLaunchKernelEx(&cfg, graph_anneal_kernel<false, kP, kTPW>, a);
}

template <int kP>
cudaError_t launch_graph_p(const GraphArgs& a, cudaStream_t st) {
  switch (a.tpw) {
    case 8: return launch_graph_pt<kP, 8>(a, st);
    case 4: return launch_graph_pt<kP, 4>(a, st);
    default: return launch_graph_pt<kP, 1>(a, st);
  }
}

}  // namespace

size_t graph_smem_bytes(int32_t n, int32_t Dmax) {
  const size_t n_pad = (static_cast<size_t>(n) + 3) & ~size_t(3);
  const size_t thr_pad = (static_cast<size_t>(Dmax) + 1 + 3) & ~size_t(3);
  return (n_pad + thr_pad + 32) * sizeof(uint32_t) + 8 * sizeof(uint4);
}

int graph_threads() { return kGraphThreads; }

// planes: enough bits for every counter value 0 .. Dmax
cudaError_t launch_graph(const GraphArgs& a, cudaStream_t st) {
  switch (a.planes) {
    case 1:
    case 2:
    case 3: return launch_graph_p<3>(a, st);
    case 4: return launch_graph_p<4>(a, st);
    case 5: return launch_graph_p<5>(a, st);
    case 6: return launch_graph_p<6>(a, st);
    case 7: return launch_graph_p<7>(a, st);
    default: return launch_graph_p<8>(a, st);
  }
}

cudaError_t launch_graph_measure(const GraphArgs& a, const int8_t* spins, int32_t k, int32_t* cuts,
                                 long long* energies, cudaStream_t st) {
  if (k <= 0) return cudaSuccess;
  graph_measure_kernel<<<k, 256, 0, st>>>(a, spins, cuts, energies);
  return cudaGetLastError();
}

namespace {
__global__ void energy_from_cut_kernel(const int32_t* __restrict__ cuts, int32_t W, int32_t k,
                                       int64_t* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < k) out[t] = static_cast<int64_t>(W) - 2 * static_cast<int64_t>(cuts[t]);
}
}  // namespace

cudaError_t launch_energy_from_cut(const int32_t* cuts, int32_t W, int32_t k, int64_t* out, cudaStream_t st) {
  if (k <= 0) return cudaSuccess;
  energy_from_cut_kernel<<<(k + 255) / 256, 256, 0, st>>>(cuts, W, k, out);
  return cudaGetLastError();
}

}  // namespace ising

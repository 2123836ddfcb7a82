// anneal_core.cuh -- the per-trial-group annealing body shared by the strip
// kernel (anneal.cu) and the persistent batched kernel (batched.cu).
//
// Method (Zick 2025, Section III: independent trials of sweeps, read out at
// the end of each trial; Eq. 1 and Eq. 2 with J = -w, h = 0).  The sweep is a
// Metropolis sweep over the two checkerboard colours.  The torus has even
// sides, so it is bipartite: all sites of one colour are updated at once, which
// equals visiting them one by one.
//
// Layout (per trial group of G <= 32 trials, bit b of a word = trial t0 + b):
//   spin word  sp[c][lr][h]   colour plane c, local row lr (0 and rows+1 are
//                              halo rows), h = x / 2; the site of colour c in
//                              global row y sits at x = 2h + ((y + c) & 1).
//   bit = 1 <=> spin +1.
// With e_j = NOT(s_i XOR s_j XOR neg_ij) marking a +1 energy term w_ij s_i s_j,
// the count m = e_L + e_R + e_U + e_D gives dE = 8 - 4m.  m >= 2: flip;
// m = 1: flip iff u < T4; m = 0: flip iff u < T8.  The counts are bit-sliced
// over the 32 trials of a word; the draws u come from Philox4x32-10 at
// counter (i, k, t / 4, 0), word t mod 4.  In the 16-bit draw mode (kU16)
// one block serves eight trials: counter (i, k, t / 8, 0), the low (t even)
// or high (t odd) half of word (t mod 8) / 2, against 16-bit thresholds that
// the host stores shifted left by 16 bits.
//
// Philox sharing: in round 1 the site index i only meets multiplier M0 and the
// quad index q only meets M1, and in round 2 the product M1 * c2 involves
// only the site-dependent word.  So the site-dependent products of rounds 1
// and 2 are computed once per site word and shared by all quads, and the
// (sweep, quad)-dependent products once per sweep and quad (in shared
// memory).  Rounds 3..10 run per quad.  The outputs are exactly those of
// Philox4x32-10.
//
// Strips: with C > 1 the rows of a group are split over the C CTAs of a
// thread-block cluster.  Half-sweep c writes only colour-c words and reads
// only colour-(1-c) words, so a boundary row pushed into a neighbour's halo
// (colour c) never races with that neighbour's reads (colour 1-c).  Each
// half-sweep updates the two boundary rows first, pushes them, arrives on the
// cluster barrier, updates the interior rows (which read no halo) and only
// then waits, so the barrier latency hides behind the interior work.
#pragma once
#include "device_common.cuh"
#include "internal.h"

namespace ising {

struct GroupJob {
  const uint8_t* flags;     // plane-order site flags [n]
  const uint32_t* thr;      // [2*S]: (T4, T8) of each sweep of the call
  const int8_t* init;       // [T][n] or null
  int8_t* out_spins;        // [T][n] or null
  int32_t* out_cuts;        // [T] or null
  int32_t X, Y, H, n;
  int32_t T, G, S;
  uint32_t k0;
  uint32_t key0, key1;
  const uint32_t* rk;       // 20 round keys (see philox_rounds_3_to_10)
  int32_t C, Rmax;
  int32_t neg_edges;
};

__device__ __forceinline__ int strip_rows(int Y, int C, int r) { return Y / C + (r < Y % C ? 1 : 0); }
__device__ __forceinline__ int strip_y0(int Y, int C, int r) { return r * (Y / C) + min(r, Y % C); }

// acc * 2 + (u >= T).  After sub.cc the carry flag is the carry-out of
// u + ~T + 1, i.e. 1 when u >= T (no borrow); addc shifts it in.  The
// caller accumulates "reject" bits and inverts them.
__device__ __forceinline__ uint32_t shift_in_ge(uint32_t acc, uint32_t u, uint32_t T) {
  uint32_t r;
  asm("{\n\t.reg .u32 t;\n\tsub.cc.u32 t, %1, %2;\n\taddc.u32 %0, %3, %3;\n\t}"
      : "=r"(r)
      : "r"(u), "r"(T), "r"(acc));
  return r;
}

// 32x32 -> 64-bit product as (hi, lo)
__device__ __forceinline__ void mulhilo(uint32_t m, uint32_t a, uint32_t& hi, uint32_t& lo) {
  uint64_t p;
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(a), "r"(m));
  lo = static_cast<uint32_t>(p);
  hi = static_cast<uint32_t>(p >> 32);
}

// Philox4x32-10 rounds 3..10 from the state after round 2.  rk holds the
// round keys: rk[2r] = key0 + r*W0, rk[2r+1] = key1 + r*W1 (r = 0..9).
__device__ __forceinline__ uint4 philox_rounds_3_to_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                       const uint32_t* __restrict__ rk) {
#pragma unroll
  for (int r = 2; r < 10; ++r) {
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo(kPhiloxM0, c0, hi0, lo0);
    mulhilo(kPhiloxM1, c2, hi1, lo1);
    const uint32_t n0 = hi1 ^ c1 ^ rk[2 * r];
    const uint32_t n2 = hi0 ^ c3 ^ rk[2 * r + 1];
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return make_uint4(c0, c1, c2, c3);
}

// (sweep k, quad q) part of rounds 1-2: returns {A, B, C, 0} such that the
// state after round 2 for site i is (hi(M1*c2') ^ A, lo(M1*c2'), B ^ lo(M0*i), C)
// with c2' = hi(M0*i) ^ key1.
__device__ __forceinline__ uint4 philox_head_sweep_quad(uint32_t k, uint32_t q, uint32_t key0, uint32_t key1) {
  uint32_t H1, L1, H2, L2;
  mulhilo(kPhiloxM1, q, H1, L1);
  const uint32_t U1 = H1 ^ k ^ key0;  // word 0 after round 1
  mulhilo(kPhiloxM0, U1, H2, L2);
  return make_uint4(L1 ^ (key0 + kPhiloxW0), H2 ^ (key1 + kPhiloxW1), L2, 0u);
}

struct CoreSmem {
  uint32_t* sp;          // [2][L][H] spin words
  unsigned char* fl;     // [2][Rmax][H] site flags of the own rows
  uint4* head;           // [2][8] per-sweep Philox heads (double buffered)
  int32_t* part;         // [32] per-trial cut partial sums
};

// Shared-memory carve; every section starts on a 16-byte boundary (the
// Philox heads are read as uint4).
__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }
__host__ __device__ inline size_t core_off_fl(int32_t H, int32_t Rmax) {
  return align16(2 * (static_cast<size_t>(Rmax) + 2) * H * 4);
}
__host__ __device__ inline size_t core_off_head(int32_t H, int32_t Rmax) {
  return core_off_fl(H, Rmax) + align16(2 * static_cast<size_t>(Rmax) * H);
}
__host__ __device__ inline size_t core_smem_bytes(int32_t H, int32_t Rmax) {
  return core_off_head(H, Rmax) + 2 * 8 * sizeof(uint4) + 32 * 4;
}

__device__ __forceinline__ CoreSmem carve(unsigned char* smem, int32_t H, int32_t Rmax) {
  CoreSmem s;
  s.sp = reinterpret_cast<uint32_t*>(smem);
  s.fl = smem + core_off_fl(H, Rmax);
  s.head = reinterpret_cast<uint4*>(smem + core_off_head(H, Rmax));
  s.part = reinterpret_cast<int32_t*>(s.head + 16);
  return s;
}

template <bool kCluster>
__device__ __forceinline__ void cluster_arrive() {
  if constexpr (kCluster) asm volatile("barrier.cluster.arrive.release;\n" ::: "memory");
}
template <bool kCluster>
__device__ __forceinline__ void cluster_wait() {
  if constexpr (kCluster) asm volatile("barrier.cluster.wait.acquire;\n" ::: "memory");
}


// one Philox block (rounds 3..10) for one quad of trials, its four draws
// compared against both thresholds and shifted into the reject masks
__device__ __forceinline__ void quad_step(uint32_t& rej4, uint32_t& rej8, const uint4 hd, uint32_t hi1, uint32_t lo1,
                                          uint32_t lo0, uint32_t T4, uint32_t T8, const uint32_t* __restrict__ rk) {
  const uint4 u = philox_rounds_3_to_10(hi1 ^ hd.x, lo1, hd.y ^ lo0, hd.z, rk);
  rej4 = shift_in_ge(rej4, u.w, T4);
  rej4 = shift_in_ge(rej4, u.z, T4);
  rej4 = shift_in_ge(rej4, u.y, T4);
  rej4 = shift_in_ge(rej4, u.x, T4);
  rej8 = shift_in_ge(rej8, u.w, T8);
  rej8 = shift_in_ge(rej8, u.z, T8);
  rej8 = shift_in_ge(rej8, u.y, T8);
  rej8 = shift_in_ge(rej8, u.x, T8);
}

// 16-bit draw mode: one Philox block for eight trials.  With thresholds
// stored as T << 16, w >= T << 16 tests the high half and (w << 16) >= T << 16
// the low half.  Trials 8j + 7 .. 8j are shifted in from the top: word w high,
// word w low, ..., word x low.
__device__ __forceinline__ void octet_step(uint32_t& rej4, uint32_t& rej8, const uint4 hd, uint32_t hi1, uint32_t lo1,
                                           uint32_t lo0, uint32_t T4, uint32_t T8, const uint32_t* __restrict__ rk) {
  const uint4 u = philox_rounds_3_to_10(hi1 ^ hd.x, lo1, hd.y ^ lo0, hd.z, rk);
  const uint32_t w[4] = {u.w, u.z, u.y, u.x};
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    rej4 = shift_in_ge(rej4, w[m], T4);
    rej4 = shift_in_ge(rej4, w[m] << 16, T4);
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    rej8 = shift_in_ge(rej8, w[m], T8);
    rej8 = shift_in_ge(rej8, w[m] << 16, T8);
  }
}

// Philox blocks per trial group of `live` trials, and the block index of the
// group's first trial t0
template <bool kU16>
__host__ __device__ __forceinline__ int decision_blocks(int live) { return kU16 ? (live + 7) >> 3 : (live + 3) >> 2; }
template <bool kU16>
__host__ __device__ __forceinline__ uint32_t decision_block0(int t0) {
  return kU16 ? static_cast<uint32_t>(t0) >> 3 : static_cast<uint32_t>(t0) >> 2;
}

// Where the per-sweep Philox heads of a word's decision blocks are read:
// through a pointer, or from a 32-bit shared-memory address.
struct HeadsAt {
  const uint4* p;
  __device__ __forceinline__ uint4 operator()(int j) const { return p[j]; }
};
struct HeadsShared {
  uint32_t addr;
  __device__ __forceinline__ uint4 operator()(int j) const {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(addr + 16u * static_cast<uint32_t>(j)));
    return v;
  }
};

// Metropolis update of one site word; returns the new word.  mL..mD: all
// ones where the edge to the left / right / upper / lower neighbour has
// w = -1, else zero.  nq: Philox blocks of the group (decision_blocks);
// heads(j): the head of block j.
template <bool kU16, class Heads>
__device__ __forceinline__ uint32_t update_word_m(uint32_t s, uint32_t nl, uint32_t nr, uint32_t nu, uint32_t nd,
                                                 uint32_t mL, uint32_t mR, uint32_t mU, uint32_t mD, uint32_t i,
                                                 const Heads& heads, int nq, uint32_t T4, uint32_t T8,
                                                 const uint32_t* __restrict__ rk) {
  // per trial: eX set where the edge to neighbour X is unsatisfied
  // (w s s' = +1, it adds to the energy); ge2: two or more (dE <= 0, always
  // flip), any: at least one (dE = 4 when not ge2, else dE = 8)
  const uint32_t eL = ~(s ^ nl ^ mL), eR = ~(s ^ nr ^ mR);
  const uint32_t eU = ~(s ^ nu ^ mU), eD = ~(s ^ nd ^ mD);
  const uint32_t abc = eL | eR | eU;
  const uint32_t any = abc | eD;
  const uint32_t ge2 = (eL & eR) | (eU & (eL | eR)) | (eD & abc);
  // site-dependent products of rounds 1 and 2
  uint32_t hi0, lo0, hi1, lo1;
  mulhilo(kPhiloxM0, i, hi0, lo0);
  mulhilo(kPhiloxM1, hi0 ^ rk[1], hi1, lo1);
  uint32_t rej4 = 0, rej8 = 0;   // bit set: draw at or above the threshold
  if constexpr (kU16) {
    if (nq == 4) {
#pragma unroll
      for (int j = 3; j >= 0; --j) octet_step(rej4, rej8, heads(j), hi1, lo1, lo0, T4, T8, rk);
    } else {
      for (int j = nq - 1; j >= 0; --j) octet_step(rej4, rej8, heads(j), hi1, lo1, lo0, T4, T8, rk);
    }
  } else {
    if (nq == 8) {  // full groups: unrolled, so consecutive blocks can overlap
#pragma unroll
      for (int j = 7; j >= 0; --j) quad_step(rej4, rej8, heads(j), hi1, lo1, lo0, T4, T8, rk);
    } else {
      for (int j = nq - 1; j >= 0; --j) quad_step(rej4, rej8, heads(j), hi1, lo1, lo0, T4, T8, rk);
    }
  }
  // ge2 trials flip whatever their draws; the others by their class's compare
  return s ^ (ge2 | (any & ~rej4) | (~any & ~rej8));
}

// The same with the edge signs as the flag byte f (bit 0: left edge has
// w = -1, bit 1 right, bit 2 up, bit 3 down).
template <bool kU16, class Heads>
__device__ __forceinline__ uint32_t update_word_h(uint32_t s, uint32_t nl, uint32_t nr, uint32_t nu, uint32_t nd,
                                                 uint32_t f, uint32_t i, const Heads& heads, int nq,
                                                 uint32_t T4, uint32_t T8, const uint32_t* __restrict__ rk) {
  return update_word_m<kU16>(s, nl, nr, nu, nd, 0u - (f & 1u), 0u - ((f >> 1) & 1u), 0u - ((f >> 2) & 1u),
                             0u - ((f >> 3) & 1u), i, heads, nq, T4, T8, rk);
}

// All ones if byte b of x has its top bit set, else zero (prmt with sign
// replication of one byte into all four)
template <int b>
__device__ __forceinline__ uint32_t byte_sign_mask(uint32_t x) {
  uint32_t r;
  asm("prmt.b32 %0, %1, 0, %2;" : "=r"(r) : "r"(x), "n"((8 + b) * 0x1111));
  return r;
}

template <bool kU16>
__device__ __forceinline__ uint32_t update_word(uint32_t s, uint32_t nl, uint32_t nr, uint32_t nu, uint32_t nd,
                                               uint32_t f, uint32_t i, const uint4* head, int nq,
                                               uint32_t T4, uint32_t T8, const uint32_t* __restrict__ rk) {
  return update_word_h<kU16>(s, nl, nr, nu, nd, f, i, HeadsAt{head}, nq, T4, T8, rk);
}

// Anneal trial group g (strip r of C) of job a.  All threads of the CTA (and
// of the cluster when kCluster) must call it.  Ends with the CTA (cluster)
// synchronised; shared memory may be reused after it returns.
template <bool kCluster, bool kU16>
__device__ __forceinline__ void anneal_group(const GroupJob& a, const int g, const int r, unsigned char* smem) {
  const int C = a.C;
  const int rows = strip_rows(a.Y, C, r);
  const int y0 = strip_y0(a.Y, C, r);
  const int H = a.H;
  const int L = a.Rmax + 2;
  const CoreSmem sm = carve(smem, H, a.Rmax);
  uint32_t* sp = sm.sp;
  unsigned char* fl = sm.fl;

  const int t0 = g * a.G;
  const int live = min(a.G, a.T - t0);
  const int nq = decision_blocks<kU16>(live);       // Philox blocks per site word and sweep
  const uint32_t q0 = decision_block0<kU16>(t0);
  const int nqi = (live + 3) >> 2;                  // the starting spins use 32-bit quads
  const uint32_t qi0 = static_cast<uint32_t>(t0) >> 2;
  const int tid = threadIdx.x, nt = blockDim.x;

  if (tid < 32) sm.part[tid] = 0;
  if (tid < nq && a.S > 0) sm.head[tid] = philox_head_sweep_quad(a.k0, q0 + tid, a.key0, a.key1);

  for (int idx = tid; idx < 2 * rows * H; idx += nt) {
    const int c = idx / (rows * H);
    const int rem = idx - c * rows * H;
    const int lr0 = rem / H;
    const int h = rem - lr0 * H;
    fl[(c * a.Rmax + lr0) * H + h] = a.flags[(static_cast<size_t>(c) * a.Y + y0 + lr0) * H + h];
  }
  // starting spins of the own rows and both halo rows (counter-based, so a
  // halo row is initialised here to the same value its owner computes)
  for (int idx = tid; idx < 2 * (rows + 2) * H; idx += nt) {
    const int c = idx / ((rows + 2) * H);
    const int rem = idx - c * (rows + 2) * H;
    const int lr = rem / H;
    const int h = rem - lr * H;
    int y = y0 - 1 + lr;
    if (y < 0) y += a.Y;
    if (y >= a.Y) y -= a.Y;
    const uint32_t i = static_cast<uint32_t>(y * a.X + 2 * h + ((y + c) & 1));
    uint32_t w = 0;
    if (a.init) {
      for (int b = 0; b < live; ++b)
        w |= static_cast<uint32_t>(a.init[static_cast<size_t>(t0 + b) * a.n + i] > 0) << b;
    } else {
      for (int j = 0; j < nqi; ++j) {
        const uint4 u = philox4x32_10(i, 0xFFFFFFFFu, qi0 + j, 0u, a.key0, a.key1);
        w |= ((u.x >> 31) | ((u.y >> 31) << 1) | ((u.z >> 31) << 2) | ((u.w >> 31) << 3)) << (4 * j);
      }
    }
    sp[(c * L + lr) * H + h] = w;
  }
  if constexpr (kCluster) cluster_barrier();
  else __syncthreads();

  const int r_up = (r + C - 1) % C, r_dn = (r + 1) % C;
  const int rows_up = strip_rows(a.Y, C, r_up);
  const int items = rows * H;
  const int nb = (rows < 2 ? rows : 2) * H;  // boundary items: rows 1 and `rows`
  const int dq = nt / H, dr = nt - (nt / H) * H;

  for (int kk = 0; kk < a.S; ++kk) {
    const uint32_t k = a.k0 + static_cast<uint32_t>(kk);
    const uint32_t T4 = __ldg(a.thr + 2 * kk);
    const uint32_t T8 = __ldg(a.thr + 2 * kk + 1);
    const uint4* head = sm.head + 8 * (kk & 1);
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
      uint32_t* self = sp + static_cast<size_t>(c) * L * H;
      const uint32_t* nb_plane = sp + static_cast<size_t>(1 - c) * L * H;
      const unsigned char* fc = fl + static_cast<size_t>(c) * a.Rmax * H;
      // the half-sweep's items in the order: row 1, row `rows`, rows 2..rows-1
      int slot = tid / H, h = tid - (tid / H) * H;
      bool arrived = false;
      for (int it = tid; it < items; it += nt) {
        if (kCluster && !arrived && it >= nb) {
          cluster_arrive<kCluster>();
          arrived = true;
        }
        const int lr = slot == 0 ? 1 : (slot == 1 ? rows : slot);
        const int y = y0 + lr - 1;
        const int par = (y + c) & 1;
        const uint32_t i = static_cast<uint32_t>(y * a.X + 2 * h + par);
        const int row = lr * H;
        const int hl = par ? h : (h == 0 ? H - 1 : h - 1);
        const int hr = par ? (h == H - 1 ? 0 : h + 1) : h;
        const uint32_t ns = update_word<kU16>(self[row + h], nb_plane[row + hl], nb_plane[row + hr],
                                        nb_plane[row - H + h], nb_plane[row + H + h],
                                        fc[(lr - 1) * H + h], i, head, nq, T4, T8, a.rk);
        self[row + h] = ns;
        if (lr == 1) {          // first own row -> bottom halo of the strip above
          if constexpr (kCluster) st_cluster_u32(smem_addr(self + (rows_up + 1) * H + h), r_up, ns);
          else self[(rows + 1) * H + h] = ns;
        }
        if (lr == rows) {       // last own row -> top halo of the strip below
          if constexpr (kCluster) st_cluster_u32(smem_addr(self + h), r_dn, ns);
          else self[h] = ns;
        }
        h += dr;
        slot += dq;
        if (h >= H) { h -= H; ++slot; }
      }
      if (kCluster && !arrived) cluster_arrive<kCluster>();
      // next sweep's Philox heads, computed while this sweep finishes
      if (c == 1 && tid < nq && kk + 1 < a.S)
        sm.head[8 * ((kk + 1) & 1) + tid] = philox_head_sweep_quad(k + 1u, q0 + tid, a.key0, a.key1);
      __syncthreads();
      cluster_wait<kCluster>();
    }
  }

  // ---- read-out: spins of the own rows
  if (a.out_spins) {
    const int span = rows * a.X;
    const size_t gbase = static_cast<size_t>(y0) * a.X;
    for (int idx = tid; idx < live * span; idx += nt) {
      const int b = idx / span;
      const int rem = idx - b * span;
      const int yl = rem / a.X;
      const int x = rem - yl * a.X;
      const int c = (x + y0 + yl) & 1;
      const uint32_t w = sp[(c * L + yl + 1) * H + (x >> 1)];
      a.out_spins[static_cast<size_t>(t0 + b) * a.n + gbase + rem] = ((w >> b) & 1u) ? int8_t(1) : int8_t(-1);
    }
  }
  // ---- exact cut: sum over own right/down edges of w [s_i != s_j], counted
  // per trial as sum(v) - #neg with v = d for w = +1 and NOT d for w = -1
  if (a.out_cuts) {
    const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
    uint32_t acc = 0;
    const int total = 2 * rows * H;
    for (int base = warp * 32; base < total; base += nwarps * 32) {
      const int idx = base + lane;
      uint32_t vr = 0, vd = 0;
      if (idx < total) {
        const int c = idx / (rows * H);
        const int rem = idx - c * rows * H;
        const int lr = 1 + rem / H;
        const int h = rem - (lr - 1) * H;
        const int par = (y0 + lr - 1 + c) & 1;
        const uint32_t s = sp[(c * L + lr) * H + h];
        const uint32_t* nbp = sp + static_cast<size_t>(1 - c) * L * H;
        const int hr = par ? (h == H - 1 ? 0 : h + 1) : h;
        const uint32_t sr = nbp[lr * H + hr];
        const uint32_t sd = nbp[(lr + 1) * H + h];
        const uint32_t f = fl[(c * a.Rmax + lr - 1) * H + h];
        vr = (s ^ sr) ^ (0u - ((f >> 1) & 1u));
        vd = (s ^ sd) ^ (0u - ((f >> 3) & 1u));
      }
#pragma unroll 4
      for (int b = 0; b < 32; ++b) {
        const uint32_t cnt = __popc(__ballot_sync(0xFFFFFFFFu, (vr >> b) & 1u)) +
                             __popc(__ballot_sync(0xFFFFFFFFu, (vd >> b) & 1u));
        if (lane == b) acc += cnt;
      }
    }
    if constexpr (kCluster) red_add_cluster_u32(smem_addr(sm.part + lane), 0u, acc);
    else atomicAdd(reinterpret_cast<unsigned int*>(sm.part + lane), acc);
  }
  if constexpr (kCluster) cluster_barrier();
  else __syncthreads();
  if (a.out_cuts && r == 0 && tid < live) a.out_cuts[t0 + tid] = sm.part[tid] - a.neg_edges;
  __syncthreads();
}

}  // namespace ising

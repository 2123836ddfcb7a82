// anneal_flow.cu -- persistent, barrier-free form of the checkerboard sweep.
//
// The same Metropolis sweep as anneal_core.cuh (Zick 2025, Section III: trials
// of sweeps read out at the end of each trial; Eq. 1, Eq. 2 with J = -w, h = 0),
// organised so that every SM works and no CTA-wide barrier separates the
// half-sweeps:
//
// * Rows of all trial groups are stacked (global row u = g*Y + y), and their
//   site words (u*H + h) are split into one contiguous range per CTA,
//   weighted by the number of Philox quads of each row's group, over exactly
//   one CTA per SM (cooperative launch, so all CTAs are resident together).
//   A range may begin or end inside a row; such a row is shared by two CTAs.
// * Inside a CTA, warps take 32-item chunks of the half-sweeps in one global
//   order (half-sweep major), round robin.  A chunk of colour c only needs the
//   colour-(1-c) words of its rows and of the rows above and below; per-row
//   completion counters in shared memory say when those are final, so a warp
//   waits for exactly its neighbours and never for the whole CTA.
// * Rows that another CTA reads ("published" rows: shared rows and the rows
//   next to a shared or another CTA's row) are also written to a global
//   mirror as tagged words: the word and its half-sweep + 1 in one 8-byte
//   store.  A reader loads the 8 bytes of each word it needs and uses them
//   once the tag is the half-sweep it waits for; no fence and no counter is
//   needed on either side (a writer cannot get a half-sweep ahead of a
//   reader of the same word, since its next update needs the reader's; the
//   readers of a word are its neighbours, and each stored word is computed
//   from the loads before it, so the PTX model's no-thin-air rule excludes a
//   load that sees the writer's next value).
//   Published rows come first in each half-sweep, so their words are usually
//   there long before anyone reads them.
//
// * Fast path: when its records fit in shared memory, every item has two
//   16-byte records with the shared addresses of its word and neighbours,
//   its site index, edge signs and counter offsets, and every chunk a list of
//   the completion counters it waits for (one per lane).  Chunks that touch
//   no mirror row then cost two record loads, one acquire per lane and the
//   word update; the others take the general path, which decodes the row
//   and item tables and reads and writes the mirror.
//
// Every wait is bounded by a cycle limit.  A wait that runs out writes
// ISING_ERR_TIMEOUT to the problem's status word and raises an abort flag that
// ends all other waits at once; the kernel then returns without results.
#include "anneal_core.cuh"

namespace ising {
namespace {

constexpr int kMaxSeg = 4;        // row segments (groups touched) per CTA
constexpr int kFlowThreads = 640;
constexpr int kFlowWarps = kFlowThreads / 32;

struct FlowSmem {
  uint32_t* sp;        // [2][LR][H] spin words (own rows and halo slots), then one spare word
  uint8_t* fl;         // [2][LR][H] site flags (own rows), then one spare byte
  uint32_t* rowcnt;    // [2][LR + 1] completed items per local row and colour
  int32_t* r_u;        // [LR] global row of the local row (own or halo)
  int32_t* r_up;       // [LR] local row above (own row or halo slot)
  int32_t* r_dn;       // [LR] local row below
  int32_t* r_xup;      // [LR] global row above when it belongs to another CTA, else -1
  int32_t* r_xdn;      // [LR] same for the row below
  int32_t* r_pub;      // [LR] 1 if another CTA reads this own row
  int32_t* r_seg;      // [LR] segment of the row
  int32_t* order;      // [LR] own rows in processing order (published rows first)
  int32_t* r_ha;       // [LR] own words of the row: h in [r_ha, r_hb)
  int32_t* r_hb;
  int32_t* r_xself;    // [LR] global row if another CTA owns some of its words, else -1
  int32_t* oitem;      // [LR + 1] first item of the oi-th row of the processing order
  uint4* whead;        // [warps][kMaxSeg][8] per-warp Philox heads
  uint2* wthr;         // [warps][kMaxSeg] per-warp (T4, T8) of each segment's group
  int32_t* meta;       // [8]: nown, nloc, nseg, ...
  int32_t* seg_g;      // [kMaxSeg] group of each segment
  int4* rowc;          // [2][LR + 1][2] per colour and local row: see the table build
  int2* xtab;          // [NC*32] per item: see the table build
  uint4* rec;          // [2][2][cap] per colour and item: the fast path's records (see their build)
  uint32_t* ccnt;      // [2][cap / 32][32] per colour and chunk: the counters the chunk waits for
};

// cap: items (own site words per colour) of the largest CTA, rounded up to
// whole chunks; rec: room for the fast path's item and chunk records
__host__ __device__ inline size_t flow_smem_layout(int32_t LR, int32_t H, int32_t cap, int32_t rec, size_t* off) {
  size_t o = 0;
  off[0] = o; o += align16((static_cast<size_t>(2) * LR * H + 1) * 4);  // sp (+ spare word)
  off[1] = o; o += align16(static_cast<size_t>(2) * LR * H + 1);        // fl (+ spare byte)
  off[2] = o; o += align16(static_cast<size_t>(2) * (LR + 1) * 4);      // rowcnt
  off[3] = o; o += align16(static_cast<size_t>(12) * (LR + 1) * 4);     // row tables (12 arrays)
  off[4] = o; o += static_cast<size_t>(kFlowWarps) * kMaxSeg * (8 * 16 + 8);   // whead, wthr
  off[5] = o; o += 16 * 4;                                               // meta + seg_g
  off[6] = o; o += static_cast<size_t>(2) * (LR + 1) * 2 * 16;          // rowc
  off[7] = o; o += static_cast<size_t>(cap) * 8;                        // xtab
  off[8] = o; o += rec ? static_cast<size_t>(2) * 2 * cap * 16 : 0;     // item records
  off[9] = o; o += rec ? static_cast<size_t>(2) * cap * 4 : 0;          // chunk counter records
  return o;
}

__device__ __forceinline__ FlowSmem flow_carve(unsigned char* smem, int32_t LR, int32_t H, int32_t cap, int32_t rec) {
  size_t off[10];
  flow_smem_layout(LR, H, cap, rec, off);
  FlowSmem s;
  s.sp = reinterpret_cast<uint32_t*>(smem + off[0]);
  s.fl = smem + off[1];
  s.rowcnt = reinterpret_cast<uint32_t*>(smem + off[2]);
  int32_t* t = reinterpret_cast<int32_t*>(smem + off[3]);
  const int L1 = LR + 1;
  s.r_u = t;
  s.r_up = t + L1;
  s.r_dn = t + 2 * L1;
  s.r_xup = t + 3 * L1;
  s.r_xdn = t + 4 * L1;
  s.r_pub = t + 5 * L1;
  s.r_seg = t + 6 * L1;
  s.order = t + 7 * L1;
  s.r_ha = t + 8 * L1;
  s.r_hb = t + 9 * L1;
  s.r_xself = t + 10 * L1;
  s.oitem = t + 11 * L1;
  s.whead = reinterpret_cast<uint4*>(smem + off[4]);
  s.wthr = reinterpret_cast<uint2*>(smem + off[4] + static_cast<size_t>(kFlowWarps) * kMaxSeg * 8 * 16);
  s.meta = reinterpret_cast<int32_t*>(smem + off[5]);
  s.seg_g = s.meta + 8;
  s.rowc = reinterpret_cast<int4*>(smem + off[6]);
  s.xtab = reinterpret_cast<int2*>(smem + off[7]);
  s.rec = reinterpret_cast<uint4*>(smem + off[8]);
  s.ccnt = reinterpret_cast<uint32_t*>(smem + off[9]);
  return s;
}


// acquire / release on the completion counters: a counter read with acquire
// orders the reader's later loads after it, and a release increment orders
// the writer's earlier stores (and, through the warp barrier before it, those
// of the other lanes of its warp) before it
__device__ __forceinline__ uint32_t ld_acquire_cta(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_cta(uint32_t addr, uint32_t v) {
  asm volatile("red.release.cta.shared::cta.add.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// Tagged mirror words: the word in the low half and (half-sweep + 1) in the
// high half, written and read as one 8-byte access (single-copy atomic), so
// a reader that sees the tag it waits for also sees that half-sweep's word;
// no fence is needed on either side.  A writer cannot overwrite a word before
// its readers took it: its next update of that word needs theirs, which need
// this one.
__device__ __forceinline__ unsigned long long ld_tagged(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_tagged(unsigned long long* p, uint32_t word, uint32_t tag) {
  const unsigned long long v = (static_cast<unsigned long long>(tag) << 32) | word;
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t tag_of(unsigned long long v) { return static_cast<uint32_t>(v >> 32); }

// Bounded wait until the shared completion counter at shared address `saddr`
// reaches `need` (read with acquire semantics).  Returns false if the wait was
// abandoned (limit reached, or another wait raised the abort flag).
__device__ __noinline__ bool wait_count(uint32_t saddr, uint32_t need, const FlowArgs& a) {
  uint32_t v = ld_acquire_cta(saddr);
  if (v >= need) return true;
  const long long t0 = clock64();
  for (uint32_t it = 0;; ++it) {
    if (it >= 8) __nanosleep(32);   // after a short spin, keep the issue slots for the warps that have work
    v = ld_acquire_cta(saddr);
    if (v >= need) return true;
    if ((it & 15u) == 15u) {
      if (*reinterpret_cast<const volatile uint32_t*>(a.abort_flag) != 0u) return false;
      if (clock64() - t0 > a.spin_limit) {
        atomicExch(a.status, ISING_ERR_TIMEOUT);
        atomicExch(a.abort_flag, 1u);
        return false;
      }
    }
  }
}

// The same for a tagged mirror word: waits until its tag is `tag` and
// returns the tagged word (whose tag differs from `tag` if the wait was
// abandoned).
__device__ __noinline__ unsigned long long wait_tag(const unsigned long long* p, uint32_t tag, const FlowArgs& a) {
  unsigned long long v = ld_tagged(p);
  const long long t0 = clock64();
  for (uint32_t it = 0; tag_of(v) != tag; ++it) {
    if (it >= 8) __nanosleep(32);
    v = ld_tagged(p);
    if ((it & 15u) == 15u && tag_of(v) != tag) {
      if (*reinterpret_cast<const volatile uint32_t*>(a.abort_flag) != 0u) return v;
      if (clock64() - t0 > a.spin_limit) {
        atomicExch(a.status, ISING_ERR_TIMEOUT);
        atomicExch(a.abort_flag, 1u);
        return v;
      }
    }
  }
  return v;
}

// kGroupThr: every trial group has its own threshold table (a.thr_group_stride)
template <bool kU16, bool kGroupThr>
__global__ void __launch_bounds__(kFlowThreads, 1) anneal_flow_kernel(const __grid_constant__ FlowArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int j = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int H = a.H, Y = a.Y;
  const FlowSmem sm = flow_carve(smem, a.LRmax, H, a.cap, a.use_rec);
  const int w0 = a.split[j], w1 = a.split[j + 1];   // own words: stacked row * H + h in [w0, w1)

  // ---- local row tables (one thread; at most a few dozen rows)
  if (tid == 0) {
    int nloc = 0, nseg = 0;
    int seg_first[kMaxSeg], seg_n[kMaxSeg];
    for (int w = w0; w < w1;) {
      const int u = w / H;
      const int g = u / Y, ya = u - g * Y;
      const int wend = min(w1, (g + 1) * Y * H);   // this group's words within the range
      const int ub = (wend - 1) / H;
      const int n = ub - u + 1;
      const int ha0 = w - u * H, hbl = wend - ub * H;
      const bool whole = (wend - w == Y * H);
      sm.seg_g[nseg] = g;
      seg_n[nseg] = n;
      // layout: [halo top][own rows][halo bottom] (no halos for a whole group)
      const int own0 = whole ? nloc : nloc + 1;
      seg_first[nseg] = own0;
      for (int q = 0; q < n; ++q) {
        const int lr = own0 + q;
        const int y = ya + q;
        const bool shared = (q == 0 && ha0 > 0) || (q == n - 1 && hbl < H);
        const bool sh_up = q > 0 && ((q - 1 == 0 && ha0 > 0));
        const bool sh_dn = q < n - 1 && ((q + 1 == n - 1 && hbl < H));
        sm.r_u[lr] = g * Y + y;
        sm.r_seg[lr] = nseg;
        sm.r_ha[lr] = q == 0 ? ha0 : 0;
        sm.r_hb[lr] = q == n - 1 ? hbl : H;
        sm.r_xself[lr] = shared ? g * Y + y : -1;
        sm.r_xup[lr] = -1;
        sm.r_xdn[lr] = -1;
        if (whole) {
          sm.r_up[lr] = own0 + (q == 0 ? n - 1 : q - 1);
          sm.r_dn[lr] = own0 + (q == n - 1 ? 0 : q + 1);
        } else {
          // rows read through the global mirror: the halo rows (another
          // CTA's) and the rows shared with another CTA
          sm.r_up[lr] = lr - 1;
          sm.r_dn[lr] = lr + 1;
          if (q == 0 || sh_up) sm.r_xup[lr] = g * Y + (y + Y - 1) % Y;
          if (q == n - 1 || sh_dn) sm.r_xdn[lr] = g * Y + (y + 1) % Y;
        }
        // published: another CTA reads it (a shared row, or a neighbour of one
        // or of a halo row)
        sm.r_pub[lr] = shared || sm.r_xup[lr] >= 0 || sm.r_xdn[lr] >= 0;
      }
      if (!whole) {
        sm.r_u[nloc] = g * Y + (ya + Y - 1) % Y;              // halo slot above
        sm.r_u[own0 + n] = g * Y + (ya + n) % Y;              // halo slot below
        for (int q = 0; q < 2; ++q) {
          const int hl = q ? own0 + n : nloc;
          sm.r_seg[hl] = nseg;
          sm.r_up[hl] = hl;
          sm.r_dn[hl] = hl;
          sm.r_xup[hl] = -1;
          sm.r_xdn[hl] = -1;
          sm.r_pub[hl] = 0;
          sm.r_ha[hl] = 0;
          sm.r_hb[hl] = 0;
          sm.r_xself[hl] = -1;
        }
        nloc += n + 2;
      } else {
        nloc += n;
      }
      ++nseg;
      w = wend;
    }
    // processing order: the published rows of every segment first (from
    // both ends), then the remaining rows of each segment from both ends
    // towards the middle, the segments interleaved.  Every row's neighbours
    // are then processed about one half-sweep before it needs them, never
    // just before.
    int no = 0;
    int lo[kMaxSeg], hi[kMaxSeg];
    for (int s = 0; s < nseg; ++s) {
      lo[s] = seg_first[s];
      hi[s] = seg_first[s] + seg_n[s] - 1;
      for (bool more = true; more;) {
        more = false;
        if (lo[s] <= hi[s] && sm.r_pub[lo[s]]) { sm.order[no++] = lo[s]++; more = true; }
        if (lo[s] <= hi[s] && sm.r_pub[hi[s]]) { sm.order[no++] = hi[s]--; more = true; }
      }
    }
    for (bool more = true; more;) {
      more = false;
      for (int s = 0; s < nseg; ++s) {
        if (lo[s] <= hi[s]) { sm.order[no++] = lo[s]++; more = true; }
        if (lo[s] <= hi[s]) { sm.order[no++] = hi[s]--; more = true; }
      }
    }
    int items = 0;
    for (int oi = 0; oi < no; ++oi) {
      sm.oitem[oi] = items;
      items += sm.r_hb[sm.order[oi]] - sm.r_ha[sm.order[oi]];
    }
    sm.oitem[no] = items;
    sm.meta[0] = no;
    sm.meta[1] = nloc;
    sm.meta[2] = nseg;
    sm.meta[3] = items;
  }
  __syncthreads();
  const int nown = sm.meta[0], nloc = sm.meta[1], nseg = sm.meta[2];
  const int items = sm.meta[3];
  const int NC = (items + 31) >> 5;
  const int NR = nloc + 1;                 // local rows, then the row of idle lanes
  const int spare = 2 * a.LRmax * H;       // spin word that idle lanes update

  // Row records, per colour c and local row lr (two int4):
  //   A = {sp index of row `up` of colour 1-c | that of row `dn` << 16,
  //        site index of the row's first colour-c site, Philox head offset
  //        (segment * 8) | blocks << 8 | parity (y + c) & 1 << 16 | shared << 17,
  //        local row up | local row dn << 16}
  // A shared row (some of its words belong to another CTA) is always
  // published, so its colour-(1-c) mirror counter is B.z ^ 1.
  //   B = {counter of the colour-(1-c) row above in the global mirror, or -1,
  //        the same for the row below, mirror counter of this row's colour-c
  //        words if another CTA reads them, or -1,
  //        sp index of the row's colour-c words | that of its colour-(1-c) words << 16}
  // The idle lanes' row has its own counters saturated, reads and writes the
  // spare word and publishes nothing.
  for (int idx = tid; idx < 2 * NR; idx += kFlowThreads) {
    const int c = idx / NR, lr = idx - c * NR;
    int4 A, B;
    if (lr < nloc) {
      const int u = sm.r_u[lr];
      const int g = u / Y, y = u - g * Y;
      const int nq = decision_blocks<kU16>(min(a.G, a.T - g * a.G));
      const int up = sm.r_up[lr], dn = sm.r_dn[lr];
      const int ownp = c * a.LRmax * H, nbp = (1 - c) * a.LRmax * H;
      const int par = (y + c) & 1;
      A = make_int4((nbp + up * H) | ((nbp + dn * H) << 16), y * a.X + par,
                    sm.r_seg[lr] * 8 | (nq << 8) | (par << 16) | ((sm.r_xself[lr] >= 0) << 17), up | (dn << 16));
      const int xup = sm.r_xup[lr], xdn = sm.r_xdn[lr];
      B = make_int4(xup >= 0 ? 2 * xup + (1 - c) : -1, xdn >= 0 ? 2 * xdn + (1 - c) : -1,
                    sm.r_pub[lr] ? 2 * u + c : -1, (ownp + lr * H) | ((nbp + lr * H) << 16));
    } else {
      A = make_int4(spare | (spare << 16), 0, (1 << 8) | (1 << 16), nloc | (nloc << 16));
      B = make_int4(-1, -1, -1, spare);   // left and right: words 0 and 1 of row 0 (read, never written)
    }
    sm.rowc[2 * idx] = A;
    sm.rowc[2 * idx + 1] = B;
    sm.rowcnt[idx] = lr < nloc ? 0u : 0xFFFFFFFFu;
  }
  // Item records (lane e % 32 of chunk e / 32): {local row | h << 16, run},
  // where run > 0 marks the last lane of a run of items of one row within the
  // chunk and counts the run's items (the completion counter's increment).
  // Idle lanes take the idle row with h = 0: they update the spare word.
  for (int e = tid; e < NC * 32; e += kFlowThreads) {
    int2 v;
    if (e < items) {
      int oi = 0;
      while (sm.oitem[oi + 1] <= e) ++oi;
      const int lr = sm.order[oi];
      const int ha = sm.r_ha[lr];
      const int h = ha + (e - sm.oitem[oi]);
      const int ln = e & 31;
      v = make_int2(lr | (h << 16), (ln == 31 || e + 1 == items || h == sm.r_hb[lr] - 1) ? min(ln, h - ha) + 1 : 0);
    } else {
      v = make_int2(nloc, 0);
    }
    sm.xtab[e] = v;
  }
  if (tid == 0) {
    sm.sp[spare] = 0u;
    sm.fl[spare] = 0;
  }

  // ---- weights of own rows, starting spins of own rows and halo slots
  for (int idx = tid; idx < 2 * nloc * H; idx += kFlowThreads) {
    const int c = idx / (nloc * H);
    const int rem = idx - c * nloc * H;
    const int lr = rem / H;
    const int h = rem - lr * H;
    const int u = sm.r_u[lr];
    const int g = u / Y, y = u - g * Y;
    const int t0 = g * a.G;
    const int live = min(a.G, a.T - t0);
    const int nq = (live + 3) >> 2;
    const uint32_t q0 = static_cast<uint32_t>(t0) >> 2;
    const uint32_t i = static_cast<uint32_t>(y * a.X + 2 * h + ((y + c) & 1));
    uint32_t w = 0;
    if (a.init) {
      for (int b = 0; b < live; ++b)
        w |= static_cast<uint32_t>(a.init[static_cast<size_t>(t0 + b) * a.n + i] > 0) << b;
    } else {
      for (int jq = 0; jq < nq; ++jq) {
        const uint4 v = philox4x32_10(i, 0xFFFFFFFFu, q0 + jq, 0u, a.key0, a.key1);
        w |= ((v.x >> 31) | ((v.y >> 31) << 1) | ((v.z >> 31) << 2) | ((v.w >> 31) << 3)) << (4 * jq);
      }
    }
    sm.sp[(c * a.LRmax + lr) * H + h] = w;
    sm.fl[(c * a.LRmax + lr) * H + h] = a.flags[(static_cast<size_t>(c) * Y + y) * H + h];
  }
  __syncthreads();

  // ---- records of the fast path (when they fit in shared memory).  Per
  // colour c and item e, two uint4 with everything the item's update reads,
  // decoded once from the row and item tables:
  //   R0 = {shared byte address of the word, of its left, right and upper
  //         neighbours (colour 1-c)},
  //   R1 = {address of the lower neighbour, site index i, the edge signs as
  //         bytes (0x80: w = -1) left, right, up, down,
  //         run | mirror << 8 | segment << 9 | blocks << 11 | byte offset of
  //         the own row's colour-c counter << 16},
  // where run is the item's increment of that counter (see the item table)
  // and mirror marks rows that exchange words with another CTA through the
  // global mirror; it is then set on every item of the chunks that take the
  // general path (a mirror row, or more than 32 counters).  Per colour and
  // chunk, 32 counter addresses: the colour-(1-c) counters of every row the
  // chunk's items read (own, above, below), then the idle row's saturated
  // counter; ~0 when they are more than 32 (the chunk then takes the general
  // path).
  const uint32_t cap = static_cast<uint32_t>(a.cap);
  const uint32_t sp32 = smem_addr(sm.sp), cnt32 = smem_addr(sm.rowcnt);
  if (a.use_rec) {
    for (int idx = tid; idx < 2 * NC * 32; idx += kFlowThreads) {
      const int c = idx / (NC * 32), e = idx - c * NC * 32;
      const int2 it = sm.xtab[e];
      const uint32_t lr = static_cast<uint32_t>(it.x) & 0xFFFFu, h = static_cast<uint32_t>(it.x) >> 16;
      const int4 A = sm.rowc[2 * (c * NR + lr)], B = sm.rowc[2 * (c * NR + lr) + 1];
      const uint32_t par = (static_cast<uint32_t>(A.z) >> 16) & 1u;
      const uint32_t own = (static_cast<uint32_t>(B.w) & 0xFFFFu) + h;
      const uint32_t nbr = static_cast<uint32_t>(B.w) >> 16;
      const uint32_t hl = h + par == 0u ? static_cast<uint32_t>(H) - 1u : h + par - 1u;
      const uint32_t hr = h + par == static_cast<uint32_t>(H) ? 0u : h + par;
      const uint32_t f = sm.fl[own];
      const uint32_t fb = ((f & 1u) << 7) | ((f & 2u) << 14) | ((f & 4u) << 21) | ((f & 8u) << 28);
      const uint32_t mir = (B.x >= 0 || B.y >= 0 || B.z >= 0) ? 1u : 0u;
      const uint32_t seg = (static_cast<uint32_t>(A.z) & 0xFFu) >> 3, nq = (static_cast<uint32_t>(A.z) >> 8) & 0xFFu;
      const uint32_t slot = static_cast<uint32_t>(c) * cap + static_cast<uint32_t>(e);
      sm.rec[slot] = make_uint4(sp32 + 4u * own, sp32 + 4u * (nbr + hl), sp32 + 4u * (nbr + hr),
                                sp32 + 4u * ((static_cast<uint32_t>(A.x) & 0xFFFFu) + h));
      sm.rec[2 * cap + slot] = make_uint4(sp32 + 4u * ((static_cast<uint32_t>(A.x) >> 16) + h),
                                          static_cast<uint32_t>(A.y) + 2u * h, fb,
                                          static_cast<uint32_t>(it.y) | (mir << 8) | (seg << 9) | (nq << 11) |
                                              ((4u * (static_cast<uint32_t>(c * NR) + lr)) << 16));
    }
    for (int idx = tid; idx < 2 * NC; idx += kFlowThreads) {
      const int c = idx / NC, kc = idx - c * NC;
      const uint32_t base = static_cast<uint32_t>((1 - c) * NR);
      uint32_t list[32];
      int nl = 0;
      bool over = false;
      int prev = -1;
      for (int l = 0; l < 32; ++l) {
        const int lr = sm.xtab[kc * 32 + l].x & 0xFFFF;
        if (lr == prev) continue;
        prev = lr;
        const int4 A = sm.rowc[2 * (c * NR + lr)];
        const uint32_t rows[3] = {static_cast<uint32_t>(lr), static_cast<uint32_t>(A.w) & 0xFFFFu,
                                  static_cast<uint32_t>(A.w) >> 16};
        for (int q = 0; q < 3; ++q) {
          const uint32_t ci = base + rows[q];
          bool seen = false;
          for (int t = 0; t < nl; ++t) seen = seen || list[t] == ci;
          if (seen) continue;
          if (nl < 32) list[nl++] = ci;
          else over = true;
        }
      }
      uint32_t* out = sm.ccnt + (static_cast<size_t>(c) * (cap >> 5) + kc) * 32;
      for (int l = 0; l < 32; ++l)
        out[l] = (over && l == 31) ? 0xFFFFFFFFu : cnt32 + 4u * (l < nl ? list[l] : base + static_cast<uint32_t>(nloc));
    }
    __syncthreads();
    // a chunk with a mirror row or too many counters takes the general path
    // as a whole: the mirror bit of every item of it is set, so that the
    // loop branches on one record field, the same in every lane
    for (int idx = tid; idx < 2 * NC; idx += kFlowThreads) {
      const int c = idx / NC, kc = idx - c * NC;
      uint4* r1 = sm.rec + 2 * cap + static_cast<uint32_t>(c) * cap + 32u * static_cast<uint32_t>(kc);
      bool gen = sm.ccnt[(static_cast<size_t>(c) * (cap >> 5) + kc) * 32 + 31] == 0xFFFFFFFFu;
      for (int l = 0; l < 32; ++l) gen = gen || ((r1[l].w >> 8) & 1u) != 0u;
      if (gen)
        for (int l = 0; l < 32; ++l) r1[l].w |= 1u << 8;
    }
  }
  __syncthreads();

  // ---- the half-sweeps, chunk by chunk
  uint4* wh = sm.whead + warp * (kMaxSeg * 8);
  uint2* wt = sm.wthr + warp * kMaxSeg;
  const uint32_t fl32 = smem_addr(sm.fl);
  const uint32_t rowc32 = smem_addr(sm.rowc), xt32 = smem_addr(sm.xtab) + 8u * lane, wh32 = smem_addr(wh);
  const uint32_t rec32 = smem_addr(sm.rec) + 16u * lane, rstride = 32u * cap;
  const uint32_t cc32 = smem_addr(sm.ccnt) + 4u * lane;
  int head_kk = -1;
  uint32_t T4 = 0, T8 = 0;
  int hs = 0, k = warp;   // this warp's chunk: half-sweep hs, chunk k of it
  while (k >= NC && NC > 0) { k -= NC; ++hs; }
  const int HS = NC > 0 ? 2 * a.S : 0;
  // sweep kk, colour c, the counter value the chunk's rows must have reached
  // and the chunk's index in the records; they change only when the warp
  // moves on to the next half-sweep
  int kk = hs >> 1, c = hs & 1;
  uint32_t need = static_cast<uint32_t>(H) * static_cast<uint32_t>(kk + c);
  uint32_t ck = static_cast<uint32_t>(c) * (cap >> 5) + static_cast<uint32_t>(k);
  while (hs < HS) {
    if (kk != head_kk) {   // Philox heads and thresholds of this sweep
      __syncwarp();
      if (lane < nseg * 8) {
        const int s = lane >> 3, jq = lane & 7;
        const uint32_t q = decision_block0<kU16>(sm.seg_g[s] * a.G) + jq;
        wh[lane] = philox_head_sweep_quad(a.k0 + static_cast<uint32_t>(kk), q, a.key0, a.key1);
      }
      if constexpr (kGroupThr) {
        if (lane < nseg) {
          const uint32_t* t = a.thr + static_cast<size_t>(sm.seg_g[lane]) * a.thr_group_stride + 2 * kk;
          wt[lane] = make_uint2(__ldg(t), __ldg(t + 1));
        }
      }
      __syncwarp();
      T4 = __ldg(a.thr + 2 * kk);
      T8 = __ldg(a.thr + 2 * kk + 1);
      head_kk = kk;
    }
    bool fast = false;
    uint4 R1;
    if (a.use_rec) {
      R1 = lds_v4u(rec32 + rstride + 512u * ck);
      fast = ((R1.w >> 8) & 1u) == 0u;   // the same in every lane of the chunk
    }
    if (fast) {
      // ---- fast path: the chunk reads and writes this CTA's shared memory
      // only; each lane acquires one of the counters the chunk waits for
      const uint32_t caddr = lds_u32(cc32 + 128u * ck);
      const uint4 R0 = lds_v4u(rec32 + 512u * ck);
      const uint32_t v = ld_acquire_cta(caddr);
      if (!__all_sync(0xFFFFFFFFu, v >= need) || a.stall_test) {
        bool lane_ok = v >= need || wait_count(caddr, need, a);
        if (a.stall_test && j == 0 && hs == 0 && k == 0) lane_ok = lane_ok && wait_count(caddr, 0xFFFFFFFFu, a);
        if (!__all_sync(0xFFFFFFFFu, lane_ok)) break;
      }
      __syncwarp();   // every lane's reads after all lanes' acquires
      const uint32_t misc = R1.w;
      const uint32_t seg = (misc >> 9) & 3u;
      uint2 tq = make_uint2(T4, T8);
      if constexpr (kGroupThr) tq = wt[seg];
      const uint32_t fb = R1.z;
      const uint32_t ns = update_word_m<kU16>(lds_u32(R0.x), lds_u32(R0.y), lds_u32(R0.z), lds_u32(R0.w),
                                              lds_u32(R1.x), byte_sign_mask<0>(fb), byte_sign_mask<1>(fb),
                                              byte_sign_mask<2>(fb), byte_sign_mask<3>(fb), R1.y,
                                              HeadsShared{wh32 + 128u * seg}, static_cast<int>((misc >> 11) & 15u),
                                              tq.x, tq.y, a.rk);
      sts_u32(R0.x, ns);
      __syncwarp();
      const uint32_t run = misc & 0xFFu;
      if (run) red_release_cta(cnt32 + (misc >> 16), run);
    } else {
      // ---- general path: some lane reads or publishes words of the global mirror
      const int2 it = lds_v2(xt32 + 256u * static_cast<uint32_t>(k));
      const uint32_t lr = static_cast<uint32_t>(it.x) & 0xFFFFu, h = static_cast<uint32_t>(it.x) >> 16;
      const uint32_t rrec = rowc32 + 32u * (static_cast<uint32_t>(c * NR) + lr);
      const int4 A = lds_v4(rrec), B = lds_v4(rrec + 16u);
      const uint32_t rc = cnt32 + 4u * static_cast<uint32_t>((1 - c) * NR);
      const uint32_t c_self = rc + 4u * lr, c_up = rc + 4u * (static_cast<uint32_t>(A.w) & 0xFFFFu),
                     c_dn = rc + 4u * (static_cast<uint32_t>(A.w) >> 16);
      // the three colour-(1-c) rows this item reads must have finished the
      // previous half-sweep.  Rows of another CTA (and a row split between
      // two CTAs) are read from the tagged mirror, whose words carry their
      // half-sweep (except in the very first half-sweep, which reads the halo
      // slots); this CTA's own rows by the completion counters.  This CTA's
      // rows that another CTA reads are published to the mirror.
      const bool gu = B.x >= 0 && need > 0, gd = B.y >= 0 && need > 0;
      const bool gs = ((A.z >> 17) & 1) && need > 0;
      const uint32_t tag = static_cast<uint32_t>(hs);   // (half-sweep hs - 1) + 1
      // the word, its left and right neighbours (the row's wrap at h = 0 / H - 1)
      const uint32_t par = (static_cast<uint32_t>(A.z) >> 16) & 1u;
      const uint32_t own = (static_cast<uint32_t>(B.w) & 0xFFFFu) + h;
      const uint32_t nbr = static_cast<uint32_t>(B.w) >> 16;
      const uint32_t hl = h + par == 0u ? static_cast<uint32_t>(H) - 1u : h + par - 1u;
      const uint32_t hr = h + par == static_cast<uint32_t>(H) ? 0u : h + par;
      const unsigned long long* gself = a.gm + (gs ? static_cast<size_t>(B.z ^ 1) * H : 0);
      const unsigned long long* gup = a.gm + (gu ? static_cast<size_t>(B.x) * H + h : 0);
      const unsigned long long* gdn = a.gm + (gd ? static_cast<size_t>(B.y) * H + h : 0);
      const unsigned long long ml = gs ? ld_tagged(gself + hl) : 0ull, mr = gs ? ld_tagged(gself + hr) : 0ull;
      const unsigned long long mu = gu ? ld_tagged(gup) : 0ull, md = gd ? ld_tagged(gdn) : 0ull;
      const uint32_t v0 = gs ? need : ld_acquire_cta(c_self);
      const uint32_t v1 = gu ? need : ld_acquire_cta(c_up);
      const uint32_t v2 = gd ? need : ld_acquire_cta(c_dn);
      uint32_t nl = static_cast<uint32_t>(ml), nr = static_cast<uint32_t>(mr);
      uint32_t nu = static_cast<uint32_t>(mu), nd = static_cast<uint32_t>(md);
      const bool ready = v0 >= need && v1 >= need && v2 >= need && (!gs || (tag_of(ml) == tag && tag_of(mr) == tag)) &&
                         (!gu || tag_of(mu) == tag) && (!gd || tag_of(md) == tag);
      // one vote for the chunk: the bounded per-lane waits run only when some
      // lane is not ready yet (the usual case needs none)
      if (!__all_sync(0xFFFFFFFFu, ready) || a.stall_test) {
        bool lane_ok = true;
        if (gs) {
          if (tag_of(ml) != tag) {
            const unsigned long long w = wait_tag(gself + hl, tag, a);
            nl = static_cast<uint32_t>(w);
            lane_ok = tag_of(w) == tag;
          }
          if (lane_ok && tag_of(mr) != tag) {
            const unsigned long long w = wait_tag(gself + hr, tag, a);
            nr = static_cast<uint32_t>(w);
            lane_ok = tag_of(w) == tag;
          }
        } else if (v0 < need) {
          lane_ok = wait_count(c_self, need, a);
        }
        if (lane_ok && gu && tag_of(mu) != tag) {
          const unsigned long long w = wait_tag(gup, tag, a);
          nu = static_cast<uint32_t>(w);
          lane_ok = tag_of(w) == tag;
        }
        if (lane_ok && !gu && v1 < need) lane_ok = wait_count(c_up, need, a);
        if (lane_ok && gd && tag_of(md) != tag) {
          const unsigned long long w = wait_tag(gdn, tag, a);
          nd = static_cast<uint32_t>(w);
          lane_ok = tag_of(w) == tag;
        }
        if (lane_ok && !gd && v2 < need) lane_ok = wait_count(c_dn, need, a);
        if (a.stall_test && j == 0 && hs == 0 && k == 0) lane_ok = lane_ok && wait_count(c_self, 0xFFFFFFFFu, a);
        if (!__all_sync(0xFFFFFFFFu, lane_ok)) break;
      }
      if (!gs) {
        nl = lds_u32(sp32 + 4u * (nbr + hl));
        nr = lds_u32(sp32 + 4u * (nbr + hr));
      }
      if (!gu) nu = lds_u32(sp32 + 4u * ((static_cast<uint32_t>(A.x) & 0xFFFFu) + h));
      if (!gd) nd = lds_u32(sp32 + 4u * ((static_cast<uint32_t>(A.x) >> 16) + h));
      uint2 tq = make_uint2(T4, T8);
      if constexpr (kGroupThr) tq = wt[(A.z & 0xFF) >> 3];
      const uint32_t ns = update_word_h<kU16>(lds_u32(sp32 + 4u * own), nl, nr, nu, nd, lds_u8(fl32 + own),
                                              static_cast<uint32_t>(A.y) + 2u * h,
                                              HeadsShared{wh32 + 16u * (static_cast<uint32_t>(A.z) & 0xFFu)},
                                              (A.z >> 8) & 0xFF, tq.x, tq.y, a.rk);
      sts_u32(sp32 + 4u * own, ns);
      if (B.z >= 0) st_tagged(a.gm + static_cast<size_t>(B.z) * H + h, ns, static_cast<uint32_t>(hs) + 1u);   // published row
      __syncwarp();
      // the last lane of each run of one row's items counts the run in the
      // CTA's counter (the warp barrier orders the other lanes' stores before
      // the release)
      if (it.y) red_release_cta(cnt32 + 4u * (static_cast<uint32_t>(c * NR) + lr), static_cast<uint32_t>(it.y));
    }
    k += kFlowWarps;
    ck += kFlowWarps;
    if (k >= NC) {
      do { k -= NC; ++hs; } while (k >= NC);
      kk = hs >> 1;
      c = hs & 1;
      need = static_cast<uint32_t>(H) * static_cast<uint32_t>(kk + c);
      ck = static_cast<uint32_t>(c) * (cap >> 5) + static_cast<uint32_t>(k);
    }
  }
  __shared__ int s_stop;
  __syncthreads();
  if (tid == 0) s_stop = *reinterpret_cast<const volatile uint32_t*>(a.abort_flag) != 0u;
  __syncthreads();
  if (s_stop) return;   // CTA-uniform: every thread returns, nobody waits on a barrier

  // ---- read-out: spins of the own rows
  if (a.out_spins) {
    const int span = nown * a.X;
    for (int idx = tid; idx < span; idx += kFlowThreads) {
      const int oi = idx / a.X;
      const int x = idx - oi * a.X;
      const int lr = sm.order[oi];
      if ((x >> 1) < sm.r_ha[lr] || (x >> 1) >= sm.r_hb[lr]) continue;   // another CTA's word
      const int u = sm.r_u[lr];
      const int g = u / Y, y = u - g * Y;
      const int t0 = g * a.G;
      const int live = min(a.G, a.T - t0);
      const int c = (x + y) & 1;
      const uint32_t w = sm.sp[(static_cast<size_t>(c) * a.LRmax + lr) * H + (x >> 1)];
      int8_t* dst = a.out_spins + static_cast<size_t>(t0) * a.n + static_cast<size_t>(y) * a.X + x;
      for (int b = 0; b < live; ++b) dst[static_cast<size_t>(b) * a.n] = ((w >> b) & 1u) ? int8_t(1) : int8_t(-1);
    }
  }
  // ---- cut partials per trial: own right and down edges, summed over lanes
  // with ballots, per segment (all lanes of a pass share the segment's group)
  if (a.out_cuts) {
    // tag of the last half-sweep of a colour-0 word (a colour-1 word's is one more)
    const uint32_t fin = 2u * static_cast<uint32_t>(a.S) - 1u;
    bool cut_ok = true;
    for (int s = 0; s < nseg && cut_ok; ++s) {
      const int g = sm.seg_g[s];
      const int t0 = g * a.G;
      const int live = min(a.G, a.T - t0);
      uint32_t accb = 0;
      // own rows of segment s, both colours
      for (int base = warp * 32; base < 2 * nown * H && cut_ok; base += kFlowThreads) {
        const int idx = base + lane;
        uint32_t vr = 0, vd = 0;
        bool mine = false;
        int lr = 0, c = 0, h = 0;
        if (idx < 2 * nown * H) {
          c = idx / (nown * H);
          const int rem = idx - c * nown * H;
          const int oi = rem / H;
          h = rem - oi * H;
          lr = sm.order[oi];
          mine = sm.r_seg[lr] == s && h >= sm.r_ha[lr] && h < sm.r_hb[lr];
        }
        bool lok = true;
        if (mine) {
          const int u = sm.r_u[lr];
          const int y = u - g * Y;
          const int par = (y + c) & 1;
          const uint32_t* self = sm.sp + static_cast<size_t>(c) * a.LRmax * H;
          const uint32_t* nb = sm.sp + static_cast<size_t>(1 - c) * a.LRmax * H;
          const uint32_t sv = self[lr * H + h];
          const int hr = par ? (h == H - 1 ? 0 : h + 1) : h;
          uint32_t sr;
          const int xs = sm.r_xself[lr];
          if (xs >= 0 && a.S > 0) {   // a shared row: its final words are in the mirror
            const unsigned long long w = wait_tag(a.gm + (static_cast<size_t>(2) * xs + (1 - c)) * H + hr, fin + (1u - c), a);
            lok = tag_of(w) == fin + (1u - c);
            sr = static_cast<uint32_t>(w);
          } else {
            sr = nb[lr * H + hr];
          }
          uint32_t sd;
          const int xdn = sm.r_xdn[lr];
          if (lok && xdn >= 0 && a.S > 0) {
            const unsigned long long w = wait_tag(a.gm + (static_cast<size_t>(2) * xdn + (1 - c)) * H + h, fin + (1u - c), a);
            lok = tag_of(w) == fin + (1u - c);
            sd = static_cast<uint32_t>(w);
          } else {
            sd = nb[sm.r_dn[lr] * H + h];
          }
          const uint32_t f = sm.fl[(c * a.LRmax + lr) * H + h];
          vr = (sv ^ sr) ^ (0u - ((f >> 1) & 1u));
          vd = (sv ^ sd) ^ (0u - ((f >> 3) & 1u));
        }
        if (!__all_sync(0xFFFFFFFFu, lok)) {
          cut_ok = false;
          break;
        }
#pragma unroll 4
        for (int b = 0; b < 32; ++b) {
          const uint32_t cnt = __popc(__ballot_sync(0xFFFFFFFFu, (vr >> b) & 1u)) +
                               __popc(__ballot_sync(0xFFFFFFFFu, (vd >> b) & 1u));
          if (lane == b) accb += cnt;
        }
      }
      if (cut_ok && lane < live && accb) atomicAdd(a.acc + t0 + lane, static_cast<int32_t>(accb));
    }
    __shared__ int s_last, s_fail;
    if (tid == 0) s_fail = 0;
    __syncthreads();
    if (!cut_ok && lane == 0) s_fail = 1;
    __threadfence();
    __syncthreads();
    if (tid == 0)
      s_last = !s_fail && atomicAdd(a.done, 1u) == static_cast<uint32_t>(a.P - 1);
    __syncthreads();
    if (s_last) {
      __threadfence();
      for (int t = tid; t < a.T; t += kFlowThreads) a.out_cuts[t] = __ldcg(a.acc + t) - a.neg_edges;
    }
  }
}

}  // namespace

size_t flow_smem_bytes(int32_t LR, int32_t H, int32_t cap, int32_t rec) {
  size_t off[10];
  return flow_smem_layout(LR, H, cap, rec, off);
}

int flow_threads() { return kFlowThreads; }
int flow_max_segments() { return kMaxSeg; }

template <bool kU16, bool kGroupThr>
cudaError_t launch_flow_mode(const FlowArgs& a, cudaStream_t stream) {
  const size_t smem = flow_smem_bytes(a.LRmax, a.H, a.cap, a.use_rec);
  cudaError_t e = cudaFuncSetAttribute(anneal_flow_kernel<kU16, kGroupThr>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.P, 1, 1);
  cfg.blockDim = dim3(kFlowThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, anneal_flow_kernel<kU16, kGroupThr>, a);
}

cudaError_t launch_flow(const FlowArgs& a, cudaStream_t stream) {
  if (a.thr_group_stride > 0)
    return a.u16 ? launch_flow_mode<true, true>(a, stream) : launch_flow_mode<false, true>(a, stream);
  return a.u16 ? launch_flow_mode<true, false>(a, stream) : launch_flow_mode<false, false>(a, stream);
}

size_t flow_static_smem() {
  const void* fns[4] = {reinterpret_cast<const void*>(anneal_flow_kernel<false, false>),
                        reinterpret_cast<const void*>(anneal_flow_kernel<true, false>),
                        reinterpret_cast<const void*>(anneal_flow_kernel<false, true>),
                        reinterpret_cast<const void*>(anneal_flow_kernel<true, true>)};
  size_t v = 0;
  for (const void* fn : fns) {
    const size_t b = static_smem_of(fn);
    if (b > v) v = b;
  }
  return v;
}

cudaError_t flow_max_ctas(size_t smem, int* per_sm) {
  const void* fns[4] = {reinterpret_cast<const void*>(anneal_flow_kernel<false, false>),
                        reinterpret_cast<const void*>(anneal_flow_kernel<true, false>),
                        reinterpret_cast<const void*>(anneal_flow_kernel<false, true>),
                        reinterpret_cast<const void*>(anneal_flow_kernel<true, true>)};
  *per_sm = 1 << 30;
  for (const void* fn : fns) {
    int v = 0;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, fn, kFlowThreads, smem);
    if (e != cudaSuccess) return e;
    if (v < *per_sm) *per_sm = v;
  }
  return cudaSuccess;
}

}  // namespace ising

// conv_tc.cu -- the network's 3x3 circular convolutions on the 5th-generation
// tensor cores (tcgen05.mma, accumulators in tensor memory).
//
// Per output row (image b, row y) the convolution is a GEMM with M = pixels,
// N = output channels and K = 9 taps x input channels.  Instead of expanding
// the nine shifted copies of the input (im2col), each staged input row is
// laid out in shared memory as [8-channel chunk][pixel][16 bytes]: eight
// consecutive pixels of one chunk are then one "core matrix" of the
// no-swizzle K-major operand layout, whatever pixel they start at.  A tap's
// x-shift is just a 16-byte move of the descriptor's start address and its
// y-shift picks one of the three staged rows, so each input row is staged
// once per output row band and read by all nine taps in place.
//
// The row layout: [chunk][X + 2 padded to the tile grid][8 x BF16], pixel
// index + 1 (index 0 holds the periodic left neighbour x = X-1, index X+1
// the right neighbour x = 0, the rest of the padding is zero).
// Descriptor (SM100 shared-memory matrix descriptor, no swizzle): start >> 4,
// leading byte offset (next 8-channel chunk) >> 4, stride byte offset (next
// 8 pixels = 128 bytes) >> 4, version 1.  Instruction: kind::f16, BF16 A and
// B, FP32 D, both K-major, M = 128, N = 16 to 96.
//
// Persistent CTAs of 256 threads (two warpgroups) walk consecutive staged
// input rows, keeping a ring of five of them (each iteration stages one,
// three iterations ahead) and a ring of four TMEM accumulators (output rows)
// per tile.  Per staged row: one thread issues, per 128-pixel tile, kx and K
// step, one MMA into the accumulators of the up to three output rows the row
// feeds (N = 32 per row, the ky weights side by side; measured on GB300, an
// M = 128, K = 16 MMA takes about as long with N = 32 as with N = 96, so this
// needs a third of the MMAs of one per output row and tap) and commits to an
// mbarrier; meanwhile all threads wait (bounded) for the previous row's MMAs,
// drain the output row they completed (tcgen05.ld, fused epilogue, zero the
// accumulator for its next row).  The weight-gradient kernel below uses 128
// threads.
#include <cuda_bf16.h>

#include <algorithm>

#include "../../include/ising.h"
#include "internal.h"

namespace ising {
namespace {

constexpr int kTcThreads = 128;        // weight-gradient kernel
constexpr int kConvThreads = 256;      // convolution kernel: two warpgroups
constexpr int kRing = 5;               // staged input rows per convolution CTA
constexpr int kAcc = 4;                // output-row accumulators per tile (a power of two)
constexpr long long kWaitCycles = 4000000000LL;

__device__ __forceinline__ uint32_t saddr(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return static_cast<uint64_t>((addr >> 4) & 0x3FFFu) | (static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16) |
         (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (static_cast<uint64_t>(1) << 46);
}

// kind::f16 instruction descriptor: D = F32 (bits 4-5 = 1), A = B = BF16
// (bits 7-9 = 1, 10-12 = 1), K-major A and B, N >> 3 at bits 17-22, M >> 4 at 24-28
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tc(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

template <int kN>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float* v);

template <>
__device__ __forceinline__ void tmem_ld<32>(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <>
__device__ __forceinline__ void tmem_ld<16>(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <>
__device__ __forceinline__ void tmem_ld<1>(uint32_t taddr, float* v) {
  uint32_t r;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  v[0] = __uint_as_float(r);
}

// Zero 16 consecutive 32-bit columns of the calling warp's 32 lanes
__device__ __forceinline__ void tmem_zero16(uint32_t taddr) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(
                   taddr),
               "r"(0u)
               : "memory");
}

__device__ __forceinline__ int wrapi(int v, int m) { return v < 0 ? v + m : (v >= m ? v - m : v); }

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_group2() { asm volatile("cp.async.wait_group 2;" ::: "memory"); }

// Bounded wait on an mbarrier phase by the calling thread: false when `limit`
// cycles pass first.
__device__ __forceinline__ bool wait_mbar(uint32_t mbar, uint32_t phase, long long limit) {
  uint32_t done = 0;
  const long long t_start = clock64();
  while (!done) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(mbar), "r"(phase)
        : "memory");
    if (!done && clock64() - t_start > limit) break;
  }
  return done != 0;
}

// kIn: 0 = features (s, w_right, w_down) of spins/eflags, 16 channels (3 used);
//      1 = BF16 activations [P][32].
// kOut: 0 = BF16 [P][32] relu(acc + bias); 1 = BF16 [P][32] acc * [mask > 0];
//       2 = FP32 [P] acc(channel 0) + bias[0].
//
// Pipeline over the staged input rows r = ya-1 .. yb+1 of one image segment
// ya..yb (a CTA's rows split at image boundaries): input rows live in a ring
// of five slots (slot = unwrapped row mod 5), output rows in a ring of kAcc
// = 4 accumulators per 128-pixel tile (row y in slot y mod 4).  Along the
// columns the slots run in descending row order, so the rows r + 1, r, r - 1
// that staged row r feeds (ky = 0, 1, 2) sit side by side: per tile, kx and K
// step one MMA with N = 32 x (the valid ky) and B = those ky's weights side by
// side, instead of one MMA per output row and tap with N = 32 (an MMA costs
// about the same whether N is 32 or 96).  A window that wraps around the ring
// takes two MMAs.  Accumulators start at zero and the epilogue zeroes each
// one it drains, so every MMA accumulates.  Iteration r: barrier (row r
// staged, row r + 1's accumulator drained) -> the MMAs of row r -> wait for
// the MMAs of row r - 1 (frees slot r - 1; row r - 2 is complete) -> start
// copying row r + 3 into slot r + 3 = r - 2 (cp.async) -> epilogue of row
// r - 2 -> wait for the copies of row r + 1.  256 threads: warp w drains TMEM
// lanes 32 (w mod 4) .. and columns 16 (w / 4) .. of an accumulator.
template <int kIn, int kOut>
__global__ void __launch_bounds__(kConvThreads, 3) conv_tc_kernel(TcConvArgs a) {
  constexpr int KC = kIn == 0 ? 2 : 4;          // 8-channel chunks of the input
  constexpr int N = kOut == 2 ? 16 : 32;         // output channels (padded)
  constexpr int NG = N / 8;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int X = a.X, Y = a.Y, n = X * Y;
  const int ntile = (X + 127) >> 7;
  const int RP = ntile * 128 + 2;                // pixels per staged chunk row
  const size_t wbytes = static_cast<size_t>(9) * KC * NG * 128;
  unsigned char* sw = smem;                                        // weights [9][KC][NG][8][16B]
  unsigned char* srow = smem + wbytes;                              // kRing slots x [KC][RP][16B]
  const size_t slot_bytes = static_cast<size_t>(KC) * RP * 16;
  // [0], [1]: MMA completion of accumulator buffers 0, 1; [2]: a spare barrier
  // nothing arrives at (the stall test waits on it)
  uint64_t* mbar = reinterpret_cast<uint64_t*>(srow + kRing * slot_bytes);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 3);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // weights: the canonical [tap][chunk][N group][128 B] blocks reordered to
  // [kx][chunk][ky][N group], so that the three ky of one (kx, chunk) form one
  // B operand of N = 3 x 32 rows
  for (int i = tid; i < static_cast<int>(wbytes / 16); i += kConvThreads) {
    const int blk = i >> 3, tap = blk / (KC * NG), rem = blk - tap * (KC * NG), kc = rem / NG, ng = rem - kc * NG;
    const int ky = tap / 3, kx = tap - 3 * ky;
    const int dst = ((kx * KC + kc) * 3 + ky) * NG + ng;
    reinterpret_cast<uint4*>(sw)[dst * 8 + (i & 7)] = reinterpret_cast<const uint4*>(a.wt)[i];
  }
  for (int i = tid; i < static_cast<int>(kRing * slot_bytes / 16); i += kConvThreads)
    reinterpret_cast<uint4*>(srow)[i] = make_uint4(0, 0, 0, 0);   // padding: never rewritten
  const uint32_t bufcols = static_cast<uint32_t>(ntile * N);
  uint32_t tcols = 32;
  while (tcols < kAcc * bufcols) tcols <<= 1;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tslot)),
                 "r"(tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(mbar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(mbar + 1)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(mbar + 2)));
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t lane_off = static_cast<uint32_t>((warp & 3) * 32) << 16;
  const int half = warp >> 2;                    // which 16 of the 32 output channels
  float bias_r[16];                              // this thread's output channels' biases
#pragma unroll
  for (int c = 0; c < 16; ++c) bias_r[c] = kOut == 0 ? __ldg(a.bias + half * 16 + c) : 0.f;
  const float bias0 = kOut == 2 ? __ldg(a.bias) : 0.f;
  // accumulator of output row y, tile t: columns t * kAcc * N + N * (kAcc - 1 - y mod kAcc)
  auto acc_col = [&](int t, int y) {
    return static_cast<uint32_t>(t * kAcc * N + N * (kAcc - 1 - (y & (kAcc - 1))));
  };
  // every accumulator starts at zero (each warp clears its lanes and columns)
  if (half * 16 < N) {
    for (int t = 0; t < ntile; ++t)
      for (int s = 0; s < kAcc; ++s) tmem_zero16(tmem + lane_off + static_cast<uint32_t>((t * kAcc + s) * N + half * 16));
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }

  // stage unwrapped input row yu of image b into its ring slot
  auto stage = [&](int b, int yu) {
    const int yy = wrapi(yu, Y);
    unsigned char* slot = srow + static_cast<size_t>((yu + kRing) % kRing) * slot_bytes;
    for (int i = tid; i < (X + 2) * KC; i += kConvThreads) {
      const int pidx = i / KC, kc = i - pidx * KC;
      const int x = wrapi(pidx - 1, X);
      unsigned char* dst = slot + (static_cast<size_t>(kc) * RP + pidx) * 16;
      if (kIn == 0) {
        const int j = yy * X + x;
        __align__(16) __nv_bfloat16 f[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) f[e] = __float2bfloat16(0.f);
        if (kc == 0) {
          const uint8_t fl = a.eflags[j];
          f[0] = __float2bfloat16(a.spins[static_cast<size_t>(b) * n + j] > 0 ? 1.f : -1.f);
          f[1] = __float2bfloat16((fl & 1u) ? -1.f : 1.f);
          f[2] = __float2bfloat16((fl & 2u) ? -1.f : 1.f);
        }
        *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(f);
      } else {
        cp_async16(saddr(dst), a.in + (static_cast<size_t>(b) * n + yy * X + x) * 32 + kc * 8);
      }
    }
  };

  // Descriptor bases: the start-address field is the low 14 bits (address >> 4)
  // and shared addresses stay below 256 KB, so offsets add without carries.
  const uint32_t lbo_a = static_cast<uint32_t>(RP) * 16;
  const uint64_t adesc0 = smem_desc(saddr(srow), lbo_a, 128);
  const uint32_t slot16 = static_cast<uint32_t>(slot_bytes >> 4);
  const uint64_t bdesc3 = smem_desc(saddr(sw), 3 * NG * 128, 128);   // K step: next chunk of the reordered weights
  // the MMAs of staged row r (unwrapped, segment ya..yb), committed to mbar[cb]
  auto issue_window = [&](int r, int ya, int yb, int cb) {
    const int kmin = r + 1 - yb > 0 ? r + 1 - yb : 0;
    const int kmax = r + 1 - ya < 2 ? r + 1 - ya : 2;
    const uint64_t ad0 = adesc0 + static_cast<uint64_t>(((r + kRing) % kRing) * slot16);
    const int qhi = (r + 1 - kmin) & (kAcc - 1);   // slot of the highest row (ky = kmin)
    const int len = kmax - kmin + 1;
    const int len0 = len < qhi + 1 ? len : qhi + 1;
    for (int run = 0; run < 2; ++run) {
      const int k0 = run == 0 ? kmin : kmin + len0;
      const int L = run == 0 ? len0 : len - len0;
      if (L <= 0) continue;
      const int y0 = r + 1 - k0;   // the run's highest row
      const uint32_t idesc = idesc_bf16(128, N * L);
      for (int t = 0; t < ntile; ++t) {
        const uint32_t d = tmem + acc_col(t, y0);
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
#pragma unroll
          for (int ks = 0; ks < KC / 2; ++ks) {
            const uint64_t ad = ad0 + static_cast<uint64_t>((2 * ks * lbo_a + (t * 128 + kx) * 16) >> 4);
            const uint64_t bd = bdesc3 + static_cast<uint64_t>((((kx * KC + 2 * ks) * 3 + k0) * NG * 128) >> 4);
            mma_tc(d, ad, bd, idesc, 1u);
          }
        }
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     saddr(mbar + cb))
                 : "memory");
  };

  // kOut 1: the ReLU mask of the row the next epilogue drains, loaded while
  // the MMAs run (the first two tiles; later tiles load in the epilogue)
  uint4 m00 = make_uint4(0, 0, 0, 0), m01 = m00, m10 = m00, m11 = m00;   // [tile][half of 16 channels]
  auto prefetch_mask = [&](int b, int y) {
    if constexpr (kOut == 1) {
      const int x0 = (warp & 3) * 32 + lane;
      const size_t p = static_cast<size_t>(b) * n + static_cast<size_t>(y) * X + x0;
      if (x0 < X) {
        const uint4* mk = reinterpret_cast<const uint4*>(a.mask + p * 32 + half * 16);
        m00 = mk[0];
        m01 = mk[1];
      }
      if (ntile > 1 && x0 + 128 < X) {
        const uint4* mk = reinterpret_cast<const uint4*>(a.mask + (p + 128) * 32 + half * 16);
        m10 = mk[0];
        m11 = mk[1];
      }
    }
  };

  auto epilogue = [&](int b, int y) {
    if (kOut == 2 && half) return;               // one logit channel: the first warpgroup alone
    for (int t = 0; t < ntile; ++t) {
      const int x = t * 128 + (warp & 3) * 32 + lane;
      const size_t p = static_cast<size_t>(b) * n + static_cast<size_t>(y) * X + x;
      const uint32_t col = tmem + lane_off + acc_col(t, y);
      if (kOut == 2) {
        float v[1];
        tmem_ld<1>(col, v);
        tmem_zero16(col);
        if (x < X) a.out_f32[p] = v[0] + bias0;
        continue;
      }
      float v[16];
      tmem_ld<16>(col + static_cast<uint32_t>(half * 16), v);
      tmem_zero16(col + static_cast<uint32_t>(half * 16));
      if (x >= X) continue;
      __align__(16) __nv_bfloat16 o[16];
      if (kOut == 0) {
#pragma unroll
        for (int c = 0; c < 16; ++c) o[c] = __float2bfloat16(fmaxf(v[c] + bias_r[c], 0.f));
      } else {
        const uint4* mk = reinterpret_cast<const uint4*>(a.mask + p * 32 + half * 16);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const uint4 mv = t == 0 ? (q ? m01 : m00) : t == 1 ? (q ? m11 : m10) : mk[q];
          const __nv_bfloat16* m8 = reinterpret_cast<const __nv_bfloat16*>(&mv);
#pragma unroll
          for (int e = 0; e < 8; ++e)
            o[q * 8 + e] = __float2bfloat16(__bfloat162float(m8[e]) > 0.f ? v[q * 8 + e] : 0.f);
        }
      }
      uint4* dst = reinterpret_cast<uint4*>(a.out_bf16 + p * 32 + half * 16);
      dst[0] = reinterpret_cast<const uint4*>(o)[0];
      dst[1] = reinterpret_cast<const uint4*>(o)[1];
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");   // the zeroed accumulator
  };

  const long long R = static_cast<long long>(a.B) * Y;
  const long long r0 = R * blockIdx.x / gridDim.x, r1 = R * (blockIdx.x + 1) / gridDim.x;
  const long long limit = a.wait_limit > 0 ? a.wait_limit : kWaitCycles;
  uint32_t phases = 0;    // bit j: parity to wait for on mbar[j]
  uint32_t pending = 0;   // bit j: MMAs committed to mbar[j] and not yet awaited
  bool stall = a.stall_test != 0 && blockIdx.x == 0;
  bool ok = true;
  for (long long row = r0; row < r1 && ok;) {
    const int b = static_cast<int>(row / Y);
    const long long img_end = static_cast<long long>(b + 1) * Y;
    const long long seg_end = r1 < img_end ? r1 : img_end;
    const int ya = static_cast<int>(row - static_cast<long long>(b) * Y);
    const int yb = static_cast<int>(seg_end - 1 - static_cast<long long>(b) * Y);
    stage(b, ya - 1);
    stage(b, ya);
    stage(b, ya + 1);
    if (kIn != 0) cp_async_commit_wait_all();
    for (int r = ya - 1; r <= yb + 1; ++r) {
      const uint32_t cb = static_cast<uint32_t>(r - ya + 1) & 1u;   // MMA barrier of staged row r
      // row r staged by every thread, row r + 1's accumulator drained and
      // zeroed by every thread; a wait that ran out anywhere ends the CTA's
      // work here
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      ok = __syncthreads_and(ok) != 0;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (!ok) break;
      if (tid == 0) issue_window(r, ya, yb, static_cast<int>(cb));
      pending |= 1u << cb;
      if (stall) {   // test switch: a bounded wait on the barrier nothing arrives at
        stall = false;
        if (!wait_mbar(saddr(mbar + 2), 0u, limit)) ok = false;
      }
      const bool out_row = r - 2 >= ya;   // row r - 2 is complete once row r - 1's MMAs are
      if (out_row) prefetch_mask(b, r - 2);
      bool prev = false;
      if (ok && r >= ya) {
        const uint32_t pb = cb ^ 1u;
        prev = wait_mbar(saddr(mbar + pb), (phases >> pb) & 1u, limit);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (prev) {
          phases ^= 1u << pb;
          pending &= ~(1u << pb);
        } else {
          ok = false;
        }
      }
      if (ok && r + 3 <= yb + 1) stage(b, r + 3);
      if (kIn != 0) cp_async_commit();           // (possibly empty) group of row r + 3
      if (prev && out_row) epilogue(b, r - 2);
      if (kIn != 0) cp_async_wait_group2();      // row r + 1 has landed
    }
    if (ok) {
      // row yb: its last contributions are staged row yb + 1's MMAs
      prefetch_mask(b, yb);
      const uint32_t lb = static_cast<uint32_t>(yb - ya + 2) & 1u;
      const bool last = wait_mbar(saddr(mbar + lb), (phases >> lb) & 1u, limit);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (last) {
        phases ^= 1u << lb;
        pending &= ~(1u << lb);
        epilogue(b, yb);
      } else {
        ok = false;
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    ok = __syncthreads_and(ok) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    row = seg_end;
  }
  if (!ok && tid == 0) atomicExch(a.status, ISING_ERR_TIMEOUT);
  // MMAs still committed but not awaited (the work ended early) finish before
  // their tensor memory is freed
  for (uint32_t j = 0; j < 2; ++j)
    if (pending & (1u << j)) wait_mbar(saddr(mbar + j), (phases >> j) & 1u, kWaitCycles);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (kIn != 0) cp_async_commit_wait_all();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols));
}

// CTAs of `threads` threads that the register file holds per SM (registers are
// allocated per warp in units of 256)
inline int regs_per_sm_limit(const void* fn, int threads) {
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess || fa.numRegs <= 0) return 1;
  const int per_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
  const int warps = (threads + 31) / 32;
  const int v = 65536 / (per_warp * warps);
  return v > 0 ? v : 1;
}

template <int kIn, int kOut>
size_t smem_bytes_for(int X) {
  constexpr int KC = kIn == 0 ? 2 : 4;
  constexpr int NG = (kOut == 2 ? 16 : 32) / 8;
  const int RP = ((X + 127) / 128) * 128 + 2;
  return static_cast<size_t>(9) * KC * NG * 128 + kRing * static_cast<size_t>(KC) * RP * 16 + 32;
}

template <int kIn, int kOut>
cudaError_t launch_one(const TcConvArgs& a, int sms, cudaStream_t st) {
  const size_t sm = smem_bytes_for<kIn, kOut>(a.X);
  cudaError_t e = cudaFuncSetAttribute(conv_tc_kernel<kIn, kOut>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(sm));
  if (e != cudaSuccess) return e;
  // residency from shared memory (per-SM capacity, 1 KB reserved per CTA) and
  // tensor memory (512 columns per SM: two accumulator buffers per CTA)
  int dev = 0, smem_sm = 0, reserved = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  if (e != cudaSuccess) return e;
  int per_sm = static_cast<int>(static_cast<size_t>(smem_sm) / (sm + static_cast<size_t>(reserved)));
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int cols = kAcc * ((a.X + 127) / 128) * (kOut == 2 ? 16 : 32);
  int tc = 32;
  while (tc < cols) tc <<= 1;
  if (tc > 512) return cudaErrorInvalidConfiguration;
  per_sm = std::min(std::min(per_sm, 512 / tc), 8);
  per_sm = std::min(per_sm, regs_per_sm_limit(reinterpret_cast<const void*>(conv_tc_kernel<kIn, kOut>), kConvThreads));
  const long long rows = static_cast<long long>(a.B) * a.Y;
  const long long grid = std::min<long long>(rows, static_cast<long long>(sms) * per_sm);
  conv_tc_kernel<kIn, kOut><<<static_cast<int>(grid), kConvThreads, sm, st>>>(a);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ weight gradients
// dW[o][c][ky][kx] = sum over images, rows y and pixels p of
//   g[y][p][o] * a[y+ky-1][p+kx-1][c]   (indices mod Y, X).
// Per output row y this is one GEMM with K = pixels:
//   D[(ky, c)][(kx, o)] += sum_p a[y+ky-1][p][c] * g[y][p-kx+1][o]
// A (M = 128: three activation rows x 32 channels, plus 32 ignored rows) is
// the three rows staged unshifted; B (N = 96: three copies of the gradient row
// shifted by kx - 1 pixels, x 32 channels) is staged three times.  Both are
// MN-major (8 channels contiguous per pixel, 8 pixels per core matrix), so the
// staged layout [8-channel block][pixel][16 B] serves as is: the leading byte
// offset steps 8 pixels (128 B), the stride byte offset one channel block.
// One FP32 accumulator (128 x N) per CTA sums all of the CTA's rows; the CTA
// writes it out once and a second kernel reduces the CTAs in a fixed order.
// Kinds: 0 = layer 1 (a = features s, w_right, w_down; g BF16 [32]);
//        1 = layers 2, 3 (a, g BF16 [32]);
//        2 = layer 4 (a BF16 [32]; g = dz FP32, split into BF16 hi + lo).
template <int kKind>
__global__ void __launch_bounds__(kTcThreads) wgrad_tc_kernel(TcWgradArgs a) {
  constexpr int NB = kKind == 2 ? 4 : 12;          // B blocks of 8 columns (kind 2: 3 used)
  constexpr int N = NB * 8;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int X = a.X, Y = a.Y, n = X * Y;
  const int ksteps = (X + 15) >> 4;
  const int RP = ksteps * 16;                        // pixels per staged block row
  const size_t blk = static_cast<size_t>(RP) * 16;   // bytes per block row
  unsigned char* sA = smem;                          // 12 blocks: [ky][chunk][pixel][16 B]
  unsigned char* sB = smem + 12 * blk;               // NB blocks: [kx][chunk][pixel][16 B]
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sB + NB * blk);   // [0] MMA completion, [1] spare (stall test)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);
  float* sbias = reinterpret_cast<float*>(tslot + 4);   // [warps][32] per-warp bias sums
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  for (int i = tid; i < static_cast<int>((12 + NB) * blk / 16); i += kTcThreads)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
  constexpr uint32_t tcols = N <= 32 ? 32 : 128;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tslot)),
                 "r"(tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(mbar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(mbar + 1)));
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const long long limit = a.wait_limit > 0 ? a.wait_limit : kWaitCycles;
  bool stall = a.stall_test != 0 && blockIdx.x == 0;

  const long long R = static_cast<long long>(a.B) * Y;
  const long long r0 = R * blockIdx.x / gridDim.x, r1 = R * (blockIdx.x + 1) / gridDim.x;
  float bsum[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) bsum[e] = 0.f;
  uint32_t phase = 0;
  bool ok = true, first = true;
  for (long long row = r0; row < r1 && ok; ++row) {
    const int b = static_cast<int>(row / Y), y = static_cast<int>(row - static_cast<long long>(b) * Y);
    const size_t ib = static_cast<size_t>(b) * n;
    // ---- A: activation rows y-1, y, y+1
    if (kKind == 0) {
      for (int i = tid; i < 3 * X; i += kTcThreads) {
        const int ky = i / X, x = i - ky * X;
        const int j = wrapi(y + ky - 1, Y) * X + x;
        const uint8_t fl = a.eflags[j];
        __align__(16) __nv_bfloat16 f[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) f[e] = __float2bfloat16(0.f);
        f[0] = __float2bfloat16(a.spins[ib + j] > 0 ? 1.f : -1.f);
        f[1] = __float2bfloat16((fl & 1u) ? -1.f : 1.f);
        f[2] = __float2bfloat16((fl & 2u) ? -1.f : 1.f);
        *reinterpret_cast<uint4*>(sA + (static_cast<size_t>(ky) * 4) * blk + static_cast<size_t>(x) * 16) =
            *reinterpret_cast<const uint4*>(f);
      }
    } else {
      // asynchronous copies: every thread's share of the three rows is in
      // flight at once, awaited once before the barrier
      const int total = 3 * X * 4;
      for (int i = tid; i < total; i += kTcThreads) {
        const int ky = i / (X * 4), rem = i - ky * X * 4, x = rem >> 2, ch = rem & 3;
        cp_async16(saddr(sA + static_cast<size_t>(ky * 4 + ch) * blk + static_cast<size_t>(x) * 16),
                   a.act + (ib + static_cast<size_t>(wrapi(y + ky - 1, Y)) * X + x) * 32 + ch * 8);
      }
    }
    // ---- B: gradient row y at positions p = x + kx - 1 (mod X) of copy kx
    if (kKind == 2) {
      const float* dz = static_cast<const float*>(a.g) + ib + static_cast<size_t>(y) * X;
      for (int x = tid; x < X; x += kTcThreads) {
        const float v = dz[x];
        bsum[0] += v;
        const __nv_bfloat16 hi = __float2bfloat16(v);
        const __nv_bfloat16 lo = __float2bfloat16(v - __bfloat162float(hi));
        __align__(16) __nv_bfloat16 f[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) f[e] = __float2bfloat16(0.f);
        f[0] = hi;
        f[1] = lo;
        const uint4 q = *reinterpret_cast<const uint4*>(f);
#pragma unroll
        for (int kx = 0; kx < 3; ++kx)
          *reinterpret_cast<uint4*>(sB + static_cast<size_t>(kx) * blk + static_cast<size_t>(wrapi(x + kx - 1, X)) * 16) = q;
      }
    } else {
      const __nv_bfloat16* g = static_cast<const __nv_bfloat16*>(a.g) + (ib + static_cast<size_t>(y) * X) * 32;
      for (int i = tid; i < X * 4; i += kTcThreads) {
        const int x = i >> 2, ch = i & 3;   // ch == tid & 3 for every i of this thread
        const uint4 q = reinterpret_cast<const uint4*>(g + static_cast<size_t>(x) * 32)[ch];
        const __nv_bfloat16* h = reinterpret_cast<const __nv_bfloat16*>(&q);
#pragma unroll
        for (int e = 0; e < 8; ++e) bsum[e] += __bfloat162float(h[e]);
#pragma unroll
        for (int kx = 0; kx < 3; ++kx)
          *reinterpret_cast<uint4*>(sB + static_cast<size_t>(kx * 4 + ch) * blk +
                                    static_cast<size_t>(wrapi(x + kx - 1, X)) * 16) = q;
      }
    }
    if (kKind != 0) cp_async_commit_wait_all();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
      const uint32_t idesc = idesc_bf16(128, N) | (1u << 15) | (1u << 16);   // A and B MN-major
      const uint32_t sbo = static_cast<uint32_t>(blk);
      for (int ks = 0; ks < ksteps; ++ks) {
        mma_tc(tmem, smem_desc(saddr(sA) + ks * 256, 128, sbo), smem_desc(saddr(sB) + ks * 256, 128, sbo), idesc,
               (first && ks == 0) ? 0u : 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(mbar))
                   : "memory");
    }
    first = false;
    bool stalled = false;
    if (stall) {   // test switch: a bounded wait on the barrier nothing arrives at
      stall = false;
      stalled = !wait_mbar(saddr(mbar + 1), 0u, limit);
    }
    // the next row's staging overwrites what these MMAs read: wait for them
    // (also after a stall, so that they finish before tensor memory is freed)
    uint32_t done = wait_mbar(saddr(mbar), phase, limit) ? 1u : 0u;
    phase ^= 1u;
    done = __syncthreads_and(done && !stalled);
    if (!done) {
      if (tid == 0) atomicExch(a.status, ISING_ERR_TIMEOUT);
      ok = false;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  // ---- bias partial sums, in a fixed order (so training is reproducible):
  // a butterfly within each warp, then the warps' sums in turn
  if (kKind == 2) {
    float v = bsum[0];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    sbias[warp * 32 + lane] = lane == 0 ? v : 0.f;
  } else {
    // lanes with equal lane & 3 hold the same eight channels
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      float v = bsum[e];
      v += __shfl_xor_sync(0xFFFFFFFFu, v, 4);
      v += __shfl_xor_sync(0xFFFFFFFFu, v, 8);
      v += __shfl_xor_sync(0xFFFFFFFFu, v, 16);
      if (lane < 4) sbias[warp * 32 + lane * 8 + e] = v;
    }
  }
  __syncthreads();
  if (tid < 32) {
    float v = 0.f;
    for (int w = 0; w < kTcThreads / 32; ++w) v += sbias[w * 32 + tid];
    a.bpart[static_cast<size_t>(blockIdx.x) * 32 + tid] = v;
  }
  // ---- accumulator rows (ky, c) = warp, lane; rows 96..127 are not used
  float* out = a.part + static_cast<size_t>(blockIdx.x) * 96 * N;
  if (ok && !first) {
#pragma unroll
    for (int c0 = 0; c0 < N; c0 += 32) {
      float v[32];
      if (N - c0 >= 32) {
        tmem_ld<32>(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c0, v);
      } else {
        tmem_ld<16>(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c0, v);
      }
      if (warp < 3) {
        const int w = N - c0 >= 32 ? 32 : 16;
        for (int q = 0; q < w; ++q) out[static_cast<size_t>(warp * 32 + lane) * N + c0 + q] = v[q];
      }
    }
  } else if (warp < 3) {
    for (int q = 0; q < N; ++q) out[static_cast<size_t>(warp * 32 + lane) * N + q] = 0.f;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols));
}

// First reduction stage: group g of kGroups sums the partials of CTAs
// g, g + kGroups, ... (increasing order) and leaves the sum in CTA g's slot.
constexpr int kGroups = 16;
template <int kKind>
__global__ void wgrad_group_kernel(float* __restrict__ part, float* __restrict__ bpart, int ncta) {
  constexpr int N = kKind == 2 ? 32 : 96;
  constexpr int E = 96 * N;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int g = blockIdx.y;
  if (g >= ncta) return;
  if (e < E) {
    float s = 0.f;
    for (int k = g; k < ncta; k += kGroups) s += part[static_cast<size_t>(k) * E + e];
    part[static_cast<size_t>(g) * E + e] = s;
  } else if (e < E + 32) {
    const int o = e - E;
    float s = 0.f;
    for (int k = g; k < ncta; k += kGroups) s += bpart[static_cast<size_t>(k) * 32 + o];
    bpart[static_cast<size_t>(g) * 32 + o] = s;
  }
}

// Second stage: sum the group results (fixed order) into dW[o][c][ky*3+kx]
// and db[o].
template <int kKind>
__global__ void wgrad_reduce_kernel(const float* __restrict__ part, const float* __restrict__ bpart, int ngroups,
                                    float* __restrict__ dW, float* __restrict__ db) {
  constexpr int C = kKind == 0 ? 3 : 32;
  constexpr int O = kKind == 2 ? 1 : 32;
  constexpr int N = kKind == 2 ? 32 : 96;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < O * C * 9) {
    const int o = t % O, rest = t / O, c = rest % C, tap = rest / C, ky = tap / 3, kx = tap - ky * 3;
    const size_t row = static_cast<size_t>(ky * 32 + c) * N;
    float s = 0.f;
    if (kKind == 2) {
      for (int k = 0; k < ngroups; ++k) {
        const float* pk = part + static_cast<size_t>(k) * 96 * N + row + kx * 8;
        s += pk[0] + pk[1];
      }
    } else {
      for (int k = 0; k < ngroups; ++k) s += part[static_cast<size_t>(k) * 96 * N + row + kx * 32 + o];
    }
    dW[(o * C + c) * 9 + tap] = s;
  } else if (t < O * C * 9 + O) {
    const int o = t - O * C * 9;
    float s = 0.f;
    for (int k = 0; k < ngroups; ++k) s += bpart[static_cast<size_t>(k) * 32 + o];
    db[o] = s;
  }
}

template <int kKind>
size_t wgrad_smem_for(int X) {
  constexpr int NB = kKind == 2 ? 4 : 12;
  const size_t RP = static_cast<size_t>((X + 15) / 16) * 16;
  return (12 + NB) * RP * 16 + 32 + (kTcThreads / 32) * 32 * sizeof(float);
}

template <int kKind>
cudaError_t launch_wgrad_one(const TcWgradArgs& a, int sms, float* dW, float* db, cudaStream_t st) {
  const size_t sm = wgrad_smem_for<kKind>(a.X);
  cudaError_t e = cudaFuncSetAttribute(wgrad_tc_kernel<kKind>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(sm));
  if (e != cudaSuccess) return e;
  int dev = 0, smem_sm = 0, reserved = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  if (e != cudaSuccess) return e;
  int per_sm = static_cast<int>(static_cast<size_t>(smem_sm) / (sm + static_cast<size_t>(reserved)));
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  per_sm = std::min(per_sm, kKind == 2 ? 16 : 4);   // tensor memory: 512 columns per SM
  per_sm = std::min(per_sm, regs_per_sm_limit(reinterpret_cast<const void*>(wgrad_tc_kernel<kKind>), kTcThreads));
  const long long rows = static_cast<long long>(a.B) * a.Y;
  long long grid = std::min<long long>(rows, static_cast<long long>(sms) * per_sm);
  grid = std::min<long long>(grid, a.max_ctas);
  wgrad_tc_kernel<kKind><<<static_cast<int>(grid), kTcThreads, sm, st>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int ncta = static_cast<int>(grid);
  const int ngroups = std::min(ncta, kGroups);
  constexpr int elems = 96 * (kKind == 2 ? 32 : 96) + 32;
  wgrad_group_kernel<kKind><<<dim3((elems + 255) / 256, ngroups), 256, 0, st>>>(a.part, a.bpart, ncta);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  constexpr int outs = (kKind == 0 ? 3 : 32) * (kKind == 2 ? 1 : 32) * 9 + (kKind == 2 ? 1 : 32);
  wgrad_reduce_kernel<kKind><<<(outs + 255) / 256, 256, 0, st>>>(a.part, a.bpart, ngroups, dW, db);
  return cudaGetLastError();
}

}  // namespace

size_t conv_tc_smem(int kind, int X) {
  switch (kind) {
    case 0: return smem_bytes_for<0, 0>(X);
    case 1: return smem_bytes_for<1, 0>(X);
    case 2: return smem_bytes_for<1, 1>(X);
    default: return smem_bytes_for<1, 2>(X);
  }
}

size_t wgrad_tc_smem(int kind, int X) {
  return kind == 2 ? wgrad_smem_for<2>(X) : wgrad_smem_for<1>(X);
}

cudaError_t launch_wgrad_tc(int kind, const TcWgradArgs& a, int sms, float* dW, float* db, cudaStream_t st) {
  switch (kind) {
    case 0: return launch_wgrad_one<0>(a, sms, dW, db, st);
    case 1: return launch_wgrad_one<1>(a, sms, dW, db, st);
    default: return launch_wgrad_one<2>(a, sms, dW, db, st);
  }
}

// kind 0: layer 1 (features -> relu); 1: 32 -> 32 relu; 2: 32 -> 32 masked (input
// gradient); 3: 32 -> 1 logits.
cudaError_t launch_conv_tc(int kind, const TcConvArgs& a, int sms, cudaStream_t st) {
  switch (kind) {
    case 0: return launch_one<0, 0>(a, sms, st);
    case 1: return launch_one<1, 0>(a, sms, st);
    case 2: return launch_one<1, 1>(a, sms, st);
    default: return launch_one<1, 2>(a, sms, st);
  }
}

}  // namespace ising

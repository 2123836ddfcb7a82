// cnn.cu -- the learned proposal network: forward, backward and Adam on the GPU.
//
// A circular-padded 3x3 CNN on the torus (this project's learned stage; the
// paper's own rule is unpublished, Section III):
//   x (3 ch: s, w_right, w_down) -> conv 32 + ReLU -> conv 32 + ReLU
//     -> conv 32 + ReLU -> conv 1 = logit per site.
// Convolution: out[y,x] = b + sum W[o,c,ky,kx] in[c,(y+ky-1) mod Y,(x+kx-1) mod X].
//
// Numerics: weights are rounded to BF16, activations are stored as BF16
// [batch][site][32], and every sum accumulates in FP32.  The two 32->32
// layers (and their input gradients) are implicit GEMMs on the tensor cores:
// per output row, M = pixels, N = 32 output channels, K = 9 taps x 32 input
// channels, with the input rows (and the periodic wrap) gathered through
// shared memory and ldmatrix row addresses.  The 3->32 and 32->1 layers and
// the weight gradients run on the CUDA cores.
//
// Parameters: one flat FP32 vector in the order W1[32,3,3,3], b1[32],
// W2[32,32,3,3], b2[32], W3[32,32,3,3], b3[32], W4[1,32,3,3], b4[1].
#include <cuda_bf16.h>

#include <cmath>
#include <new>

#include "../../include/ising.h"
#include "internal.h"

namespace ising {
namespace {

constexpr int OFF_W1 = 0, OFF_B1 = 864, OFF_W2 = 896, OFF_B2 = 10112, OFF_W3 = 10144, OFF_B3 = 19360,
              OFF_W4 = 19392, OFF_B4 = 19680, NPARAM = 19681;
constexpr int PIX_STRIDE = 40;   // bf16 per pixel row in shared memory (32 + 8 padding: no bank conflicts)

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16(v)); }

// ------------------------------------------------------------------ weights
// fp32 master -> BF16-rounded copies used by the kernels:
//   w1r[864], w4r[288]          fp32 values already rounded to BF16
//   wf2/wf3 [9][32 out][40]     forward weights, BF16, [tap][out][in] (+pad)
//   wb2/wb3 [9][32 in][40]      input-gradient weights: W'[in][out][tap'] = W[out][in][8-tap]
__global__ void prepare_weights_kernel(const float* __restrict__ master, float* __restrict__ w1r,
                                       float* __restrict__ w4r, __nv_bfloat16* __restrict__ wf2,
                                       __nv_bfloat16* __restrict__ wf3, __nv_bfloat16* __restrict__ wb2,
                                       __nv_bfloat16* __restrict__ wb3) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < 864) w1r[t] = bf16r(master[OFF_W1 + t]);
  if (t < 288) w4r[t] = bf16r(master[OFF_W4 + t]);
  if (t < 9 * 32 * PIX_STRIDE) {
    const int tap = t / (32 * PIX_STRIDE);
    const int rem = t - tap * 32 * PIX_STRIDE;
    const int o = rem / PIX_STRIDE, i = rem - o * PIX_STRIDE;
    float f2 = 0.f, f3 = 0.f, b2 = 0.f, b3 = 0.f;
    if (i < 32) {
      f2 = master[OFF_W2 + (o * 32 + i) * 9 + tap];
      f3 = master[OFF_W3 + (o * 32 + i) * 9 + tap];
      // input gradient: output channel o is the forward input channel, input
      // channel i the forward output channel, taps mirrored
      b2 = master[OFF_W2 + (i * 32 + o) * 9 + (8 - tap)];
      b3 = master[OFF_W3 + (i * 32 + o) * 9 + (8 - tap)];
    }
    wf2[t] = __float2bfloat16(f2);
    wf3[t] = __float2bfloat16(f3);
    wb2[t] = __float2bfloat16(b2);
    wb3[t] = __float2bfloat16(b3);
  }
}

// ------------------------------------------------------------------ layer 1
// x = (s, w_right, w_down) at the 9 neighbours -> relu(conv + b1) as BF16.
__global__ void __launch_bounds__(256) layer1_kernel(const int8_t* __restrict__ spins,
                                                     const uint8_t* __restrict__ eflags, int B, int X, int Y,
                                                     const float* __restrict__ w1r, const float* __restrict__ master,
                                                     __nv_bfloat16* __restrict__ h1) {
  __shared__ float w[864];
  __shared__ float bias[32];
  for (int i = threadIdx.x; i < 864; i += blockDim.x) w[i] = w1r[i];
  if (threadIdx.x < 32) bias[threadIdx.x] = master[OFF_B1 + threadIdx.x];
  __syncthreads();
  const int n = X * Y;
  const long long p = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= static_cast<long long>(B) * n) return;
  const int b = static_cast<int>(p / n);
  const int site = static_cast<int>(p - static_cast<long long>(b) * n);
  const int y = site / X, x = site - y * X;
  float in[3][9];
  for (int ky = 0; ky < 3; ++ky) {
    int yy = y + ky - 1;
    yy = yy < 0 ? yy + Y : (yy >= Y ? yy - Y : yy);
    for (int kx = 0; kx < 3; ++kx) {
      int xx = x + kx - 1;
      xx = xx < 0 ? xx + X : (xx >= X ? xx - X : xx);
      const int j = yy * X + xx;
      const uint8_t f = eflags[j];
      in[0][ky * 3 + kx] = spins[static_cast<size_t>(b) * n + j] > 0 ? 1.f : -1.f;
      in[1][ky * 3 + kx] = (f & 1u) ? -1.f : 1.f;
      in[2][ky * 3 + kx] = (f & 2u) ? -1.f : 1.f;
    }
  }
  __align__(16) __nv_bfloat16 out[32];
#pragma unroll 4
  for (int o = 0; o < 32; ++o) {
    float acc = bias[o];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int t = 0; t < 9; ++t) acc = fmaf(w[(o * 3 + c) * 9 + t], in[c][t], acc);
    out[o] = __float2bfloat16(fmaxf(acc, 0.f));
  }
  uint4* dst = reinterpret_cast<uint4*>(h1 + static_cast<size_t>(p) * 32);
  const uint4* src = reinterpret_cast<const uint4*>(out);
#pragma unroll
  for (int q = 0; q < 4; ++q) dst[q] = src[q];
}

// ------------------------------------------------------------------ 32 -> 32 on tensor cores
__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float* d, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// One CTA per (image b, output row y).  mode 0: out = relu(conv + bias);
// mode 1: out = conv * [mask > 0] (input gradient through the previous ReLU).
template <int kMode>
__global__ void __launch_bounds__(256) conv32_kernel(const __nv_bfloat16* __restrict__ in,
                                                     const __nv_bfloat16* __restrict__ wt,
                                                     const float* __restrict__ bias,
                                                     const __nv_bfloat16* __restrict__ mask, int X, int Y,
                                                     __nv_bfloat16* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem[];
  __nv_bfloat16* sw = reinterpret_cast<__nv_bfloat16*>(smem);            // [9][32][40]
  __nv_bfloat16* sin = sw + 9 * 32 * PIX_STRIDE;                          // [3][X][40]
  const int b = blockIdx.y, y = blockIdx.x;
  const int n = X * Y;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // weights: 9*32 rows of 80 bytes
  for (int i = tid; i < 9 * 32 * PIX_STRIDE / 8; i += blockDim.x)
    reinterpret_cast<uint4*>(sw)[i] = reinterpret_cast<const uint4*>(wt)[i];
  // input rows y-1, y, y+1 (periodic), 64 bytes per pixel into 80-byte rows
  for (int i = tid; i < 3 * X * 4; i += blockDim.x) {
    const int r = i / (X * 4);
    const int rem = i - r * X * 4;
    const int px = rem >> 2, q = rem & 3;
    int yy = y + r - 1;
    yy = yy < 0 ? yy + Y : (yy >= Y ? yy - Y : yy);
    const uint4 v = reinterpret_cast<const uint4*>(in + (static_cast<size_t>(b) * n + yy * X + px) * 32)[q];
    reinterpret_cast<uint4*>(sin + (r * X + px) * PIX_STRIDE)[q] = v;
  }
  __syncthreads();
  const uint32_t sin_base = static_cast<uint32_t>(__cvta_generic_to_shared(sin));
  const uint32_t sw_base = static_cast<uint32_t>(__cvta_generic_to_shared(sw));
  const int mt_count = (X + 15) >> 4;
  const int g = lane >> 2, tg = lane & 3;
  for (int mt = warp; mt < mt_count; mt += 8) {
    float acc[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[nt][e] = 0.f;
    // this lane's ldmatrix row: pixel x0 + (lane & 15), channel half (lane >> 4)
    const int prow = (mt << 4) + (lane & 15);
    const int pxl = prow < X ? prow : X - 1;   // rows past the end read a valid pixel, results dropped
#pragma unroll 1
    for (int tap = 0; tap < 9; ++tap) {
      const int ky = tap / 3, kx = tap - ky * 3;
      int sx = pxl + kx - 1;
      sx = sx < 0 ? sx + X : (sx >= X ? sx - X : sx);
      const uint32_t arow = sin_base + ((ky * X + sx) * PIX_STRIDE + (lane >> 4) * 8) * 2;
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        uint32_t a0, a1, a2, a3;
        ldsm_x4(arow + ks * 32, a0, a1, a2, a3);
#pragma unroll
        for (int np = 0; np < 2; ++np) {   // two n8 tiles per ldmatrix.x4
          const int nrow = np * 16 + ((lane >> 4) << 3) + (lane & 7);
          const int kcol = ks * 16 + ((lane >> 3) & 1) * 8;
          uint32_t b0, b1, b2, b3;
          ldsm_x4(sw_base + ((tap * 32 + nrow) * PIX_STRIDE + kcol) * 2, b0, b1, b2, b3);
          mma_bf16(acc[np * 2 + 0], a0, a1, a2, a3, b0, b1);
          mma_bf16(acc[np * 2 + 1], a0, a1, a2, a3, b2, b3);
        }
      }
    }
    // epilogue: rows g and g+8 of the tile, channels nt*8 + 2tg, +1
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int px = (mt << 4) + g + half * 8;
      if (px >= X) continue;
      const size_t pix = static_cast<size_t>(b) * n + y * X + px;
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int ch = nt * 8 + 2 * tg;
        float v0 = acc[nt][half * 2 + 0], v1 = acc[nt][half * 2 + 1];
        if (kMode == 0) {
          v0 = fmaxf(v0 + bias[ch], 0.f);
          v1 = fmaxf(v1 + bias[ch + 1], 0.f);
        } else {
          const __nv_bfloat162 m = *reinterpret_cast<const __nv_bfloat162*>(mask + pix * 32 + ch);
          v0 = __bfloat162float(m.x) > 0.f ? v0 : 0.f;
          v1 = __bfloat162float(m.y) > 0.f ? v1 : 0.f;
        }
        *reinterpret_cast<__nv_bfloat162*>(out + pix * 32 + ch) = __floats2bfloat162_rn(v0, v1);
      }
    }
  }
}

// ------------------------------------------------------------------ layer 4
__global__ void __launch_bounds__(256) layer4_kernel(const __nv_bfloat16* __restrict__ h3, int B, int X, int Y,
                                                     const float* __restrict__ w4r, const float* __restrict__ master,
                                                     float* __restrict__ z) {
  __shared__ float w[288];
  for (int i = threadIdx.x; i < 288; i += blockDim.x) w[i] = w4r[i];
  __syncthreads();
  const int n = X * Y;
  const long long p = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= static_cast<long long>(B) * n) return;
  const int b = static_cast<int>(p / n);
  const int site = static_cast<int>(p - static_cast<long long>(b) * n);
  const int y = site / X, x = site - y * X;
  float acc = master[OFF_B4];
  for (int ky = 0; ky < 3; ++ky) {
    int yy = y + ky - 1;
    yy = yy < 0 ? yy + Y : (yy >= Y ? yy - Y : yy);
    for (int kx = 0; kx < 3; ++kx) {
      int xx = x + kx - 1;
      xx = xx < 0 ? xx + X : (xx >= X ? xx - X : xx);
      const uint4* src = reinterpret_cast<const uint4*>(h3 + (static_cast<size_t>(b) * n + yy * X + xx) * 32);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint4 v = src[q];
        const __nv_bfloat162* hv = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float2 f = __bfloat1622float2(hv[e]);
          const int c = q * 8 + e * 2;
          acc = fmaf(w[c * 9 + ky * 3 + kx], f.x, acc);
          acc = fmaf(w[(c + 1) * 9 + ky * 3 + kx], f.y, acc);
        }
      }
    }
  }
  z[p] = acc;
}

// ------------------------------------------------------------------ loss
// dz = (sigmoid(z) - y) / N; loss += softplus(z) - y z (stable form), / N
__global__ void __launch_bounds__(256) loss_kernel(const float* __restrict__ z, const uint8_t* __restrict__ tgt,
                                                   long long N, float* __restrict__ dz, float* __restrict__ loss) {
  __shared__ float red[8];
  const long long p = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (p < N) {
    const float v = z[p];
    const float yv = tgt[p] ? 1.f : 0.f;
    const float sg = 1.f / (1.f + expf(-v));
    dz[p] = (sg - yv) / static_cast<float>(N);
    l = (fmaxf(v, 0.f) - v * yv + log1pf(expf(-fabsf(v)))) / static_cast<float>(N);
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xFFFFFFFFu, l, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < 8; ++w) t += red[w];
    atomicAdd(loss, t);
  }
}

// ------------------------------------------------------------------ layer 4 backward
// g3[p][c] = [h3[p][c] > 0] * sum_tap W4[c][tap] dz[p - tap + 1]
__global__ void __launch_bounds__(256) layer4_back_kernel(const float* __restrict__ dz,
                                                          const __nv_bfloat16* __restrict__ h3, int B, int X, int Y,
                                                          const float* __restrict__ w4r,
                                                          __nv_bfloat16* __restrict__ g3) {
  __shared__ float w[288];
  for (int i = threadIdx.x; i < 288; i += blockDim.x) w[i] = w4r[i];
  __syncthreads();
  const int n = X * Y;
  const long long p = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= static_cast<long long>(B) * n) return;
  const int b = static_cast<int>(p / n);
  const int site = static_cast<int>(p - static_cast<long long>(b) * n);
  const int y = site / X, x = site - y * X;
  float d[9];
  for (int ky = 0; ky < 3; ++ky) {
    int yy = y - ky + 1;
    yy = yy < 0 ? yy + Y : (yy >= Y ? yy - Y : yy);
    for (int kx = 0; kx < 3; ++kx) {
      int xx = x - kx + 1;
      xx = xx < 0 ? xx + X : (xx >= X ? xx - X : xx);
      d[ky * 3 + kx] = dz[static_cast<size_t>(b) * n + yy * X + xx];
    }
  }
  const __nv_bfloat16* hp = h3 + static_cast<size_t>(p) * 32;
  __align__(16) __nv_bfloat16 out[32];
#pragma unroll 4
  for (int c = 0; c < 32; ++c) {
    float acc = 0.f;
#pragma unroll
    for (int t = 0; t < 9; ++t) acc = fmaf(w[c * 9 + t], d[t], acc);
    out[c] = __float2bfloat16(__bfloat162float(hp[c]) > 0.f ? acc : 0.f);
  }
  uint4* dst = reinterpret_cast<uint4*>(g3 + static_cast<size_t>(p) * 32);
  const uint4* src = reinterpret_cast<const uint4*>(out);
#pragma unroll
  for (int q = 0; q < 4; ++q) dst[q] = src[q];
}

// ------------------------------------------------------------------ weight gradients (CUDA cores)
// dW[o][c][tap] += sum_p g[p][o] * a[p + tap - 1][c], db[o] += sum_p g[p][o], over
// kRows output rows of one image per CTA.  Inputs:
//   kind 0: a = features of (spins, eflags) (3 channels), g BF16 [32]   (layer 1)
//   kind 1: a = BF16 [32], g BF16 [32]                                   (layers 2, 3)
//   kind 2: a = BF16 [32], g = dz FP32 [1]                               (layer 4)
// Thread t owns outputs t, t + 256, ... of the layer's O*C*9 weights.
template <int kKind>
__global__ void __launch_bounds__(256) wgrad_kernel(const void* __restrict__ gsrc, const __nv_bfloat16* __restrict__ act,
                                                    const int8_t* __restrict__ spins,
                                                    const uint8_t* __restrict__ eflags, int B, int X, int Y,
                                                    int rows_per_cta, float* __restrict__ dW, float* __restrict__ db) {
  constexpr int C = kKind == 0 ? 3 : 32;
  constexpr int O = kKind == 2 ? 1 : 32;
  constexpr int NW = O * C * 9;
  constexpr int PER = (NW + 255) / 256;
  extern __shared__ __align__(16) float sm[];
  float* sa = sm;                       // [3][X][C] activations of rows y-1, y, y+1
  float* sg = sa + 3 * X * C;           // [X][O] gradients of row y
  const int n = X * Y;
  const int b = blockIdx.y;
  float acc[PER];
#pragma unroll
  for (int e = 0; e < PER; ++e) acc[e] = 0.f;
  float bacc = 0.f;
  const int y_begin = blockIdx.x * rows_per_cta;
  const int y_end = min(Y, y_begin + rows_per_cta);
  for (int y = y_begin; y < y_end; ++y) {
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * X * C; i += blockDim.x) {
      const int r = i / (X * C);
      const int rem = i - r * X * C;
      const int px = rem / C, c = rem - px * C;
      int yy = y + r - 1;
      yy = yy < 0 ? yy + Y : (yy >= Y ? yy - Y : yy);
      const int j = yy * X + px;
      float v;
      if (kKind == 0) {
        if (c == 0) v = spins[static_cast<size_t>(b) * n + j] > 0 ? 1.f : -1.f;
        else v = (eflags[j] & (c == 1 ? 1u : 2u)) ? -1.f : 1.f;
      } else {
        v = __bfloat162float(act[(static_cast<size_t>(b) * n + j) * 32 + c]);
      }
      sa[i] = v;
    }
    for (int i = threadIdx.x; i < X * O; i += blockDim.x) {
      const int px = i / O, o = i - px * O;
      const size_t q = static_cast<size_t>(b) * n + y * X + px;
      sg[i] = kKind == 2 ? static_cast<const float*>(gsrc)[q]
                         : __bfloat162float(static_cast<const __nv_bfloat16*>(gsrc)[q * 32 + o]);
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < PER; ++e) {
      const int wi = threadIdx.x + e * 256;
      if (wi < NW) {
        const int o = wi / (C * 9);
        const int rem = wi - o * C * 9;
        const int c = rem / 9, tap = rem - c * 9;
        const int ky = tap / 3, kx = tap - ky * 3;
        float s = 0.f;
        for (int px = 0; px < X; ++px) {
          int sx = px + kx - 1;
          sx = sx < 0 ? sx + X : (sx >= X ? sx - X : sx);
          s = fmaf(sg[px * O + o], sa[(ky * X + sx) * C + c], s);
        }
        acc[e] += s;
      }
    }
    if (threadIdx.x < O) {
      float s = 0.f;
      for (int px = 0; px < X; ++px) s += sg[px * O + threadIdx.x];
      bacc += s;
    }
  }
#pragma unroll
  for (int e = 0; e < PER; ++e) {
    const int wi = threadIdx.x + e * 256;
    if (wi < NW) atomicAdd(dW + wi, acc[e]);
  }
  if (threadIdx.x < O) atomicAdd(db + threadIdx.x, bacc);
}

// ------------------------------------------------------------------ Adam
__global__ void adam_kernel(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, int count, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace
}  // namespace ising

// ======================================================================= ABI
struct ising_cnn {
  float* master = nullptr;   // [NPARAM]
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  float* w1r = nullptr;      // [864]
  float* w4r = nullptr;      // [288]
  __nv_bfloat16* wf2 = nullptr;
  __nv_bfloat16* wf3 = nullptr;
  __nv_bfloat16* wb2 = nullptr;
  __nv_bfloat16* wb3 = nullptr;
  int64_t step = 0;
};

namespace {

using namespace ising;

int cnn_map(cudaError_t e) {
  if (e == cudaSuccess) return ISING_OK;
  if (e == cudaErrorMemoryAllocation) return ISING_ERR_OOM;
  return ISING_ERR_CUDA;
}

constexpr size_t kWT = 9 * 32 * PIX_STRIDE;   // bf16 elements per prepared 32x32 weight set

cudaError_t refresh(ising_cnn* net, cudaStream_t st) {
  prepare_weights_kernel<<<(static_cast<int>(kWT) + 255) / 256, 256, 0, st>>>(net->master, net->w1r, net->w4r,
                                                                                net->wf2, net->wf3, net->wb2,
                                                                                net->wb3);
  return cudaGetLastError();
}

size_t act_bytes(int32_t B, int32_t n) { return static_cast<size_t>(B) * n * 32 * sizeof(__nv_bfloat16); }
size_t al256(size_t v) { return (v + 255) & ~size_t(255); }

// workspace: h1, h2, h3 (BF16 [B][n][32]); for training also z, dz (FP32 [B][n]),
// g3, g2, g1 (BF16 [B][n][32])
struct WS {
  __nv_bfloat16 *h1, *h2, *h3, *g1, *g2, *g3;
  float *z, *dz;
};

size_t ws_layout(int32_t B, int32_t n, int train, WS* w, unsigned char* base) {
  size_t o = 0;
  const size_t A = al256(act_bytes(B, n));
  const size_t Z = al256(static_cast<size_t>(B) * n * sizeof(float));
  auto take = [&](size_t bytes) {
    unsigned char* p = base ? base + o : nullptr;
    o += bytes;
    return p;
  };
  WS t{};
  t.h1 = reinterpret_cast<__nv_bfloat16*>(take(A));
  t.h2 = reinterpret_cast<__nv_bfloat16*>(take(A));
  t.h3 = reinterpret_cast<__nv_bfloat16*>(take(A));
  if (train) {
    t.z = reinterpret_cast<float*>(take(Z));
    t.dz = reinterpret_cast<float*>(take(Z));
    t.g3 = reinterpret_cast<__nv_bfloat16*>(take(A));
    t.g2 = reinterpret_cast<__nv_bfloat16*>(take(A));
    t.g1 = reinterpret_cast<__nv_bfloat16*>(take(A));
  }
  if (w) *w = t;
  return o;
}

size_t conv_smem(int X) { return (9 * 32 + 3 * static_cast<size_t>(X)) * PIX_STRIDE * sizeof(__nv_bfloat16); }

cudaError_t forward_pass(const ising_cnn* net, const ising_problem* p, const int8_t* spins, int32_t B, float* z,
                         const WS& w, cudaStream_t st) {
  const long long N = static_cast<long long>(B) * p->n;
  const int blocks = static_cast<int>((N + 255) / 256);
  layer1_kernel<<<blocks, 256, 0, st>>>(spins, p->d_eflags, B, p->X, p->Y, net->w1r, net->master, w.h1);
  const size_t sm = conv_smem(p->X);
  cudaError_t e = cudaFuncSetAttribute(conv32_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(sm));
  if (e != cudaSuccess) return e;
  const dim3 grid(p->Y, B);
  conv32_kernel<0><<<grid, 256, sm, st>>>(w.h1, net->wf2, net->master + OFF_B2, nullptr, p->X, p->Y, w.h2);
  conv32_kernel<0><<<grid, 256, sm, st>>>(w.h2, net->wf3, net->master + OFF_B3, nullptr, p->X, p->Y, w.h3);
  layer4_kernel<<<blocks, 256, 0, st>>>(w.h3, B, p->X, p->Y, net->w4r, net->master, z);
  return cudaGetLastError();
}

}  // namespace

extern "C" {

int ising_cnn_create(const float* params, ising_cnn** out) {
  if (!params || !out) return ISING_ERR_ARG;
  ising_cnn* net = new (std::nothrow) ising_cnn();
  if (!net) return ISING_ERR_OOM;
  cudaError_t e = cudaMalloc(&net->master, NPARAM * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&net->adam_m, NPARAM * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&net->adam_v, NPARAM * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&net->w1r, 864 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&net->w4r, 288 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&net->wf2, kWT * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMalloc(&net->wf3, kWT * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMalloc(&net->wb2, kWT * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMalloc(&net->wb3, kWT * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMemcpy(net->master, params, NPARAM * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(net->adam_m, 0, NPARAM * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(net->adam_v, 0, NPARAM * sizeof(float));
  if (e == cudaSuccess) e = refresh(net, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    ising_cnn_destroy(net);
    return cnn_map(e);
  }
  *out = net;
  return ISING_OK;
}

void ising_cnn_destroy(ising_cnn* net) {
  if (!net) return;
  cudaFree(net->master);
  cudaFree(net->adam_m);
  cudaFree(net->adam_v);
  cudaFree(net->w1r);
  cudaFree(net->w4r);
  cudaFree(net->wf2);
  cudaFree(net->wf3);
  cudaFree(net->wb2);
  cudaFree(net->wb3);
  delete net;
}

int ising_cnn_get_params(const ising_cnn* net, float* params) {
  if (!net || !params) return ISING_ERR_ARG;
  return cnn_map(cudaMemcpy(params, net->master, NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
}

int ising_cnn_set_params(ising_cnn* net, const float* params) {
  if (!net || !params) return ISING_ERR_ARG;
  cudaError_t e = cudaMemcpy(net->master, params, NPARAM * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(net->adam_m, 0, NPARAM * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(net->adam_v, 0, NPARAM * sizeof(float));
  if (e == cudaSuccess) e = refresh(net, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  net->step = 0;
  return cnn_map(e);
}

size_t ising_cnn_workspace_bytes(int32_t B, int32_t n, int32_t train) {
  if (B <= 0 || n <= 0) return 0;
  return ws_layout(B, n, train, nullptr, nullptr);
}

int ising_cnn_forward(const ising_cnn* net, const ising_problem* p, const int8_t* spins, int32_t B, float* logits,
                      void* ws, size_t ws_bytes, void* cuda_stream) {
  if (!net || !p || B < 0 || (B > 0 && (!spins || !logits || !ws))) return ISING_ERR_ARG;
  if (B == 0) return ISING_OK;
  if (ws_bytes < ws_layout(B, p->n, 0, nullptr, nullptr)) return ISING_ERR_ARG;
  if (conv_smem(p->X) > 227 * 1024) return ISING_ERR_UNSUPPORTED;
  WS w;
  ws_layout(B, p->n, 0, &w, static_cast<unsigned char*>(ws));
  return cnn_map(forward_pass(net, p, spins, B, logits, w, static_cast<cudaStream_t>(cuda_stream)));
}

int ising_cnn_grad(const ising_cnn* net, const ising_problem* p, const int8_t* spins, const uint8_t* targets,
                   int32_t B, float* grad, float* loss, void* ws, size_t ws_bytes, void* cuda_stream) {
  if (!net || !p || B <= 0 || !spins || !targets || !grad || !loss || !ws) return ISING_ERR_ARG;
  if (ws_bytes < ws_layout(B, p->n, 1, nullptr, nullptr)) return ISING_ERR_ARG;
  if (conv_smem(p->X) > 227 * 1024) return ISING_ERR_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  WS w;
  ws_layout(B, p->n, 1, &w, static_cast<unsigned char*>(ws));
  cudaError_t e = cudaMemsetAsync(grad, 0, NPARAM * sizeof(float), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, sizeof(float), st);
  if (e == cudaSuccess) e = forward_pass(net, p, spins, B, w.z, w, st);
  if (e != cudaSuccess) return cnn_map(e);
  const long long N = static_cast<long long>(B) * p->n;
  const int blocks = static_cast<int>((N + 255) / 256);
  const int X = p->X, Y = p->Y;
  loss_kernel<<<blocks, 256, 0, st>>>(w.z, targets, N, w.dz, loss);
  layer4_back_kernel<<<blocks, 256, 0, st>>>(w.dz, w.h3, B, X, Y, net->w4r, w.g3);
  const size_t sm = conv_smem(X);
  e = cudaFuncSetAttribute(conv32_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
  if (e != cudaSuccess) return cnn_map(e);
  const dim3 grid(Y, B);
  conv32_kernel<1><<<grid, 256, sm, st>>>(w.g3, net->wb3, nullptr, w.h2, X, Y, w.g2);
  conv32_kernel<1><<<grid, 256, sm, st>>>(w.g2, net->wb2, nullptr, w.h1, X, Y, w.g1);
  // weight gradients
  const int rows = 4;
  const dim3 wgrid((Y + rows - 1) / rows, B);
  const size_t sm32 = (3 * static_cast<size_t>(X) * 32 + static_cast<size_t>(X) * 32) * sizeof(float);
  const size_t sm4 = (3 * static_cast<size_t>(X) * 32 + static_cast<size_t>(X) * 1) * sizeof(float);
  const size_t sm1 = (3 * static_cast<size_t>(X) * 3 + static_cast<size_t>(X) * 32) * sizeof(float);
  if (sm32 > 227 * 1024) return ISING_ERR_UNSUPPORTED;
  e = cudaFuncSetAttribute(wgrad_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm32));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(wgrad_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm4));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(wgrad_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm1));
  if (e != cudaSuccess) return cnn_map(e);
  wgrad_kernel<2><<<wgrid, 256, sm4, st>>>(w.dz, w.h3, nullptr, nullptr, B, X, Y, rows, grad + OFF_W4, grad + OFF_B4);
  wgrad_kernel<1><<<wgrid, 256, sm32, st>>>(w.g3, w.h2, nullptr, nullptr, B, X, Y, rows, grad + OFF_W3, grad + OFF_B3);
  wgrad_kernel<1><<<wgrid, 256, sm32, st>>>(w.g2, w.h1, nullptr, nullptr, B, X, Y, rows, grad + OFF_W2, grad + OFF_B2);
  wgrad_kernel<0><<<wgrid, 256, sm1, st>>>(w.g1, nullptr, spins, p->d_eflags, B, X, Y, rows, grad + OFF_W1,
                                           grad + OFF_B1);
  return cnn_map(cudaGetLastError());
}

int ising_cnn_adam_step(ising_cnn* net, const float* grad, float lr, float beta1, float beta2, float eps,
                        void* cuda_stream) {
  if (!net || !grad || !(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) ||
      !(eps > 0.f))
    return ISING_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  net->step += 1;
  const float c1 = 1.f - std::pow(beta1, static_cast<float>(net->step));
  const float c2 = 1.f - std::pow(beta2, static_cast<float>(net->step));
  adam_kernel<<<(NPARAM + 255) / 256, 256, 0, st>>>(net->master, net->adam_m, net->adam_v, grad, NPARAM, lr, beta1,
                                                     beta2, eps, c1, c2);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = refresh(net, st);
  return cnn_map(e);
}

}  // extern "C"

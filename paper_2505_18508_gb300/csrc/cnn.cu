// cnn.cu -- the learned proposal network: forward, backward and Adam on the GPU.
//
// A circular-padded 3x3 CNN on the torus (this project's learned stage; the
// paper's own rule is unpublished, Section III):
//   x (3 ch: s, w_right, w_down) -> conv 32 + ReLU -> conv 32 + ReLU
//     -> conv 32 + ReLU -> conv 1 = logit per site.
// Convolution: out[y,x] = b + sum W[o,c,ky,kx] in[c,(y+ky-1) mod Y,(x+kx-1) mod X].
//
// Numerics: weights are rounded to BF16, activations are stored as BF16
// [batch][site][32], and every sum accumulates in FP32.  All four forward
// convolutions and the two 32->32 input gradients are implicit GEMMs on the
// tcgen05 tensor cores (conv_tc.cu: per output row, M = pixels, N = output
// channels, K = 9 taps x input channels, accumulators in tensor memory).  The
// weight gradients are tensor-core GEMMs over the pixels as well; the layer-4
// input gradient and the loss run on the CUDA cores.
//
// Parameters: one flat FP32 vector in the order W1[32,3,3,3], b1[32],
// W2[32,32,3,3], b2[32], W3[32,32,3,3], b3[32], W4[1,32,3,3], b4[1].
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <new>

#include "../../include/ising.h"
#include "internal.h"

namespace ising {
namespace {

constexpr int OFF_W1 = 0, OFF_B1 = 864, OFF_W2 = 896, OFF_B2 = 10112, OFF_W3 = 10144, OFF_B3 = 19360,
              OFF_W4 = 19392, OFF_B4 = 19680, NPARAM = 19681;

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16(v)); }

// ------------------------------------------------------------------ weights
// fp32 master -> the copies the kernels read: w4r[288], W4 rounded to BF16
// (held in fp32) for the layer-4 backward, and the BF16 tensor-core operands.
__global__ void prepare_w4r_kernel(const float* __restrict__ master, float* __restrict__ w4r) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < 288) w4r[t] = bf16r(master[OFF_W4 + t]);
}

// Canonical tensor-core layouts: element (tap, k, n) at
// (((tap*KC + k/8)*NG + n/8)*8 + n%8)*8 + k%8, KC = K/8 input chunks, NG = N/8.
__device__ __forceinline__ int tc_index(int tap, int k, int n, int KC, int NG) {
  return (((tap * KC + (k >> 3)) * NG + (n >> 3)) * 8 + (n & 7)) * 8 + (k & 7);
}

// tc1: layer 1 (K = 16 with 3 used, N = 32); tc2f/tc3f: forward 32 -> 32;
// tc2b/tc3b: input gradients W'[in][out][tap'] = W[out][in][8 - tap'];
// tc4: layer 4 (K = 32, N = 16 with 1 used)
__global__ void prepare_tc_weights_kernel(const float* __restrict__ master, __nv_bfloat16* __restrict__ tc1,
                                          __nv_bfloat16* __restrict__ tc2f, __nv_bfloat16* __restrict__ tc3f,
                                          __nv_bfloat16* __restrict__ tc2b, __nv_bfloat16* __restrict__ tc3b,
                                          __nv_bfloat16* __restrict__ tc4) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < 9 * 16 * 32) {                       // (tap, k < 16, n < 32)
    const int tap = t / 512, rem = t - tap * 512, k = rem / 32, n = rem - k * 32;
    tc1[tc_index(tap, k, n, 2, 4)] = __float2bfloat16(k < 3 ? master[OFF_W1 + (n * 3 + k) * 9 + tap] : 0.f);
  }
  if (t < 9 * 32 * 32) {                       // (tap, k < 32, n < 32)
    const int tap = t / 1024, rem = t - tap * 1024, k = rem / 32, n = rem - k * 32;
    const int i = tc_index(tap, k, n, 4, 4);
    tc2f[i] = __float2bfloat16(master[OFF_W2 + (n * 32 + k) * 9 + tap]);
    tc3f[i] = __float2bfloat16(master[OFF_W3 + (n * 32 + k) * 9 + tap]);
    tc2b[i] = __float2bfloat16(master[OFF_W2 + (k * 32 + n) * 9 + (8 - tap)]);
    tc3b[i] = __float2bfloat16(master[OFF_W3 + (k * 32 + n) * 9 + (8 - tap)]);
  }
  if (t < 9 * 32 * 16) {                       // (tap, k < 32, n < 16)
    const int tap = t / 512, rem = t - tap * 512, k = rem / 16, n = rem - k * 16;
    tc4[tc_index(tap, k, n, 4, 2)] = __float2bfloat16(n == 0 ? master[OFF_W4 + k * 9 + tap] : 0.f);
  }
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
// g3[p][c] = [h3[p][c] > 0] * sum_tap W4[c][tap] dz[p - tap + 1].  One thread
// per (pixel, 8-channel chunk): a warp reads and writes 8 whole pixels
// (512 contiguous bytes) of h3 and g3.
__global__ void __launch_bounds__(256) layer4_back_kernel(const float* __restrict__ dz,
                                                          const __nv_bfloat16* __restrict__ h3, int B, int X, int Y,
                                                          const float* __restrict__ w4r,
                                                          __nv_bfloat16* __restrict__ g3) {
  __shared__ float w[288];
  for (int i = threadIdx.x; i < 288; i += blockDim.x) w[i] = w4r[i];
  __syncthreads();
  const int n = X * Y;
  const long long q = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= static_cast<long long>(B) * n * 4) return;
  const long long p = q >> 2;
  const int ch = static_cast<int>(q & 3);
  const int b = static_cast<int>(p / n);
  const int site = static_cast<int>(p - static_cast<long long>(b) * n);
  const int y = site / X, x = site - y * X;
  float d[9];
#pragma unroll
  for (int ky = 0; ky < 3; ++ky) {
    int yy = y - ky + 1;
    yy = yy < 0 ? yy + Y : (yy >= Y ? yy - Y : yy);
#pragma unroll
    for (int kx = 0; kx < 3; ++kx) {
      int xx = x - kx + 1;
      xx = xx < 0 ? xx + X : (xx >= X ? xx - X : xx);
      d[ky * 3 + kx] = dz[static_cast<size_t>(b) * n + yy * X + xx];
    }
  }
  const uint4 hv = reinterpret_cast<const uint4*>(h3 + static_cast<size_t>(p) * 32)[ch];
  const __nv_bfloat16* hp = reinterpret_cast<const __nv_bfloat16*>(&hv);
  __align__(16) __nv_bfloat16 out[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int c = ch * 8 + e;
    float acc = 0.f;
#pragma unroll
    for (int t = 0; t < 9; ++t) acc = fmaf(w[c * 9 + t], d[t], acc);
    out[e] = __float2bfloat16(__bfloat162float(hp[e]) > 0.f ? acc : 0.f);
  }
  reinterpret_cast<uint4*>(g3 + static_cast<size_t>(p) * 32)[ch] = *reinterpret_cast<const uint4*>(out);
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
  float* w4r = nullptr;      // [288]
  __nv_bfloat16* tc1 = nullptr;    // canonical tensor-core layouts
  __nv_bfloat16* tc2f = nullptr;
  __nv_bfloat16* tc3f = nullptr;
  __nv_bfloat16* tc2b = nullptr;
  __nv_bfloat16* tc3b = nullptr;
  __nv_bfloat16* tc4 = nullptr;
  int64_t step = 0;
  long long wait_limit = 0;   // cycles one tensor-core wait may take (0: about two seconds)
  int32_t stall_test = 0;     // 1: CTA 0 of every tensor-core launch waits once on a barrier nothing arrives at
};

namespace {

using namespace ising;

int cnn_map(cudaError_t e) {
  if (e == cudaSuccess) return ISING_OK;
  if (e == cudaErrorMemoryAllocation) return ISING_ERR_OOM;
  return ISING_ERR_CUDA;
}


cudaError_t refresh(ising_cnn* net, cudaStream_t st) {
  prepare_w4r_kernel<<<2, 256, 0, st>>>(net->master, net->w4r);
  prepare_tc_weights_kernel<<<(9 * 32 * 32 + 255) / 256, 256, 0, st>>>(net->master, net->tc1, net->tc2f, net->tc3f,
                                                                       net->tc2b, net->tc3b, net->tc4);
  return cudaGetLastError();
}

int sm_count() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      v <= 0)
    v = 152;
  return v;
}

TcConvArgs tc_args(const ising_cnn* net, const ising_problem* p, int32_t B) {
  TcConvArgs a{};
  a.X = p->X;
  a.Y = p->Y;
  a.B = B;
  a.eflags = p->d_eflags;
  a.status = p->d_status;
  a.wait_limit = net->wait_limit;
  a.stall_test = net->stall_test;
  return a;
}

size_t act_bytes(int32_t B, int32_t n) { return static_cast<size_t>(B) * n * 32 * sizeof(__nv_bfloat16); }
size_t al256(size_t v) { return (v + 255) & ~size_t(255); }

// workspace: h1, h2, h3 (BF16 [B][n][32]); for training also z, dz (FP32 [B][n]),
// g3, g2, g1 (BF16 [B][n][32])
struct WS {
  __nv_bfloat16 *h1, *h2, *h3, *g1, *g2, *g3;
  float *z, *dz, *part, *bpart;
  int max_ctas;
};

// CTAs of one weight-gradient launch: at most one per output row (B*Y <= B*n/4
// since X >= 4) and at most kWgradMaxCtas
int wgrad_ctas(int32_t B, int32_t n) {
  const long long rows = std::max<long long>(1, static_cast<long long>(B) * n / 4);
  return static_cast<int>(std::min<long long>(rows, kWgradMaxCtas));
}

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
    t.max_ctas = wgrad_ctas(B, n);
    t.part = reinterpret_cast<float*>(take(al256(static_cast<size_t>(t.max_ctas) * 96 * 96 * sizeof(float))));
    t.bpart = reinterpret_cast<float*>(take(al256(static_cast<size_t>(t.max_ctas) * 32 * sizeof(float))));
  }
  if (w) *w = t;
  return o;
}

cudaError_t forward_pass(const ising_cnn* net, const ising_problem* p, const int8_t* spins, int32_t B, float* z,
                         const WS& w, cudaStream_t st) {
  const int sms = sm_count();
  TcConvArgs a = tc_args(net, p, B);
  a.spins = spins;
  a.wt = net->tc1;
  a.bias = net->master + OFF_B1;
  a.out_bf16 = w.h1;
  cudaError_t e = launch_conv_tc(0, a, sms, st);
  if (e != cudaSuccess) return e;
  a = tc_args(net, p, B);
  a.in = w.h1;
  a.wt = net->tc2f;
  a.bias = net->master + OFF_B2;
  a.out_bf16 = w.h2;
  e = launch_conv_tc(1, a, sms, st);
  if (e != cudaSuccess) return e;
  a.in = w.h2;
  a.wt = net->tc3f;
  a.bias = net->master + OFF_B3;
  a.out_bf16 = w.h3;
  e = launch_conv_tc(1, a, sms, st);
  if (e != cudaSuccess) return e;
  a = tc_args(net, p, B);
  a.in = w.h3;
  a.wt = net->tc4;
  a.bias = net->master + OFF_B4;
  a.out_f32 = z;
  return launch_conv_tc(3, a, sms, st);
}

bool tc_supported(const ising_problem* p) {
  // four 32-column accumulators per 128-pixel tile within 512 tensor-memory columns
  return p->X <= 512 && conv_tc_smem(1, p->X) <= 227 * 1024;
}

}  // namespace

namespace ising {

int cnn_forward_ws(const ising_cnn* net, const ising_problem* p, const int8_t* spins, int32_t B, float* logits,
                   void* ws, size_t ws_bytes, cudaStream_t st) {
  if (!net || !p || B < 0 || (B > 0 && (!spins || !logits || !ws))) return ISING_ERR_ARG;
  if (p->graph) return ISING_ERR_UNSUPPORTED;   // the network reads the torus layout
  if (B == 0) return ISING_OK;
  if (ws_bytes < ws_layout(B, p->n, 0, nullptr, nullptr)) return ISING_ERR_ARG;
  if (!tc_supported(p)) return ISING_ERR_UNSUPPORTED;
  WS w;
  ws_layout(B, p->n, 0, &w, static_cast<unsigned char*>(ws));
  return cnn_map(forward_pass(net, p, spins, B, logits, w, st));
}

}  // namespace ising

extern "C" {

int ising_cnn_create(const float* params, ising_cnn** out) {
  if (!params || !out) return ISING_ERR_ARG;
  ising_cnn* net = new (std::nothrow) ising_cnn();
  if (!net) return ISING_ERR_OOM;
  cudaError_t e = ising::dev_malloc(&net->master, NPARAM * sizeof(float));
  if (e == cudaSuccess) e = ising::dev_malloc(&net->adam_m, NPARAM * sizeof(float));
  if (e == cudaSuccess) e = ising::dev_malloc(&net->adam_v, NPARAM * sizeof(float));
  if (e == cudaSuccess) e = ising::dev_malloc(&net->w4r, 288 * sizeof(float));
  if (e == cudaSuccess) e = ising::dev_malloc(&net->tc1, 9 * 16 * 32 * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = ising::dev_malloc(&net->tc2f, 9 * 32 * 32 * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = ising::dev_malloc(&net->tc3f, 9 * 32 * 32 * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = ising::dev_malloc(&net->tc2b, 9 * 32 * 32 * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = ising::dev_malloc(&net->tc3b, 9 * 32 * 32 * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = ising::dev_malloc(&net->tc4, 9 * 32 * 16 * sizeof(__nv_bfloat16));
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
  cudaFree(net->w4r);
  cudaFree(net->tc1);
  cudaFree(net->tc2f);
  cudaFree(net->tc3f);
  cudaFree(net->tc2b);
  cudaFree(net->tc3b);
  cudaFree(net->tc4);
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
  return ising::cnn_forward_ws(net, p, spins, B, logits, ws, ws_bytes, static_cast<cudaStream_t>(cuda_stream));
}

int ising_cnn_grad(const ising_cnn* net, const ising_problem* p, const int8_t* spins, const uint8_t* targets,
                   int32_t B, float* grad, float* loss, void* ws, size_t ws_bytes, void* cuda_stream) {
  if (!net || !p || B <= 0 || !spins || !targets || !grad || !loss || !ws) return ISING_ERR_ARG;
  if (p->graph) return ISING_ERR_UNSUPPORTED;
  if (ws_bytes < ws_layout(B, p->n, 1, nullptr, nullptr)) return ISING_ERR_ARG;
  if (!tc_supported(p) || wgrad_tc_smem(1, p->X) > 227 * 1024) return ISING_ERR_UNSUPPORTED;
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
  layer4_back_kernel<<<static_cast<int>((4 * N + 255) / 256), 256, 0, st>>>(w.dz, w.h3, B, X, Y, net->w4r, w.g3);
  {
    TcConvArgs a = tc_args(net, p, B);
    a.in = w.g3;
    a.wt = net->tc3b;
    a.mask = w.h2;
    a.out_bf16 = w.g2;
    e = launch_conv_tc(2, a, sm_count(), st);
    if (e == cudaSuccess) {
      a.in = w.g2;
      a.wt = net->tc2b;
      a.mask = w.h1;
      a.out_bf16 = w.g1;
      e = launch_conv_tc(2, a, sm_count(), st);
    }
    if (e != cudaSuccess) return cnn_map(e);
  }
  // weight gradients (tensor cores), layer 4 first
  {
    TcWgradArgs a{};
    a.X = X;
    a.Y = Y;
    a.B = B;
    a.part = w.part;
    a.bpart = w.bpart;
    a.status = p->d_status;
    a.max_ctas = w.max_ctas;
    a.wait_limit = net->wait_limit;
    a.stall_test = net->stall_test;
    const int sms = sm_count();
    a.act = w.h3;
    a.g = w.dz;
    e = launch_wgrad_tc(2, a, sms, grad + OFF_W4, grad + OFF_B4, st);
    if (e == cudaSuccess) {
      a.act = w.h2;
      a.g = w.g3;
      e = launch_wgrad_tc(1, a, sms, grad + OFF_W3, grad + OFF_B3, st);
    }
    if (e == cudaSuccess) {
      a.act = w.h1;
      a.g = w.g2;
      e = launch_wgrad_tc(1, a, sms, grad + OFF_W2, grad + OFF_B2, st);
    }
    if (e == cudaSuccess) {
      a.act = nullptr;
      a.spins = spins;
      a.eflags = p->d_eflags;
      a.g = w.g1;
      e = launch_wgrad_tc(0, a, sms, grad + OFF_W1, grad + OFF_B1, st);
    }
    if (e != cudaSuccess) return cnn_map(e);
  }
  return cnn_map(cudaGetLastError());
}

int ising_cnn_set_wait_limit(ising_cnn* net, int64_t cycles, int32_t stall_test) {
  if (!net || cycles < 0 || stall_test < 0 || stall_test > 1) return ISING_ERR_ARG;
  net->wait_limit = cycles;
  net->stall_test = stall_test;
  return ISING_OK;
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

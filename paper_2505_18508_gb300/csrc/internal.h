// internal.h -- host-side structures shared by the ABI and the kernel launchers.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/ising.h"

struct ising_problem {
  int32_t X = 0, Y = 0, n = 0, H = 0;   // H = X / 2 sites per colour per row
  int32_t neg_edges = 0;                // edges with w = -1
  int32_t weight_sum = 0;               // W = sum of w over the 2n edges
  int device = 0;
  // Plane-order site flags, index (c*Y + y)*H + h for the site of colour c in
  // row y at x = 2h + ((y + c) & 1): bit0 left edge w=-1, bit1 right, bit2 up,
  // bit3 down.
  uint8_t* d_flags = nullptr;
  // Natural-order edge flags, index y*X + x: bit0 right edge w=-1, bit1 down.
  uint8_t* d_eflags = nullptr;
  // device status word: bounded waits that ran out leave ISING_ERR_TIMEOUT here
  int32_t* d_status = nullptr;
  // launch overrides (0 = automatic) and the last shape used
  int32_t cfg_group = 0, cfg_strips = 0, cfg_threads = 0, cfg_kernel = 0;
  int32_t cfg_graph_tpw = 0;       // general graphs: threads per site word (0: automatic)
  int32_t draw_bits = 32;   // 32: the default decision stream; 16: the 16-bit draw mode
  int32_t last_group = 0, last_strips = 0, last_threads = 0, last_grid = 0, last_kernel = 0;
  // bounded-wait limit (cycles) and the forced-stall switch used by tests
  long long wait_limit = 0;
  int32_t stall_test = 0;
  // general sparse graph (ising_graph_create); X = Y = 0 then
  int32_t graph = 0;
  int32_t ncol = 0, Dmax = 0, planes = 0;
  int64_t nnz = 0;
  uint32_t* d_nb = nullptr;        // [nnz] col | (J < 0) << 24 | (|J| - 1) << 25
  int4* d_rowinfo = nullptr;       // [n] {first entry, degree, h, D = sum |J| + |h|}
  int32_t* d_sites = nullptr;      // [n] sites by colour class, increasing index within a class
  int32_t* d_colour_off = nullptr; // [ncol + 1]
};

namespace ising {

// host_util.cu: device allocations through a test hook (ising_debug_fail_allocs)
// and the ISING_LOG level
cudaError_t dev_malloc(void** p, size_t bytes);
cudaError_t dev_malloc_async(void** p, size_t bytes, cudaStream_t st);
template <typename T>
inline cudaError_t dev_malloc(T** p, size_t bytes) {
  return dev_malloc(reinterpret_cast<void**>(p), bytes);
}
template <typename T>
inline cudaError_t dev_malloc_async(T** p, size_t bytes, cudaStream_t st) {
  return dev_malloc_async(reinterpret_cast<void**>(p), bytes, st);
}
int log_level();
// Static shared memory of a kernel (cudaFuncGetAttributes), which counts
// against the per-block opt-in limit together with the dynamic size; 1 KiB
// when the attributes cannot be read.
size_t static_smem_of(const void* kernel);
// Entry points that stage per-call tables from host memory (or wait on the
// stream) cannot be recorded into a CUDA graph: ISING_ERR_UNSUPPORTED while
// `st` is capturing, checked before anything is queued so that the caller's
// capture stays valid; ISING_OK otherwise.
int refuse_capture(cudaStream_t st);

// Everything the strip kernel reads; passed by value as the kernel parameter.
struct AnnealArgs {
  const uint8_t* flags;     // plane-order site flags [n]
  const uint32_t* thr;      // [2*S]: (T4_k, T8_k) for call sweep k
  const int8_t* init;       // [T][n] or null
  int8_t* out_spins;        // [T][n] or null
  int32_t* out_cuts;        // [T] or null
  int32_t X, Y, H, n;
  int32_t T;                // trials
  int32_t G;                // trials per group (multiple of 4, of 8 in the 16-bit mode; <= 32)
  int32_t S;                // sweeps in this call
  uint32_t k0;              // global index of the first sweep
  uint32_t key0, key1;      // Philox key
  uint32_t rk[20];          // round keys: rk[2r] = key0 + r*W0, rk[2r+1] = key1 + r*W1
  int32_t C;                // strips (CTAs) per group = cluster size
  int32_t Rmax;             // ceil(Y / C)
  int32_t neg_edges;
  int32_t u16;              // 1: 16-bit draw mode (G a multiple of 8, thresholds stored << 16)
  int32_t thr_group_stride; // words between the threshold tables of consecutive trial groups (0: one table)
};

// Everything the persistent flow kernel reads (anneal_flow.cu).
struct FlowArgs {
  const uint8_t* flags;     // plane-order site flags [n]
  const uint32_t* thr;      // [2*S]
  const int8_t* init;       // [T][n] or null
  int8_t* out_spins;        // [T][n] or null
  int32_t* out_cuts;        // [T] or null
  int32_t X, Y, H, n, T, G, S;
  uint32_t k0, key0, key1;
  uint32_t rk[20];
  int32_t RT;               // rows of all groups stacked: groups * Y
  int32_t P;                // CTAs (one per SM)
  int32_t LRmax;            // local rows (own rows and halo slots) of the largest CTA
  int32_t neg_edges;
  const int32_t* split;     // [P+1] first stacked site word (row * H + h) of each CTA
  unsigned long long* gm;   // [RT][2][H] mirror of rows read by another CTA: word | (half-sweep + 1) << 32 (zeroed)
  int32_t* acc;             // [T] per-trial cut partial sums (zeroed)
  uint32_t* done;           // CTAs finished (zeroed)
  uint32_t* abort_flag;     // set by a wait that ran out (zeroed)
  int32_t* status;          // the problem's status word
  long long spin_limit;     // cycles one wait may take
  int32_t stall_test;       // 1: the first chunk of CTA 0 waits for a count nothing reaches
  int32_t u16;              // 1: 16-bit draw mode
  int32_t thr_group_stride; // 0: one table for all groups; else group g's table at thr + g * stride
  int32_t cap;              // own site words per colour of the largest CTA, rounded up to a multiple of 32
  int32_t use_rec;          // 1: the fast path's records fit in shared memory
};
size_t flow_smem_bytes(int32_t LR, int32_t H, int32_t cap, int32_t rec);
int flow_threads();
int flow_max_segments();
cudaError_t launch_flow(const FlowArgs& a, cudaStream_t stream);
cudaError_t flow_max_ctas(size_t smem, int* per_sm);
size_t flow_static_smem();   // the largest over the kernel's instantiations

}  // namespace ising

// A persistent flow-kernel run planned and allocated once for repeated
// launches on one problem (abi.cu).
struct FlowRun;

namespace ising {

// Plans the run for `trials` trials and allocates its device arena, with room
// for `thr_words` threshold words (flow_run_thresholds).  Returns
// ISING_ERR_UNSUPPORTED when the flow kernel cannot take the problem.
int flow_run_create(ising_problem* p, int32_t trials, size_t thr_words, FlowRun** out, cudaStream_t st);
uint32_t* flow_run_thresholds(FlowRun* r);
// One launch: S sweeps from sweep k0 with the thresholds at d_thr (group g's
// at d_thr + g * thr_group_stride when the stride is not 0).
int flow_run_launch(FlowRun* r, const uint32_t* d_thr, int32_t thr_group_stride, int32_t S, uint32_t k0,
                    uint64_t seed, const int8_t* init_spins, int8_t* out_spins, int32_t* out_cuts, cudaStream_t st);
void flow_run_destroy(FlowRun* r, cudaStream_t st);

// One 3x3 circular convolution layer on the tensor cores (conv_tc.cu).
struct TcConvArgs {
  const __nv_bfloat16* in;      // [B*n][32] input activations (kinds 1-3)
  const int8_t* spins;          // [B][n] (kind 0: features s, w_right, w_down)
  const uint8_t* eflags;        // [n]    (kind 0)
  const __nv_bfloat16* wt;      // weights in the canonical [tap][chunk][n-group][8][8] layout
  const float* bias;            // [32] (kinds 0, 1) or [1] (kind 3)
  const __nv_bfloat16* mask;    // [B*n][32] (kind 2)
  __nv_bfloat16* out_bf16;      // [B*n][32] (kinds 0-2)
  float* out_f32;               // [B*n] (kind 3)
  int32_t* status;              // bounded-wait failures
  int X, Y, B;
  long long wait_limit;         // cycles one mbarrier wait may take (0: about two seconds)
  int32_t stall_test;           // 1: CTA 0 waits once on a barrier nothing arrives at
};
size_t conv_tc_smem(int kind, int X);

// Weight and bias gradients of one convolution layer on the tensor cores
// (conv_tc.cu).  kind 0: layer 1 (features of spins/eflags, g BF16 [32]);
// 1: 32 -> 32 (act and g BF16 [32]); 2: layer 4 (act BF16 [32], g FP32 [1]).
struct TcWgradArgs {
  const __nv_bfloat16* act;     // [B*n][32] layer input (kinds 1, 2)
  const int8_t* spins;          // kind 0
  const uint8_t* eflags;        // kind 0
  const void* g;                // gradient at the layer output: BF16 [B*n][32] or FP32 [B*n]
  float* part;                  // [max_ctas][96][96] per-CTA accumulators
  float* bpart;                 // [max_ctas][32]
  int32_t* status;
  int X, Y, B;
  int max_ctas;
  long long wait_limit;         // as TcConvArgs
  int32_t stall_test;
};
constexpr int kWgradMaxCtas = 640;
size_t wgrad_tc_smem(int kind, int X);
cudaError_t launch_wgrad_tc(int kind, const TcWgradArgs& a, int sms, float* dW, float* db, cudaStream_t st);
cudaError_t launch_conv_tc(int kind, const TcConvArgs& a, int sms, cudaStream_t st);

// Reading R3 (abi.cu): T = min(floor(exp(-x) 2^bits), 2^bits - 1) for the
// exponent x = beta dE of an uphill move, stored shifted left by 16 bits when
// bits = 16.  Every table the library uploads (annealing, replica exchange,
// the no-allocation entry point) is built from this one function.
uint32_t accept_threshold(double x, int bits);
// (T4_k, T8_k) = (accept_threshold(4 beta_k), accept_threshold(8 beta_k)) into
// out[2k], out[2k + 1] for k < S; ISING_ERR_ARG when some beta_k is not > 0.
int threshold_table(const double* betas, int32_t S, int bits, uint32_t* out);

// Launch shape of the strip kernel (abi.cu): trials per group G (0: the
// handle's, else 32 or all trials rounded up to a Philox block), strips per
// cluster C, threads per CTA and rows per strip.  ISING_ERR_UNSUPPORTED when
// no strip width fits shared memory or the grid is too tall.
struct StripShape {
  int G, C, threads, Rmax;
};
int strip_shape(const ising_problem* p, int32_t T, int32_t G, StripShape* out);
// Records a strip-kernel launch in the handle (ising_last_launch,
// ising_last_kernel) and logs it at ISING_LOG >= 1.
void record_strip_launch(ising_problem* p, int32_t trials, int32_t S, const StripShape& sh);

size_t anneal_smem_bytes(int32_t H, int32_t Rmax);
// grid = (C, ceil(T/G)); cluster (C,1,1) when C > 1
cudaError_t launch_anneal(const AnnealArgs& a, int threads, cudaStream_t stream);
cudaError_t launch_cut(const ising_problem* p, const int8_t* spins, int32_t k, int32_t* out,
                       cudaStream_t stream);

// ---------------------------------------------------------------- batched
struct BatchInst {                 // one instance of a batch (device-side descriptor)
  const uint8_t* flags;
  const uint32_t* thr;             // [2*S]
  const int8_t* init;              // [T][n] starting spins, or null (the Philox start)
  int8_t* out_spins;               // [T][n] or null (may equal init)
  int32_t* out_cuts;               // [T] or null
  int32_t X, Y, H, n;
  int32_t T, S;
  uint32_t key0, key1;
  int32_t neg_edges;
  int32_t G;                       // trials per work unit for this instance
  int32_t u16;                     // 1: 16-bit draw mode
  uint32_t k0;                     // global index of the first sweep (the Philox counter)
};
struct BatchUnit {                 // one work item: one trial group of one instance
  int32_t inst;
  int32_t group;
};
struct BatchArgs {
  const BatchInst* inst;
  const BatchUnit* units;
  int32_t n_units;
  uint32_t* counter;               // work-queue head, zero before the launch
};
// Everything the general-graph kernel reads (graph.cu).
struct GraphArgs {
  const uint32_t* nb;
  const int4* rowinfo;
  const int32_t* sites;
  const int32_t* colour_off;
  const uint32_t* thr;       // [S][Dmax]: entry q - 1 = T(dE = 2q)
  const int8_t* init;        // [T][n] or null
  int8_t* out_spins;         // [T][n] or null
  int32_t* out_cuts;         // [T] or null
  int32_t n, n_pad, thr_pad; // n and Dmax + 1, each rounded up to a multiple of 4
  int32_t Dmax, planes, ncol;
  int32_t T, S, C;           // trials, sweeps, CTAs per 32-trial group (cluster size)
  uint32_t k0, key0, key1;
  int32_t tpw;               // threads per site word: 1, 4 or 8
  uint32_t rk[20];           // Philox round keys: rk[2r] = key0 + r*W0, rk[2r+1] = key1 + r*W1
};
size_t graph_smem_bytes(int32_t n, int32_t Dmax);
int graph_threads();
cudaError_t launch_graph(const GraphArgs& a, cudaStream_t st);
cudaError_t launch_graph_measure(const GraphArgs& a, const int8_t* spins, int32_t k, int32_t* cuts,
                                 long long* energies, cudaStream_t st);
cudaError_t launch_energy_from_cut(const int32_t* cuts, int32_t W, int32_t k, int64_t* out, cudaStream_t st);

// The network's logits for B configurations of one torus problem (cnn.cu;
// the checks and errors of ising_cnn_forward).
int cnn_forward_ws(const ising_cnn* net, const ising_problem* p, const int8_t* spins, int32_t B, float* logits,
                   void* ws, size_t ws_bytes, cudaStream_t st);
// Cluster proposals (clusters.cu; ising_propose_clusters), adding the
// accepted counts to `accepted` when accumulate is 1.
int propose_clusters_launch(const ising_problem* const* probs, int32_t m, int8_t* spins, int32_t B,
                            const float* logits, int32_t* accepted, int accumulate, cudaStream_t st);

// Partner moves (clusters.cu; ising_transcribe), adding to `accepted` when
// accumulate is 1.
int transcribe_launch(const ising_problem* const* probs, int32_t m, const int8_t* spins, int8_t* out, int32_t B,
                      int32_t shift, int32_t* accepted, int accumulate, cudaStream_t st);

size_t batched_smem_bytes(int32_t H, int32_t Y);
cudaError_t batched_prepare(size_t smem);
size_t batched_static_smem();
cudaError_t launch_batched(const BatchArgs& a, int grid, int threads, size_t smem, cudaStream_t stream);

}  // namespace ising

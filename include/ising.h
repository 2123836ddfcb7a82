/*
 * ising.h -- C ABI of the GB300 toroidal Ising / Max-Cut annealer.
 *
 * Problem (Zick 2025, Section II, Eq. 1 and Eq. 2): n = X*Y spins s_i in
 * {-1,+1} on an X-by-Y periodic square grid (Section I, Appendix A), site
 * i = y*X + x, each site coupled to its four nearest neighbours with weights
 * w_ij in {-1,+1}.  The Ising form uses J_ij = -w_ij and h_i = 0, so
 *     H(s)   = -sum_{i<j} J_ij s_i s_j = sum_{i<j} w_ij s_i s_j,
 *     cut(s) = 1/2 sum_{i<j} w_ij (1 - s_i s_j) = (W - H(s)) / 2,
 * with W = sum_{i<j} w_ij.
 *
 * Method: independent trials of sweeps (Section III: the sweep is the
 * fundamental step; solutions are read out at the end of each trial).  The
 * paper leaves its own update rule unpublished, so a sweep here is a
 * Metropolis sweep over the checkerboard: colour (x+y) mod 2 = 0 first, then
 * colour 1; a spin flips when its energy change dE = -2 s_i sum_j w_ij s_j is
 * <= 0, or when the 32-bit draw u is below the threshold
 * T_dE = min(floor(exp(-beta_k dE) 2^32), 2^32 - 1) of the sweep's inverse
 * temperature beta_k.  The draw for trial t, sweep k, site i is word
 * (t mod 4) of Philox4x32-10 (Salmon et al., SC'11) at counter
 * (i, k, t/4, 0) with key (seed mod 2^32, seed / 2^32); the random starting
 * spin is +1 when bit 31 of the word at counter (i, 0xFFFFFFFF, t/4, 0) is
 * set.  Results are a pure function of (instance, trial index, sweep index,
 * betas, seed): they do not depend on the launch configuration.
 *
 * Conventions for every entry point:
 *   - Return 0 (ISING_OK) on success, a negative ISING_ERR_* code otherwise.
 *     No C++ exception crosses this boundary.  ising_strerror names a code.
 *   - "host" pointers are read during the call and may be freed on return;
 *     "device" pointers are CUDA device (or managed) memory owned by the
 *     caller, which must stay valid until the work queued on the stream is
 *     done.
 *   - Work is queued asynchronously on `cuda_stream` (a cudaStream_t; NULL is
 *     the legacy default stream).  Errors found by argument checks return
 *     before anything is queued.
 *   - Spins are int8: any value > 0 reads as +1, anything else as -1; spins
 *     written by the library are exactly +1 or -1.  Spin arrays are
 *     row-major [trials][n].  Cuts are int32 (|cut| <= |E| = 2n).
 *   - A problem handle is bound to the device that was current at creation;
 *     do not use one handle from two streams at the same time.
 *   - CUDA graphs: ising_anneal, ising_anneal_trace, ising_anneal_batched,
 *     ising_anneal_pt, ising_batch_create, ising_learned_create and
 *     ising_get_status copy per-call tables from host memory or wait on the
 *     stream, so they cannot be recorded into a graph: while `cuda_stream`
 *     is capturing they return ISING_ERR_UNSUPPORTED before queuing
 *     anything, and the capture stays valid.  For replayable work use
 *     ising_batch_create / ising_learned_create (each one graph, created
 *     outside any capture).
 *     Calls that only queue kernels on device memory may be captured:
 *     ising_cut, ising_cnn_forward, ising_propose, ising_propose_clusters,
 *     ising_droplet_targets and ising_transcribe (the learned plan's graph
 *     records the same launches).
 */
#ifndef ISING_H
#define ISING_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ISING_OK                 0
#define ISING_ERR_ARG           -1  /* bad pointer, size, beta <= 0 or NaN, J not +-1 */
#define ISING_ERR_NOT_TORUS     -2  /* CSR is not the symmetric 4-neighbour X-by-Y torus */
#define ISING_ERR_ODD_DIM       -3  /* X or Y odd: the checkerboard is not bipartite */
#define ISING_ERR_H_UNSUPPORTED -4  /* a non-zero local field h_i was given */
#define ISING_ERR_OOM           -5  /* host or device allocation failed */
#define ISING_ERR_CUDA          -6  /* a CUDA runtime call or kernel launch failed */
#define ISING_ERR_TIMEOUT       -7  /* a bounded device-side wait ran out */
#define ISING_ERR_UNSUPPORTED   -8  /* valid input beyond what this library handles */

typedef struct ising_problem ising_problem;

/*
 * ising_create -- validate a toroidal instance and pack it on the device.
 * (Eq. 2 with J = -w, h = 0; the Gset toroidal grids of Section I.)
 *
 * n        number of spins, must equal X*Y.
 * row_ptr  host, n+1 int64 CSR row offsets (row_ptr[0] = 0, nondecreasing).
 * col_idx  host, row_ptr[n] int32 column indices.
 * J        host, row_ptr[n] int8 couplings, each -1 or +1 (J = -w).
 * h        host, n int8 local fields, or NULL; every entry must be 0.
 * X, Y     torus width and height, both even and >= 4.
 * out      receives the new handle (unchanged on error).
 *
 * Row i must list exactly the four torus neighbours of i (any order) and J
 * must be symmetric.  Errors: ISING_ERR_ARG (NULL pointer, n != X*Y, |J| != 1,
 * X or Y < 4), ISING_ERR_ODD_DIM, ISING_ERR_NOT_TORUS, ISING_ERR_H_UNSUPPORTED,
 * ISING_ERR_OOM, ISING_ERR_CUDA.  All argument checks run before any CUDA call.
 */
int ising_create(int32_t n, const int64_t* row_ptr, const int32_t* col_idx,
                 const int8_t* J, const int8_t* h, int32_t X, int32_t Y,
                 ising_problem** out);

/* ising_destroy -- free a handle and its device memory (NULL is a no-op).
 * Synchronises with nothing: the caller must not destroy a handle while work
 * that uses it is still queued. */
void ising_destroy(ising_problem* p);

/*
 * ising_anneal -- run `trials` independent trials of S Metropolis sweeps
 * (Section III: trials, sweeps, read-out at the end of each trial).
 *
 * trials        number of trials T >= 0 (T = 0 queues nothing).
 * betas         host, S doubles, inverse temperature of each sweep, each > 0
 *               (+inf allowed: zero temperature).
 * S             number of sweeps >= 0; sweep j of the call is global sweep
 *               sweep_offset + j, which selects its random draws.
 * seed          64-bit Philox key.
 * sweep_offset  first global sweep index (resume: a run of S1 + S2 sweeps
 *               equals S1 sweeps, then S2 more from the saved spins with
 *               sweep_offset = S1 and betas[S1..]).
 * init_spins    device [T][n] starting spins, or NULL for the Philox start.
 * out_spins     device [T][n] final spins, or NULL.
 * out_cuts      device [T] final Eq. 1 cuts, or NULL.
 * cuda_stream   stream to queue on.
 *
 * Scratch: the per-sweep threshold table (8*S bytes) and, on the persistent
 * kernel, its row tables and the mirror of the rows two CTAs share (8 bytes
 * per word of those rows) are allocated and freed in stream order
 * (cudaMallocFromPoolAsync / cudaFreeAsync) from a memory pool of the
 * library's own per device, which keeps the memory it has held until the
 * process exits, so that a call after a synchronisation does not map its
 * scratch again.
 * Errors: ISING_ERR_ARG, ISING_ERR_UNSUPPORTED (no launch shape fits, or
 * cuda_stream is capturing a graph), ISING_ERR_OOM, ISING_ERR_CUDA.
 */
int ising_anneal(ising_problem* p, int32_t trials, const double* betas, int32_t S,
                 uint64_t seed, uint32_t sweep_offset, const int8_t* init_spins,
                 int8_t* out_spins, int32_t* out_cuts, void* cuda_stream);

/*
 * ising_cut -- exact Eq. 1 cut of k configurations on the device.
 *
 * spins     device [k][n] int8.
 * k         number of configurations >= 0.
 * out_cuts  device [k] int32.
 * Errors: ISING_ERR_ARG, ISING_ERR_CUDA.
 */
int ising_cut(const ising_problem* p, const int8_t* spins, int32_t k,
              int32_t* out_cuts, void* cuda_stream);

/*
 * ising_anneal_batched -- anneal m instances of uneven sizes, trial counts and
 * sweep counts in one persistent launch (Section III campaigns, run as one
 * batch).  Instance q behaves exactly like
 *   ising_anneal(probs[q], trials[q], betas[q], sweeps[q], seeds[q], 0, NULL,
 *                out_spins[q], out_cuts[q], stream).
 *
 * probs      host array of m handles (all on the current device).
 * trials     host, m trial counts >= 0.     sweeps  host, m sweep counts >= 0.
 * betas      host array of m host pointers, betas[q] has sweeps[q] doubles.
 * seeds      host, m seeds.
 * out_spins  host array of m device pointers ([trials[q]][n_q] int8) or NULL
 *            (the array itself or any entry).
 * out_cuts   host array of m device pointers ([trials[q]] int32) or NULL.
 * Scratch: descriptors, work list and thresholds in one stream-ordered
 * allocation from the library's pool (as ising_anneal), freed in stream
 * order.
 * Errors: ISING_ERR_ARG (NULL arrays, negative counts, a beta <= 0 or NaN,
 * handles on different devices), ISING_ERR_UNSUPPORTED (a general-graph
 * handle, a torus too large for one CTA's shared memory, or cuda_stream
 * capturing a graph), ISING_ERR_OOM, ISING_ERR_CUDA.
 */
int ising_anneal_batched(ising_problem* const* probs, int32_t m, const int32_t* trials,
                         const int32_t* sweeps, const double* const* betas,
                         const uint64_t* seeds, int8_t* const* out_spins,
                         int32_t* const* out_cuts, void* cuda_stream);

/*
 * Batch plans: the same work as ising_anneal_batched (Section III campaigns
 * as one batch), prepared once (tables
 * uploaded, work list sorted longest first) and replayed as a CUDA graph.
 * ising_batch_create queues the uploads on `cuda_stream`; every
 * ising_batch_launch replays the graph (reset the work counter, persistent
 * kernel) on the given stream.  The output pointers are baked into the plan.
 * group_trials (4..32, multiple of 4, or 0 = auto) and ctas_per_sm (1..4, or
 * 0 = auto) set the work-unit width and the persistent grid.
 * ising_batch_create errors: those of ising_anneal_batched, and
 * ISING_ERR_ARG for a NULL `out` or group_trials / ctas_per_sm out of range.
 */
typedef struct ising_batch ising_batch;
int ising_batch_create(ising_problem* const* probs, int32_t m, const int32_t* trials,
                       const int32_t* sweeps, const double* const* betas,
                       const uint64_t* seeds, int8_t* const* out_spins,
                       int32_t* const* out_cuts, int32_t group_trials,
                       int32_t ctas_per_sm, void* cuda_stream, ising_batch** out);
/* ising_batch_launch -- replay the plan on cuda_stream (asynchronous).
 * Errors: ISING_ERR_ARG (NULL plan), ISING_ERR_CUDA. */
int ising_batch_launch(ising_batch* b, void* cuda_stream);
/* Frees the plan; waits for the plan's last launch to finish first (NULL is
 * a no-op). */
void ising_batch_destroy(ising_batch* b);

/*
 * ising_set_launch -- fix the launch shape used by ising_anneal for this
 * handle (the autotuner's knob).  0 in any field restores the automatic
 * choice.
 * group_trials   trials packed per 32-bit word, multiple of 4 in [4, 32].
 * strips         CTAs that share one trial group as row strips (thread-block
 *                cluster of that size, 1..16), at most Y; for a general
 *                graph handle the cluster that shares a 32-trial group,
 *                1..8 (group_trials and threads do not apply there).
 * threads        threads per CTA, multiple of 32 in [64, 1024].
 * Errors: ISING_ERR_ARG.  Results do not depend on the shape.
 */
int ising_set_launch(ising_problem* p, int32_t group_trials, int32_t strips, int32_t threads);

/* ising_last_launch -- the shape the last ising_anneal call on this handle
 * used (any pointer may be NULL).  Errors: ISING_ERR_ARG (NULL handle). */
int ising_last_launch(const ising_problem* p, int32_t* group_trials, int32_t* strips,
                      int32_t* threads, int32_t* grid_ctas);

/*
 * ising_set_kernel -- choose the kernel ising_anneal uses for this handle:
 *   0 automatic (default): the persistent kernel when the instance has at
 *     least 2,048 spins, its trial groups of 32 stack to at least four rows
 *     per SM, and no strip shape is fixed; else the strip kernel;
 *   1 strip kernel: each trial group annealed by a thread-block cluster of
 *     row strips (ising_set_launch sets its shape);
 *   2 persistent kernel: the rows of all trial groups stacked and split over
 *     one CTA per SM, the rows another CTA reads exchanged through an L2
 *     mirror of words tagged with their half-sweep; ISING_ERR_UNSUPPORTED
 *     from ising_anneal if a CTA would touch more than 4 trial groups or its
 *     rows do not fit in shared memory.
 * Results do not depend on the kernel.  Errors: ISING_ERR_ARG.
 */
int ising_set_kernel(ising_problem* p, int32_t kind);

/*
 * ising_batch_schedule -- the schedule ising_batch_create / ising_anneal_batched
 * would give m torus instances (host only; no GPU, no handles): X[q] x Y[q]
 * tori (even, >= 4), trials[q] trials of sweeps[q] sweeps, all in the given
 * draw mode (32 or 16).  group_trials and ctas_per_sm as in
 * ising_anneal_batched (0: automatic); sms: the GPU's SMs; smem_per_cta_max:
 * its shared memory per CTA (0: 227 KiB).  Writes the CTAs per SM and threads
 * per CTA, G[q] (trials per work unit of instance q, host int32 [m]) and, if
 * units is not NULL, the work units in the order the CTAs take them, as
 * (instance, group) pairs (host int32 [cap][2]); *nunits receives their
 * count.  A unit's cost is n (sweeps + 1) x (3 + its Philox blocks per site
 * word); units are taken longest first.  An instance whose 32-trial unit fits
 * in a CTA's average load keeps G = 32; the others share the multiple of the
 * Philox block (32 down to one block) whose units finish first under that
 * longest-first list schedule on sms x per_sm CTAs (ties: the wider).
 * Errors: ISING_ERR_ARG (bad sizes, cap too small), ISING_ERR_UNSUPPORTED (a
 * whole trial group does not fit in shared memory).
 */
int ising_batch_schedule(int32_t m, const int32_t* X, const int32_t* Y, const int32_t* trials, const int32_t* sweeps,
                         int32_t draw_bits, int32_t group_trials, int32_t ctas_per_sm, int32_t sms,
                         int32_t smem_per_cta_max, int32_t* per_sm, int32_t* threads, int32_t* G, int32_t* units,
                         int32_t cap, int32_t* nunits);

/*
 * ising_thresholds -- the acceptance thresholds every annealing call of this
 * library uploads for its schedule (host only; no GPU, no handle).  The
 * Metropolis rule accepts an uphill move of dE > 0 with probability
 * exp(-beta dE) (the paper leaves its own rule unpublished, Section III; on
 * the +-1 torus dE is 4 or 8, from Eq. 2 with J = -w, h = 0): a draw u is
 * accepted iff u < T_dE.  betas: host double [S], each > 0 (+inf allowed).
 * out: host uint32 [S][2] receives (T_4, T_8) per sweep, with
 * T_d = min(floor(exp(-beta d) 2^32), 2^32 - 1); with draw_bits 16,
 * min(floor(exp(-beta d) 2^16), 2^16 - 1) stored shifted left by 16 bits
 * (the form the kernels compare against).  exp is the host C library's, in
 * double precision.  Errors: ISING_ERR_ARG (S < 0, a NULL pointer with
 * S > 0, draw_bits not 16 or 32, a beta that is not > 0), ISING_ERR_OOM.
 */
int ising_thresholds(const double* betas, int32_t S, int32_t draw_bits, uint32_t* out);

/*
 * ising_flow_split -- the persistent kernel's division of work, for
 * inspection and tests (host only; no GPU, no handle).  The rows of all
 * ceil(trials / group_trials) trial groups of a Y-row torus with H = X/2 site
 * words per row and colour are stacked, and their words (row * H + h) split
 * into ctas = min(sms, rows) contiguous ranges of equal weight: a word weighs
 * its group's Philox blocks per sweep (ceil(live trials / 4), or / 8 with
 * draw_bits 16) when `weighted`, else 1.  Ranges may start and end inside a
 * row (a row then shared by two CTAs), except with draw_bits 16, where they
 * end at row boundaries.  Writes the ctas + 1 range starts into split_out
 * (host int32, cap entries), and, unless NULL, the most local rows (own rows,
 * plus two halo rows per trial group not wholly owned) and the most trial
 * groups any CTA touches.  ising_anneal refuses the persistent kernel when
 * those exceed its shared memory or 4 groups.  Errors: ISING_ERR_ARG (bad
 * sizes, draw_bits not 16 or 32, cap too small), ISING_ERR_UNSUPPORTED (more
 * than 2^30 rows or words).
 */
int ising_flow_split(int32_t Y, int32_t H, int32_t trials, int32_t group_trials, int32_t draw_bits, int32_t sms,
                     int32_t weighted, int32_t* split_out, int32_t cap, int32_t* ctas, int32_t* local_rows_max,
                     int32_t* segments_max);

/*
 * ising_set_graph_threads_per_site -- general-graph handles: how many
 * threads share one site word's update in ising_anneal (Section II's general
 * form; the sweep and its decisions are unchanged).  1: one thread counts the
 * neighbours and draws all Philox blocks; 4 or 8: the threads split the
 * neighbours and the blocks and combine their counts with warp shuffles, for
 * graphs whose colour classes are too small to occupy the GPU one word per
 * thread.  0 (default) chooses by the average class size.  Results do not
 * depend on it.  Errors: ISING_ERR_ARG (NULL handle, other values).
 */
int ising_set_graph_threads_per_site(ising_problem* p, int32_t threads_per_site);

/*
 * ising_philox -- the library's Philox4x32-10 generator (Salmon et al.,
 * SC'11), the source of every start spin and decision draw: for each of k
 * counters ctr[j] (device uint32 [k][4], 16-byte aligned) writes the block
 * out[j] (device uint32 [k][4], 16-byte aligned) under the key
 * (seed mod 2^32, seed / 2^32).  Trial t at site i in sweep k draws word
 * t mod 4 of the block at counter (i, k, t/4, 0); its start spin is bit 31 of
 * word t mod 4 at counter (i, 0xFFFFFFFF, t/4, 0).  For reproducing
 * individual draws.  Asynchronous on cuda_stream.  Errors: ISING_ERR_ARG.
 */
int ising_philox(const uint32_t* ctr, uint64_t seed, int32_t k, uint32_t* out, void* cuda_stream);

/*
 * ising_spins_to_hex / ising_hex_to_spins -- a configuration (host int8 [n],
 * > 0 means +1) as hexadecimal digits, the form in which the paper prints its
 * best cuts (App. C-E): digit d holds spins 4d .. 4d+3, the first of them in
 * the most significant bit, bit 1 for +1 and 0 for -1, the last digit padded
 * with 0 bits (the paper does not state the bit order; this reading is the
 * library's).  to_hex writes ceil(n/4) digits and a terminating NUL into out
 * (cap bytes, host).  from_hex skips whitespace and needs exactly ceil(n/4)
 * digits with zero padding bits.  Errors: ISING_ERR_ARG.
 */
int ising_spins_to_hex(const int8_t* spins, int32_t n, char* out, int64_t cap);
int ising_hex_to_spins(const char* hex, int32_t n, int8_t* out);

/*
 * ising_debug_fail_allocs -- a test hook: the next `count` device allocations
 * the library makes report failure, so the calls that make them return
 * ISING_ERR_OOM (host-side fault injection; nothing is done on the GPU).
 * 0 clears it.  Errors: ISING_ERR_ARG (count < 0).
 */
int ising_debug_fail_allocs(int32_t count);

/*
 * ising_anneal_pt -- replica exchange (parallel tempering) on a torus handle:
 * `temps` temperatures betas[0..temps-1] (host, positive, finite) times
 * `chains` chains (a multiple of 32).  Slot t = r * chains + c holds chain c
 * at temperature r.  Each of `rounds` rounds runs sweeps_per_round sweeps of
 * every slot at its constant beta (global sweeps q L .. q L + L - 1; slot t
 * keeps the decision stream of trial index t), then exchanges the pairs
 * (r, r+1), r = q mod 2, q mod 2 + 2, ..., chain by chain: with
 * d = E_r - E_{r+1} (Eq. 2, E = W - 2 cut) the swap is taken iff d <= 0 or
 * u < min(floor(exp(-(beta_{r+1} - beta_r) d) 2^32), 2^32 - 1), u = word 0 of
 * Philox4x32-10 at counter (c, q, r, 0xFFFFFFFD).  Start: the start spins of
 * every slot.  out_spins (device int8 [temps*chains][n]) and out_cuts
 * (device int32 [temps*chains]) receive the final slots; out_swaps (device
 * int32 or NULL) the number of swaps taken.  The sweeps run on the kernel
 * ising_anneal would choose for temps*chains trials (the persistent kernel
 * with one threshold table per 32-slot group, else the strip kernel);
 * ising_set_kernel(p, 1) forces the strip kernel.  Asynchronous on
 * cuda_stream; allocates its tables, one spin-sized buffer and the persistent
 * kernel's scratch in stream order.
 * Errors: ISING_ERR_ARG, ISING_ERR_UNSUPPORTED (general-graph handle, 16-bit
 * mode, no launch shape), ISING_ERR_OOM, ISING_ERR_CUDA.  The paper has no
 * counterpart (its update rule is unpublished, Section III).
 */
int ising_anneal_pt(ising_problem* p, int32_t temps, const double* betas, int32_t chains, int32_t rounds,
                    int32_t sweeps_per_round, uint64_t seed, int8_t* out_spins, int32_t* out_cuts, int32_t* out_swaps,
                    void* cuda_stream);

/*
 * ising_graph_create -- a general sparse instance: any simple undirected
 * graph as a symmetric CSR (host pointers, copied; row_ptr int64 [n+1],
 * col_idx int32 [nnz], J int8 [nnz] with J_ij = J_ji, 1 <= |J| <= 127, no
 * self loops or repeated neighbours) and integer fields h (int8 [n],
 * |h| <= 127, or NULL).  Eq. 2 in full: H = -sum_{i<j} J_ij s_i s_j -
 * sum_i h_i s_i; the Max-Cut weights are w = -J (Eq. 1).  n <= 2^24, and per
 * site sum |J| + |h| <= 255.  The sweep visits the classes of the first-fit
 * colouring (ising_greedy_colouring) in order; ising_anneal, ising_cut,
 * ising_energy and ising_anneal_trace accept the handle (the batched, the
 * 16-bit and the no-allocation paths return ISING_ERR_UNSUPPORTED).  One
 * 32-trial group's spins must fit in shared memory (about 56,000 sites).
 * Errors: ISING_ERR_ARG (malformed or asymmetric CSR), ISING_ERR_UNSUPPORTED,
 * ISING_ERR_OOM, ISING_ERR_CUDA.  The paper frames the problem this way
 * (Section II); its own runs use the toroidal instances only.
 */
int ising_graph_create(int32_t n, const int64_t* row_ptr, const int32_t* col_idx, const int8_t* J,
                       const int8_t* h, ising_problem** out);

/*
 * ising_greedy_colouring -- the colouring the general-graph sweep uses
 * (Eq. 2 with general J and h; a checkerboard needs a proper colouring; host
 * only, no GPU): site i takes the smallest colour no neighbour j < i
 * holds.  colour: int32 [n] (host, caller-owned); *ncol: classes used.
 * Errors: ISING_ERR_ARG (n < 0 or a NULL pointer), ISING_ERR_OOM.
 */
int ising_greedy_colouring(int32_t n, const int64_t* row_ptr, const int32_t* col_idx, int32_t* colour,
                           int32_t* ncol);

/* ising_graph_info -- n, colour classes and the largest sum |J| + |h| of a
 * general-graph handle.  Errors: ISING_ERR_ARG (NULL or torus handle). */
int ising_graph_info(const ising_problem* p, int32_t* n, int32_t* ncol, int32_t* Dmax);

/*
 * ising_energy -- Eq. 2 of k configurations (device int8 [k][n]) into
 * out_energies (device int64 [k]); asynchronous on cuda_stream.  For a torus
 * handle H = W - 2 cut, through a k-int32 cut buffer allocated in stream
 * order.  Errors: ISING_ERR_ARG, ISING_ERR_OOM, ISING_ERR_CUDA.
 */
int ising_energy(const ising_problem* p, const int8_t* spins, int32_t k, int64_t* out_energies, void* cuda_stream);

/*
 * ising_anneal_trace -- ising_anneal with read-out along the trajectory
 * (Section III reads each trial out at its end; Fig. 1 plots the cut against
 * sweeps).  After sweep j of the call (counting from 1) for every j that is a
 * multiple of trace_every, and after the last sweep, the Eq. 1 cut of every
 * trial is written to out_trace[p][t], p = 0 .. ceil(S / trace_every) - 1 in
 * sweep order (device int32, points x trials, or NULL).  out_best[t] (device
 * int32 [trials] or NULL) receives the largest of those cuts and
 * out_best_spins[t][.] (device int8 [trials][n] or NULL, 4-byte aligned) the
 * first configuration reaching it; with S = 0 the best is the starting
 * configuration.  out_spins (required, 4-byte aligned) and out_cuts (or
 * NULL) receive the final state as in ising_anneal; init_spins must not be
 * out_spins.  The trajectory, and every other output, equals that of one
 * ising_anneal call with the same arguments: the work runs as chunks of
 * trace_every sweeps, each resuming from the previous one at its global
 * sweep.  Asynchronous on cuda_stream; allocates one spin-sized scratch
 * buffer in stream order.  Errors: ISING_ERR_ARG (trace_every <= 0, bad
 * pointers or betas), and those of ising_anneal.  The paper has no such
 * entry point.
 */
int ising_anneal_trace(ising_problem* p, int32_t trials, const double* betas, int32_t S, uint64_t seed,
                       uint32_t sweep_offset, const int8_t* init_spins, int8_t* out_spins, int32_t* out_cuts,
                       int32_t trace_every, int32_t* out_trace, int32_t* out_best, int8_t* out_best_spins,
                       void* cuda_stream);

/*
 * ising_set_draw_bits -- the decision stream of this handle's anneals
 * (ising_anneal, ising_anneal_noalloc and the batch entry points):
 *   32 (default): trial t at site i in sweep k draws word t mod 4 of the
 *     Philox4x32-10 block at counter (i, k, t/4, 0) and compares it with
 *     T_d = min(floor(exp(-beta d) 2^32), 2^32 - 1);
 *   16: one block serves eight trials -- trial t draws the low (t even) or
 *     high (t odd) 16-bit half of word (t mod 8)/2 of the block at counter
 *     (i, k, t/8, 0) and compares it with T_d = min(floor(exp(-beta d) 2^16),
 *     2^16 - 1).  About half the Philox work per update; the acceptance
 *     probabilities are quantised to 2^-16.
 * The starting spins are the same in both modes.  The paper has no
 * counterpart (its update rule is unpublished, Section III); the 16-bit mode
 * is a variant of this library.  In the 16-bit mode a fixed trials-per-group
 * (ising_set_launch, the batch group_trials) must be a multiple of 8, else
 * the anneal returns ISING_ERR_ARG.  Errors: ISING_ERR_ARG (bits not 16 or 32).
 */
int ising_set_draw_bits(ising_problem* p, int32_t bits);

/* ising_last_kernel -- the kernel (1 or 2) the last ising_anneal call used.
 * Errors: ISING_ERR_ARG (NULL pointer). */
int ising_last_kernel(const ising_problem* p, int32_t* kind);

/*
 * ising_get_status -- wait for `cuda_stream`, then read and clear the handle's
 * device status word.  *code is ISING_OK, or ISING_ERR_TIMEOUT when a bounded
 * device-side wait of the persistent kernel ran out (the results of that call
 * are then undefined; the CUDA context stays usable).
 * Errors: ISING_ERR_ARG (NULL pointer), ISING_ERR_UNSUPPORTED (cuda_stream
 * capturing a graph), ISING_ERR_CUDA.
 */
int ising_get_status(ising_problem* p, void* cuda_stream, int32_t* code);

/*
 * ising_set_wait_limit -- (this project's failure detection; the paper has no
 * counterpart) cycles one device-side wait of the persistent kernel
 * may take before it gives up (0 restores the default of 4e9 cycles), and a
 * test switch: stall_test = 1 makes the first chunk of the first CTA wait for
 * a count that is never reached, so the limit runs out on purpose.
 * Errors: ISING_ERR_ARG.
 */
int ising_set_wait_limit(ising_problem* p, int64_t cycles, int32_t stall_test);

/* ising_problem_info -- X, Y and W = sum of the weights over the 2n edges
 * (so that H = W - 2 cut); any pointer may be NULL.  Errors: ISING_ERR_ARG
 * (NULL handle). */
int ising_problem_info(const ising_problem* p, int32_t* X, int32_t* Y, int32_t* weight_sum);

/*
 * ising_anneal_noalloc -- ising_anneal for callers that cannot allocate
 * device memory while they run (for example an application whose framework
 * has already reserved the device memory it may use, or a loop that must not
 * enter the CUDA allocator once started).  The paper has no counterpart; this
 * is an interface variant of ising_anneal, with the same arguments and
 * results, bit for bit, for the same launch shape.
 *
 * The call allocates nothing: the per-sweep threshold table goes into one
 * fixed array inside the library's device image, at most 32,768 sweeps
 * (256 KiB, held by every GPU that loads the library until the process
 * exits).  The table reaches that array through the parameters of small
 * copy kernels queued on cuda_stream ahead of the anneal (one per 1,024
 * sweeps), so no host buffer has to outlive the call.  The anneal itself
 * always runs on the cluster-strip kernel (the persistent kernel needs a
 * per-call work area).  The first call on a device looks up that array's
 * device address, with the problem's device current; make that first call
 * before any stream capture.  All calls share the array and it keeps the
 * last call's contents: calls whose work overlaps on the GPU (unordered
 * streams) race on it.  Nothing in the array needs to start at zero.
 *
 * Errors: those of ising_anneal, with four differences:
 *   ISING_ERR_UNSUPPORTED  S > 32,768, or a general-graph handle
 *                          (ising_graph_create), which ising_anneal accepts;
 *   ISING_ERR_ARG          the current device is not the problem's device;
 *   a capturing cuda_stream is not refused: after the first call on a
 *   device the call queues only kernel launches, with the table's words in
 *   their parameters (recording it into a graph is not tested).
 * Each error is returned before anything is queued.  The launch this call used is
 * what ising_last_launch and ising_last_kernel then report.
 */
int ising_anneal_noalloc(ising_problem* p, int32_t trials, const double* betas, int32_t S,
                         uint64_t seed, uint32_t sweep_offset, const int8_t* init_spins,
                         int8_t* out_spins, int32_t* out_cuts, void* cuda_stream);

/* ======================================================================
 * Learned proposals (this project's extension; the paper's own update rule
 * is unpublished, Section III).  A circular-padded CNN on the torus with
 * four 3x3 convolutions of 32 channels (ReLU between them) maps, per site,
 * the inputs (s_i, w right, w down) to a logit for "flip this spin".
 * Proposals built from the logits are accepted only by their exact integer
 * energy change (Eq. 2), so they can never make a trial worse.
 *
 * Parameters: ISING_CNN_PARAMS floats in the order W1[32,3,3,3], b1[32],
 * W2[32,32,3,3], b2[32], W3[32,32,3,3], b3[32], W4[1,32,3,3], b4[1], each
 * weight laid out (out channel, in channel, ky, kx); convolution:
 * out[y,x] = b + sum W[o,c,ky,kx] in[c,(y+ky-1) mod Y,(x+kx-1) mod X].
 * Weights are used rounded to BF16, activations are stored in BF16, sums
 * accumulate in FP32.
 * ====================================================================== */
#define ISING_CNN_PARAMS 19681
typedef struct ising_cnn ising_cnn;

/* ising_cnn_create -- copy ISING_CNN_PARAMS host floats to a new network on
 * the current device (Adam state zeroed).  Errors: ISING_ERR_ARG, _OOM, _CUDA. */
int ising_cnn_create(const float* params, ising_cnn** out);
/* ising_cnn_destroy -- free the network's device memory (NULL is a no-op);
 * the caller must not destroy it while work that uses it is still queued. */
void ising_cnn_destroy(ising_cnn* net);
/* host copy of the FP32 master parameters (synchronous).  Errors:
 * ISING_ERR_ARG (NULL pointer), ISING_ERR_CUDA. */
int ising_cnn_get_params(const ising_cnn* net, float* params);
/* replace the parameters (host) and reset the Adam state (synchronous).
 * Errors: ISING_ERR_ARG (NULL pointer), ISING_ERR_CUDA. */
int ising_cnn_set_params(ising_cnn* net, const float* params);

/* Device workspace (bytes) for B configurations of n spins; train != 0 for
 * ising_cnn_grad.  The caller allocates it; the calls allocate nothing. */
size_t ising_cnn_workspace_bytes(int32_t B, int32_t n, int32_t train);

/*
 * ising_cnn_forward -- logits for B configurations of problem p (learned
 * stage, this project's extension; the network is the one defined above).
 * spins    device [B][n] int8 (>0 is +1).
 * logits   device [B][n] float (site order y*X + x).
 * ws       device workspace of at least ising_cnn_workspace_bytes(B, n, 0).
 * The convolutions run on the tensor cores; a device-side wait on them that
 * runs out (after about two seconds) leaves ISING_ERR_TIMEOUT in the
 * handle's status word (ising_get_status).
 * Errors: ISING_ERR_ARG, ISING_ERR_UNSUPPORTED (torus width above 512, or a
 * general-graph handle), ISING_ERR_CUDA.
 */
int ising_cnn_forward(const ising_cnn* net, const ising_problem* p, const int8_t* spins, int32_t B,
                      float* logits, void* ws, size_t ws_bytes, void* cuda_stream);

/*
 * ising_cnn_grad -- (learned stage, this project's extension) mean binary
 * cross-entropy of the logits against the flip
 * targets and its gradient with respect to the parameters.
 * targets  device [B][n] uint8 (1 = the site should flip).
 * grad     device ISING_CNN_PARAMS floats (overwritten).
 * loss     device float (overwritten).
 * ws       device workspace of at least ising_cnn_workspace_bytes(B, n, 1).
 * Device-side timeouts as in ising_cnn_forward.  Errors: ISING_ERR_ARG,
 * ISING_ERR_UNSUPPORTED (torus width above 512, or a general-graph handle),
 * ISING_ERR_CUDA.
 */
int ising_cnn_grad(const ising_cnn* net, const ising_problem* p, const int8_t* spins, const uint8_t* targets,
                   int32_t B, float* grad, float* loss, void* ws, size_t ws_bytes, void* cuda_stream);

/*
 * ising_cnn_set_wait_limit -- cycles one device-side wait of the network's
 * tensor-core kernels (for the completion of its MMAs) may take before the
 * CTA gives up (0 restores the default of about two seconds), and a test
 * switch: stall_test = 1 makes CTA 0 of every tensor-core launch of this
 * network wait once, with that limit, on an mbarrier nothing arrives at, so
 * the wait runs out on purpose.  A CTA whose wait ran out stops its work,
 * still waits for the MMAs it has committed before it frees its tensor
 * memory, and leaves ISING_ERR_TIMEOUT in the problem's status word
 * (ising_get_status); that call's results are undefined.  This project's
 * failure detection; the paper has no counterpart.  Errors: ISING_ERR_ARG.
 */
int ising_cnn_set_wait_limit(ising_cnn* net, int64_t cycles, int32_t stall_test);

/* ising_cnn_adam_step -- one Adam update of the FP32 master parameters with
 * the device gradient `grad`, then refresh the BF16 copies.  The bias
 * corrections use the step count kept on the host, so a captured step would
 * replay with stale ones.  Errors: ISING_ERR_ARG (NULL pointer, lr < 0,
 * beta1 or beta2 outside [0, 1), eps <= 0), ISING_ERR_CUDA. */
int ising_cnn_adam_step(ising_cnn* net, const float* grad, float lr, float beta1, float beta2, float eps,
                        void* cuda_stream);

/*
 * ising_propose -- (learned stage, this project's extension) apply proposals
 * built from the logits, each accepted iff its exact Eq. 2 energy change dE = -2 sum_{i in B, j ~ i, j not in B} w_ij s_i s_j
 * is <= 0.
 * tile > 0: B = sites with logit > 0 in each tile of side `tile`; tiles with
 *   even (tx + ty) first, then odd.  The number of tiles along each side must
 *   be 1 or even (ISING_ERR_ARG otherwise).
 * tile = 0: B = all sites with logit > 0 (whole-lattice proposal).
 * spins    device [B][n] int8, updated in place.
 * accepted device [B] int32 or NULL: proposals taken per configuration.
 * Errors: ISING_ERR_ARG, ISING_ERR_UNSUPPORTED (a general-graph handle),
 * ISING_ERR_CUDA.
 */
int ising_propose(const ising_problem* p, int8_t* spins, int32_t B, const float* logits, int32_t tile,
                  int32_t* accepted, void* cuda_stream);

/*
 * ising_propose_clusters -- block flips built from connected components
 * (this project's learned stage; the paper's own update rule is unpublished,
 * Section III).  For each configuration, the sites with logit > 0 split into
 * connected components under 4-neighbour adjacency on the torus (periodic
 * wrap included); components are never adjacent, so flipping component C
 * changes Eq. 2's energy by its own boundary terms,
 * dE_C = -2 sum_{i in C, j ~ i, j not in C} w_ij s_i s_j, and every component
 * with dE_C <= 0 is flipped.  The energy never rises.
 * probs    m >= 1 torus problems of one shape (m <= 16); configuration
 *          q * B + b belongs to probs[q].
 * spins    device [m * B][n] int8, updated in place.
 * logits   device [m * B][n] float.
 * accepted device [m * B] int32 or NULL: components flipped per configuration.
 * One CTA per configuration with all of its state in shared memory (9 bytes
 * per site).  Errors: ISING_ERR_UNSUPPORTED above that (about 25,000 sites)
 * and for general-graph handles; ISING_ERR_ARG for mixed shapes or bad
 * pointers; ISING_ERR_CUDA when the launch fails.
 */
int ising_propose_clusters(const ising_problem* const* probs, int32_t m, int8_t* spins, int32_t B,
                           const float* logits, int32_t* accepted, void* cuda_stream);

/*
 * ising_droplet_targets -- (learned stage, this project's extension; dE from
 * Eq. 2) training targets of the cluster proposals: with
 * r' = ref or -ref gauge-aligned to s (as ising_flip_targets), the sites
 * where s and r' differ split into connected components on the torus;
 * targets_i = 1 iff i lies in a component whose flip alone lowers the energy
 * of s (dE_C < 0, dE_C as above), an exact energy-lowering move from s
 * towards r'.  spins, ref: device [B][n] int8; targets: device [B][n] uint8.
 * Limits and errors as ising_propose_clusters.
 */
int ising_droplet_targets(const ising_problem* p, const int8_t* spins, const int8_t* ref, int32_t B,
                          uint8_t* targets, void* cuda_stream);

/*
 * ising_transcribe -- partner moves: block flips whose blocks come from
 * another trial of the same instance instead of the network (this project's
 * extension of the block flips; the paper's own rule is unpublished,
 * Section III).  Configuration t of problem q takes partner
 * p = (t + shift) mod B of the same problem; the sites where s_t differs
 * from the gauge-aligned s_p (as ising_flip_targets) split into connected
 * components on the torus, and every component whose flip alone lowers the
 * energy of s_t (dE_C < 0, as ising_propose_clusters) is flipped.  All
 * configurations read the partners' states before any move: out receives
 * the new states and must not alias spins.  Each configuration's energy
 * drops by exactly the sum of its flipped components' changes.
 * probs    m (1..16) torus problems of one shape; spins / out device
 *          [m * B][n] int8; accepted device [m * B] int32 or NULL:
 *          components flipped per configuration.
 * Limits and errors as ising_propose_clusters; ISING_ERR_ARG also for
 * shift < 0 or out == spins.
 */
int ising_transcribe(const ising_problem* const* probs, int32_t m, const int8_t* spins, int8_t* out, int32_t B,
                     int32_t shift, int32_t* accepted, void* cuda_stream);

/*
 * ising_learned_create / _launch / _destroy -- the learned form of the
 * annealer for m torus problems of one shape (this project's extension; the
 * paper's own update rule is unpublished, Section III), prepared once and
 * replayed as one CUDA graph: no host round trip between its steps.
 *   1. sweeps [0, k_first) of the schedule from the Philox start, all
 *      problems in one persistent batched launch (k_first = 0: the start);
 *      with warm = 1 the network's whole-lattice proposal (ising_propose,
 *      tile 0) is applied to the start state first;
 *   2. for every chunk [k, k + every) of the rest (the last may be shorter):
 *      the chunk's sweeps, resumed at global sweep k, in one batched launch;
 *      then, with a network, its logits for each problem's configurations
 *      (ising_cnn_forward) and its block flips over all problems
 *      (ising_propose_clusters); then, with partner_period P > 0, partner
 *      moves (ising_transcribe) with offset 1 + (j mod P) in chunk j;
 *   3. the cut of every configuration (Eq. 1).
 * With no chunk (k_first = S) this is the plain annealer, bit for bit; with
 * chunks, the sweeps between proposals are the plain annealer's resumed
 * exactly, so the proposals are the only difference.
 * probs    m (1..16) torus problems of one shape, on the current device.
 * betas    host [S], seeds host [m] (problem q's decision stream).
 * net      the network or NULL (no network proposals, no warm start); its
 *          current weights are read at every launch.
 * spins    device [m * trials][n] int8: the state, written by every launch
 *          (problem q's configurations at rows q * trials ...).
 * cuts     device [m * trials] int32, written at the end of every launch.
 * accepted device [m * trials] int32 or NULL: block flips and partner
 *          components taken over all chunks, per configuration.
 * logits   device [m * trials][n] float (scratch), ws / ws_bytes: the
 *          network's workspace for `trials` configurations
 *          (ising_cnn_workspace_bytes(trials, n, 0)); needed with a network.
 *          All owned by the caller and used by every launch, so launches of
 *          one plan must not overlap.
 * The buffers and arguments are bound into the graph at creation; create
 * allocates the plan's own device memory (the thresholds of every launch and,
 * with partner moves, a second state buffer), copies the thresholds and
 * synchronises cuda_stream.  launch enqueues the graph on cuda_stream.
 * Errors: ISING_ERR_ARG (bad pointers or sizes, mixed shapes, warm start
 * without a network), ISING_ERR_UNSUPPORTED (a general-graph handle, an
 * instance the batched launch, the network or the cluster kernel cannot
 * take, or cuda_stream capturing a graph), ISING_ERR_OOM, ISING_ERR_CUDA;
 * ising_learned_launch: ISING_ERR_ARG (NULL plan), ISING_ERR_CUDA.
 * ising_learned_destroy frees the plan (NULL is a no-op) without waiting:
 * the caller must not destroy it while one of its launches is queued.
 */
typedef struct ising_learned ising_learned;
int ising_learned_create(ising_problem* const* probs, int32_t m, int32_t trials, const double* betas, int32_t S,
                         const uint64_t* seeds, int32_t k_first, int32_t every, const ising_cnn* net,
                         int32_t partner_period, int32_t warm, int8_t* spins, int32_t* cuts, int32_t* accepted,
                         float* logits, void* ws, size_t ws_bytes, void* cuda_stream, ising_learned** out);
int ising_learned_launch(ising_learned* plan, void* cuda_stream);
void ising_learned_destroy(ising_learned* plan);

/*
 * ising_flip_targets -- (learned stage, this project's extension; the global
 * flip symmetry follows from Eq. 2 with h = 0) training targets for the
 * network: for each of B
 * configurations, y_i = [s_i != r'_i] where r' is ref or -ref, whichever is
 * closer to s in Hamming distance (on a tie, the one that keeps site 0); the
 * global flip s -> -s is a symmetry of H, so only the relative orientation
 * is meaningful.  spins, ref: device [B][n] int8; targets: device [B][n] uint8.
 * Errors: ISING_ERR_ARG (B < 0, n <= 0, a NULL pointer with B > 0),
 * ISING_ERR_CUDA.
 */
int ising_flip_targets(const int8_t* spins, const int8_t* ref, int32_t B, int32_t n, uint8_t* targets,
                       void* cuda_stream);

/* ising_strerror -- static description of a status code. */
const char* ising_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* ISING_H */

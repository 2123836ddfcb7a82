/*
 * ising_oracle.c -- CPU oracle for the toroidal Ising / Max-Cut annealer.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, single-threaded
 * definition that the CUDA path is checked against.  Only the tests, the smoke
 * run and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or constant generator with the library under
 * paper_2505_18508_gb300/csrc, and it works on the general CSR graph rather
 * than on any packed or bit-sliced layout.
 *
 * What it computes (paper: Zick 2025, "Performance report of heuristic
 * algorithm that cracked the largest Gset Ising problems"):
 *
 *   - Max-Cut objective, Eq. 1: cut(x) = 1/2 sum_{i<j} w_ij (1 - x_i x_j).
 *     Written here as sum over edges of w_ij [s_i != s_j], which is the same
 *     number for x_i, s_i in {-1,+1}.
 *   - Ising Hamiltonian, Eq. 2, with J_ij = -w_ij and h_i = 0:
 *     H(s) = sum_{i<j} w_ij s_i s_j.  Flipping spin i changes H by
 *     dE_i = -2 s_i f_i, with local field f_i = sum_j w_ij s_j.
 *   - The "sweep" of Section III (one pass of update attempts over all n
 *     spins) and the read-out at the end of each trial.  The paper does not
 *     publish its update rule (Section III, Section IV), so the sweep here is
 *     a Metropolis sweep: visit colour 0 then colour 1 of the checkerboard,
 *     sites in increasing index; flip when dE <= 0, otherwise flip when the
 *     uniform 32-bit draw u is below T_dE = min(floor(exp(-beta dE) 2^32),
 *     2^32 - 1).  On a torus with even sides, same-colour sites are never
 *     adjacent, so this sequential order gives the same result as updating a
 *     whole colour at once.
 *   - Random draws: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
 *     random numbers: as easy as 1, 2, 3", SC'11), counter
 *     (site i, sweep k, trial/4, 0), key (seed low 32 bits, seed high 32
 *     bits); trial t uses output word t mod 4.  The starting spin of trial t
 *     at site i is +1 when bit 31 of word t mod 4 of the block for counter
 *     (i, 0xFFFFFFFF, t/4, 0) is set.
 *   - 16-bit draw mode (a variant of this project, not of the paper: one
 *     Philox block serves eight trials instead of four).  Trial t at site i
 *     in sweep k draws the 16-bit half (t mod 2: low half for even t, high
 *     half for odd t) of word (t mod 8)/2 of the block at counter
 *     (i, k, t/8, 0), and the thresholds are
 *     T_dE = min(floor(exp(-beta dE) 2^16), 2^16 - 1).  The starting spins
 *     are the same as in the 32-bit mode.
 *
 * Every function returns 0 on success and a negative value on bad input.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from the round function of Salmon et al. (SC'11, Sec. 5):  */
/* two 32x32->64 multiplications per round, the high halves XORed with the  */
/* other two counter words and the round key, the round key advanced by the */
/* Weyl constants after each round.                                          */
/* ------------------------------------------------------------------------ */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += ORC_PHILOX_W0;
        k1 += ORC_PHILOX_W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* one 32-bit draw: word (t mod 4) of the block at counter (a, b, t/4, 0) */
static uint32_t draw(uint32_t a, uint32_t b, int32_t t, uint64_t seed)
{
    uint32_t ctr[4] = {a, b, (uint32_t)t >> 2, 0u};
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    return out[t & 3];
}

/* one 16-bit draw: half (t mod 2) of word (t mod 8)/2 of the block at      */
/* counter (a, b, t/8, 0); the low half for even t                          */
static uint32_t draw16(uint32_t a, uint32_t b, int32_t t, uint64_t seed)
{
    uint32_t ctr[4] = {a, b, (uint32_t)t >> 3, 0u};
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    uint32_t word = out[(t & 7) >> 1];
    return (t & 1) ? (word >> 16) : (word & 0xFFFFu);
}

/* exported for the pins: the decision draw of either mode */
uint32_t oracle_draw(uint32_t i, uint32_t k, int32_t t, uint64_t seed, int32_t bits)
{
    return bits == 16 ? draw16(i, k, t, seed) : draw(i, k, t, seed);
}

/* ------------------------------------------------------------------------ */
/* Acceptance thresholds for the Metropolis test, one pair per sweep:        */
/*   T_d = min(floor(exp(-beta d) * 2^32), 2^32 - 1),  d in {4, 8}.          */
/* beta must be a positive number (+inf allowed, giving T = 0).              */
/* ------------------------------------------------------------------------ */
static int threshold_one(double beta, double d, uint32_t* out)
{
    if (!(beta > 0.0)) return -1;               /* also rejects NaN */
    double p = exp(-(beta * d));                /* Metropolis probability */
    double scaled = p * 4294967296.0;           /* times 2^32 */
    double fl = floor(scaled);
    if (fl >= 4294967295.0) *out = 0xFFFFFFFFu;
    else *out = (uint32_t)fl;
    return 0;
}

/* the 16-bit mode: T_d = min(floor(exp(-beta d) * 2^16), 2^16 - 1) */
static int threshold16_one(double beta, double d, uint32_t* out)
{
    if (!(beta > 0.0)) return -1;
    double p = exp(-(beta * d));
    double fl = floor(p * 65536.0);
    if (fl >= 65535.0) *out = 0xFFFFu;
    else *out = (uint32_t)fl;
    return 0;
}

int oracle_thresholds16(const double* betas, int32_t S, uint32_t* T4, uint32_t* T8)
{
    if (S < 0) return -1;
    for (int32_t k = 0; k < S; ++k) {
        if (threshold16_one(betas[k], 4.0, &T4[k]) != 0) return -1;
        if (threshold16_one(betas[k], 8.0, &T8[k]) != 0) return -1;
    }
    return 0;
}

int oracle_thresholds(const double* betas, int32_t S, uint32_t* T4, uint32_t* T8)
{
    if (S < 0) return -1;
    for (int32_t k = 0; k < S; ++k) {
        if (threshold_one(betas[k], 4.0, &T4[k]) != 0) return -1;
        if (threshold_one(betas[k], 8.0, &T8[k]) != 0) return -1;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Eq. 1 on a CSR graph: each undirected edge {i,j} appears as i->j and j->i */
/* with J_ij = -w_ij; count it once (i < j).                                 */
/* ------------------------------------------------------------------------ */
int32_t oracle_cut(int32_t n, const int64_t* row_ptr, const int32_t* col,
                   const int8_t* J, const int8_t* spins)
{
    int32_t cut = 0;
    for (int32_t i = 0; i < n; ++i) {
        int si = spins[i] > 0 ? 1 : -1;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int32_t j = col[e];
            if (j <= i) continue;
            int sj = spins[j] > 0 ? 1 : -1;
            int w = -(int)J[e];
            if (si != sj) cut += w;
        }
    }
    return cut;
}

/* Eq. 2 with h = 0: H = -sum_{i<j} J_ij s_i s_j. */
int64_t oracle_energy(int32_t n, const int64_t* row_ptr, const int32_t* col,
                      const int8_t* J, const int8_t* spins)
{
    int64_t H = 0;
    for (int32_t i = 0; i < n; ++i) {
        int si = spins[i] > 0 ? 1 : -1;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int32_t j = col[e];
            if (j <= i) continue;
            int sj = spins[j] > 0 ? 1 : -1;
            H -= (int64_t)J[e] * si * sj;
        }
    }
    return H;
}

/* ------------------------------------------------------------------------ */
/* The annealer.                                                             */
/*                                                                           */
/* Runs trials t_begin .. t_begin + t_count - 1 (global trial indices, which */
/* select the random stream) for S sweeps.  Sweep j of the call is global    */
/* sweep k = sweep_offset + j and uses betas[j].  X is the torus width, used */
/* only for the checkerboard colour (x + y) mod 2 of site i = y X + x.       */
/* init: NULL for the random start, else t_count x n spins (>0 means +1).    */
/* out_spins: t_count x n int8 in {-1,+1}; out_cuts: t_count Eq. 1 cuts.     */
/* check_fields != 0: after every sweep, recompute every local field from    */
/* scratch and compare with the incrementally maintained ones (returns -3 on */
/* a mismatch).                                                              */
/* Returns 0, -1 for bad arguments, -2 for a dE outside {-8,-4,0,4,8}.      */
/* ------------------------------------------------------------------------ */
/* Eq. 1 cut of the configuration s (+-1 ints) on the CSR graph */
static int32_t cut_of(int32_t n, const int64_t* row_ptr, const int32_t* col, const int8_t* J, const int* s)
{
    int32_t cut = 0;
    for (int32_t i = 0; i < n; ++i)
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
            if (col[e] > i && s[i] != s[col[e]]) cut += -(int)J[e];
    return cut;
}

/* draw_bits: 32 (the default stream) or 16 (the 16-bit draw mode).         */
/* Read-out along the trajectory (trace_every > 0): after sweep j of the    */
/* call (counting from 1) with j a multiple of trace_every or j = S, the     */
/* Eq. 1 cut goes to out_trace[p][tt] (p = 0, 1, ... in sweep order,         */
/* ceil(S / trace_every) points), and the best of those cuts per trial to   */
/* out_best[tt], with its configuration (the first one reaching it) in      */
/* out_best_spins[tt][.] when that is not NULL.  With S = 0 there are no    */
/* points; the best is then the cut of the starting configuration.          */
int oracle_anneal_trace(int32_t n, const int64_t* row_ptr, const int32_t* col, const int8_t* J,
                        int32_t X, int32_t t_begin, int32_t t_count,
                        const double* betas, int32_t S, uint64_t seed, uint32_t sweep_offset,
                        const int8_t* init, int8_t* out_spins, int32_t* out_cuts,
                        int32_t check_fields, int32_t draw_bits,
                        int32_t trace_every, int32_t* out_trace, int32_t* out_best, int8_t* out_best_spins)
{
    if (n <= 0 || X <= 0 || n % X != 0 || t_begin < 0 || t_count < 0 || S < 0) return -1;
    if (draw_bits != 32 && draw_bits != 16) return -1;
    if (trace_every < 0) return -1;
    uint32_t* T4 = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(S > 0 ? S : 1));
    uint32_t* T8 = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(S > 0 ? S : 1));
    int* s = (int*)malloc(sizeof(int) * (size_t)n);
    int* f = (int*)malloc(sizeof(int) * (size_t)n);
    int* colour = (int*)malloc(sizeof(int) * (size_t)n);
    int rc = 0;
    if (!T4 || !T8 || !s || !f || !colour) { rc = -1; goto done; }
    if (draw_bits == 16) {
        if (oracle_thresholds16(betas, S, T4, T8) != 0) { rc = -1; goto done; }
    } else {
        if (oracle_thresholds(betas, S, T4, T8) != 0) { rc = -1; goto done; }
    }
    for (int32_t i = 0; i < n; ++i) colour[i] = ((i % X) + (i / X)) & 1;

    for (int32_t tt = 0; tt < t_count; ++tt) {
        int32_t t = t_begin + tt;
        /* starting configuration */
        for (int32_t i = 0; i < n; ++i) {
            if (init) s[i] = init[(size_t)tt * n + i] > 0 ? 1 : -1;
            else s[i] = (draw((uint32_t)i, 0xFFFFFFFFu, t, seed) >> 31) ? 1 : -1;
        }
        /* local fields f_i = sum_j w_ij s_j, w = -J */
        for (int32_t i = 0; i < n; ++i) {
            int acc = 0;
            for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) acc += -(int)J[e] * s[col[e]];
            f[i] = acc;
        }
        int32_t best = 0, have_best = 0;
        for (int32_t j = 0; j < S; ++j) {
            uint32_t k = sweep_offset + (uint32_t)j;
            for (int c = 0; c < 2; ++c) {
                for (int32_t i = 0; i < n; ++i) {
                    if (colour[i] != c) continue;
                    int dE = -2 * s[i] * f[i];
                    int flip;
                    if (dE <= 0) {
                        flip = 1;
                    } else {
                        uint32_t thr;
                        if (dE == 4) thr = T4[j];
                        else if (dE == 8) thr = T8[j];
                        else { rc = -2; goto done; }
                        uint32_t u = draw_bits == 16 ? draw16((uint32_t)i, k, t, seed)
                                                     : draw((uint32_t)i, k, t, seed);
                        flip = u < thr;
                    }
                    if (flip) {
                        s[i] = -s[i];
                        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
                            f[col[e]] += 2 * (-(int)J[e]) * s[i];
                    }
                }
            }
            if (check_fields) {
                for (int32_t i = 0; i < n; ++i) {
                    int acc = 0;
                    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) acc += -(int)J[e] * s[col[e]];
                    if (acc != f[i]) { rc = -3; goto done; }
                }
            }
            if (trace_every > 0 && ((j + 1) % trace_every == 0 || j + 1 == S)) {
                int32_t c = cut_of(n, row_ptr, col, J, s);
                if (out_trace) out_trace[(size_t)((j + 1 + trace_every - 1) / trace_every - 1) * t_count + tt] = c;
                if (!have_best || c > best) {
                    best = c;
                    have_best = 1;
                    if (out_best_spins)
                        for (int32_t i = 0; i < n; ++i) out_best_spins[(size_t)tt * n + i] = (int8_t)s[i];
                }
            }
        }
        if (trace_every > 0) {
            if (!have_best) {      /* no sweeps: the starting configuration */
                best = cut_of(n, row_ptr, col, J, s);
                if (out_best_spins)
                    for (int32_t i = 0; i < n; ++i) out_best_spins[(size_t)tt * n + i] = (int8_t)s[i];
            }
            if (out_best) out_best[tt] = best;
        }
        for (int32_t i = 0; i < n; ++i) {
            if (out_spins) out_spins[(size_t)tt * n + i] = (int8_t)s[i];
        }
        if (out_cuts) out_cuts[tt] = cut_of(n, row_ptr, col, J, s);
    }
done:
    free(T4); free(T8); free(s); free(f); free(colour);
    return rc;
}

int oracle_anneal_bits(int32_t n, const int64_t* row_ptr, const int32_t* col, const int8_t* J,
                       int32_t X, int32_t t_begin, int32_t t_count,
                       const double* betas, int32_t S, uint64_t seed, uint32_t sweep_offset,
                       const int8_t* init, int8_t* out_spins, int32_t* out_cuts,
                       int32_t check_fields, int32_t draw_bits)
{
    return oracle_anneal_trace(n, row_ptr, col, J, X, t_begin, t_count, betas, S, seed, sweep_offset,
                               init, out_spins, out_cuts, check_fields, draw_bits, 0, NULL, NULL, NULL);
}

int oracle_anneal(int32_t n, const int64_t* row_ptr, const int32_t* col, const int8_t* J,
                  int32_t X, int32_t t_begin, int32_t t_count,
                  const double* betas, int32_t S, uint64_t seed, uint32_t sweep_offset,
                  const int8_t* init, int8_t* out_spins, int32_t* out_cuts,
                  int32_t check_fields)
{
    return oracle_anneal_bits(n, row_ptr, col, J, X, t_begin, t_count, betas, S, seed, sweep_offset,
                              init, out_spins, out_cuts, check_fields, 32);
}

/* ======================================================================== */
/* General sparse graphs (integer couplings J, fields h).                   */
/*                                                                          */
/* Eq. 2 in full: H(s) = -sum_{i<j} J_ij s_i s_j - sum_i h_i s_i.  Flipping */
/* spin i changes it by dE_i = 2 s_i (sum_j J_ij s_j + h_i).  The sweep      */
/* visits the colour classes of a proper colouring in order (colour 0, 1,   */
/* ...), sites in increasing index within a class; sites of one class are   */
/* never adjacent, so this equals updating a class at once.  Metropolis:    */
/* flip when dE <= 0, otherwise when the 32-bit draw (same stream as on the */
/* torus) is below T(dE) = min(floor(exp(-beta dE) 2^32), 2^32 - 1).        */
/* ======================================================================== */

/* First-fit colouring in index order: site i takes the smallest colour not */
/* used by a neighbour j < i.  Returns the number of colours (or -1).       */
int32_t oracle_greedy_colouring(int32_t n, const int64_t* row_ptr, const int32_t* col, int32_t* colour)
{
    if (n < 0) return -1;
    int32_t ncol = 0;
    int32_t cap = 64;
    int* used = (int*)calloc((size_t)cap, sizeof(int));   /* used[c] == i + 1: taken for site i */
    if (!used) return -1;
    for (int32_t i = 0; i < n; ++i) {
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int32_t j = col[e];
            if (j < i) {
                int32_t c = colour[j];
                if (c >= cap) {
                    int32_t nc = cap * 2;
                    while (nc <= c) nc *= 2;
                    int* u2 = (int*)realloc(used, sizeof(int) * (size_t)nc);
                    if (!u2) { free(used); return -1; }
                    for (int32_t q = cap; q < nc; ++q) u2[q] = 0;
                    used = u2;
                    cap = nc;
                }
                used[c] = i + 1;
            }
        }
        int32_t c = 0;
        while (c < cap && used[c] == i + 1) ++c;
        if (c >= cap) {
            int* u2 = (int*)realloc(used, sizeof(int) * (size_t)(cap * 2));
            if (!u2) { free(used); return -1; }
            for (int32_t q = cap; q < cap * 2; ++q) u2[q] = 0;
            used = u2;
            cap *= 2;
        }
        colour[i] = c;
        if (c + 1 > ncol) ncol = c + 1;
    }
    free(used);
    return ncol;
}

/* Eq. 2 with fields: H = -sum_{i<j} J_ij s_i s_j - sum_i h_i s_i */
int64_t oracle_energy_h(int32_t n, const int64_t* row_ptr, const int32_t* col, const int8_t* J,
                        const int8_t* h, const int8_t* spins)
{
    int64_t H = 0;
    for (int32_t i = 0; i < n; ++i) {
        int si = spins[i] > 0 ? 1 : -1;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int32_t j = col[e];
            if (j <= i) continue;
            int sj = spins[j] > 0 ? 1 : -1;
            H -= (int64_t)J[e] * si * sj;
        }
        if (h) H -= (int64_t)h[i] * si;
    }
    return H;
}

static uint32_t threshold_of(double beta, int dE)
{
    double fl = floor(exp(-(beta * (double)dE)) * 4294967296.0);
    return fl >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)fl;
}

/* The annealer on a general graph.  colour: a proper colouring with ncol    */
/* classes (the caller's, e.g. oracle_greedy_colouring).  h may be NULL.     */
/* Outputs as oracle_anneal: spins, and the Eq. 1 cut sum_{i<j} w_ij         */
/* [s_i != s_j] with w = -J.  Returns 0, -1 for bad arguments (including an  */
/* improper colouring or a non-positive beta), -3 on a field mismatch.       */
int oracle_anneal_graph(int32_t n, const int64_t* row_ptr, const int32_t* col, const int8_t* J,
                        const int8_t* h, const int32_t* colour, int32_t ncol,
                        int32_t t_begin, int32_t t_count, const double* betas, int32_t S, uint64_t seed,
                        uint32_t sweep_offset, const int8_t* init, int8_t* out_spins, int32_t* out_cuts,
                        int32_t check_fields)
{
    if (n <= 0 || ncol <= 0 || t_begin < 0 || t_count < 0 || S < 0) return -1;
    for (int32_t k = 0; k < S; ++k)
        if (!(betas[k] > 0.0)) return -1;
    for (int32_t i = 0; i < n; ++i) {
        if (colour[i] < 0 || colour[i] >= ncol) return -1;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
            if (col[e] == i || colour[col[e]] == colour[i]) return -1;
    }
    int* s = (int*)malloc(sizeof(int) * (size_t)n);
    int* f = (int*)malloc(sizeof(int) * (size_t)n);   /* f_i = sum_j J_ij s_j */
    int rc = 0;
    if (!s || !f) { rc = -1; goto out; }
    for (int32_t tt = 0; tt < t_count; ++tt) {
        int32_t t = t_begin + tt;
        for (int32_t i = 0; i < n; ++i) {
            if (init) s[i] = init[(size_t)tt * n + i] > 0 ? 1 : -1;
            else s[i] = (draw((uint32_t)i, 0xFFFFFFFFu, t, seed) >> 31) ? 1 : -1;
        }
        for (int32_t i = 0; i < n; ++i) {
            int acc = 0;
            for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) acc += (int)J[e] * s[col[e]];
            f[i] = acc;
        }
        for (int32_t jj = 0; jj < S; ++jj) {
            uint32_t k = sweep_offset + (uint32_t)jj;
            for (int32_t c = 0; c < ncol; ++c) {
                for (int32_t i = 0; i < n; ++i) {
                    if (colour[i] != c) continue;
                    int dE = 2 * s[i] * (f[i] + (h ? (int)h[i] : 0));
                    int flip = dE <= 0 ? 1 : draw((uint32_t)i, k, t, seed) < threshold_of(betas[jj], dE);
                    if (flip) {
                        s[i] = -s[i];
                        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) f[col[e]] += 2 * (int)J[e] * s[i];
                    }
                }
            }
            if (check_fields) {
                for (int32_t i = 0; i < n; ++i) {
                    int acc = 0;
                    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) acc += (int)J[e] * s[col[e]];
                    if (acc != f[i]) { rc = -3; goto out; }
                }
            }
        }
        if (out_spins)
            for (int32_t i = 0; i < n; ++i) out_spins[(size_t)tt * n + i] = (int8_t)s[i];
        if (out_cuts) out_cuts[tt] = cut_of(n, row_ptr, col, J, s);
    }
out:
    free(s); free(f);
    return rc;
}

// abi.cu -- the C ABI declared in include/ising.h: argument checks, instance
// packing, per-sweep thresholds and the choice of launch shape.
//
// Everything here is host code; the kernels live in anneal.cu, cut.cu and
// batched.cu.  No C++ exception leaves an extern "C" function.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <algorithm>
#include <functional>
#include <utility>
#include <vector>

#include "../../include/ising.h"
#include "internal.h"

namespace {

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// ISING_LOG >= 1: one line per anneal on stderr with the kernel and shape used
void log_launch(const ising_problem* p, int32_t trials, int32_t S) {
  if (ising::log_level() < 1) return;
  static const char* names[4] = {"?", "strip", "persistent", "graph"};
  std::fprintf(stderr, "ising: anneal n=%d trials=%d sweeps=%d kernel=%s group=%d strips=%d threads=%d grid=%d bits=%d\n",
               p->n, trials, S, names[p->last_kernel & 3], p->last_group, p->last_strips, p->last_threads,
               p->last_grid, p->draw_bits);
}

int map_cuda(cudaError_t e) {
  if (e == cudaSuccess) return ISING_OK;
  if (e == cudaErrorMemoryAllocation) return ISING_ERR_OOM;
  return ISING_ERR_CUDA;
}

// The table of ising_anneal: (T4_k, T8_k) for every sweep k (reading R3,
// ising::threshold_table).
int make_thresholds(const double* betas, int32_t S, std::vector<uint32_t>& out, int bits = 32) {
  out.assign(static_cast<size_t>(2) * (S > 0 ? S : 0), 0u);
  return S > 0 ? ising::threshold_table(betas, S, bits, out.data()) : ISING_OK;
}

// trials per group when the handle does not fix it: 32, or all trials rounded
// up to a multiple of the Philox block (4 trials, 8 in the 16-bit mode)
int default_group(const ising_problem* p, int32_t T) {
  const int unit = p->draw_bits == 16 ? 8 : 4;
  return T >= 32 ? 32 : ((T + unit - 1) / unit) * unit;
}

int num_sms_of(int device) {
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || v <= 0) v = 152;
  return v;
}

int max_smem_of(int device) {
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess || v <= 0)
    v = 227 * 1024;
  return v;
}

using Shape = ising::StripShape;

}  // namespace

// ---------------------------------------------------------------- shared host rules
namespace ising {

// Reading R3: T = min(floor(exp(-x) 2^B), 2^B - 1) for the exponent x =
// beta dE of an uphill move, the Metropolis acceptance probability
// min(1, exp(-beta dE)) as an integer threshold for a uniform B-bit draw
// (accept iff u < T).  B = 16 stores T shifted left by 16 bits: the kernels
// compare draws placed in the top half of a word.
uint32_t accept_threshold(double x, int bits) {
  const double scale = bits == 16 ? 65536.0 : 4294967296.0;
  const double top = scale - 1.0;
  const double v = std::floor(std::exp(-x) * scale);
  const uint32_t T = v >= top ? static_cast<uint32_t>(top) : static_cast<uint32_t>(v);
  return bits == 16 ? T << 16 : T;
}

int threshold_table(const double* betas, int32_t S, int bits, uint32_t* out) {
  for (int32_t k = 0; k < S; ++k) {
    const double beta = betas[k];
    if (!(beta > 0.0)) return ISING_ERR_ARG;
    out[2 * static_cast<size_t>(k)] = accept_threshold(beta * 4.0, bits);
    out[2 * static_cast<size_t>(k) + 1] = accept_threshold(beta * 8.0, bits);
  }
  return ISING_OK;
}

// threads per CTA: many warps hide the Philox dependency chains, so take
// the multiple of 32 in [768, 1024] that leaves the fewest idle item slots
// over a half-sweep (ties -> more threads); fewer when a strip has fewer items.
int pick_threads(int items) {
  if (items <= 768) return std::max(64, ((items + 31) / 32) * 32);
  int best = 1024;
  double best_eff = -1.0;
  for (int t = 768; t <= 1024; t += 32) {
    const int iters = (items + t - 1) / t;
    const double eff = static_cast<double>(items) / (static_cast<double>(iters) * t);
    if (eff > best_eff + 1e-9 || (std::fabs(eff - best_eff) <= 1e-9 && t > best)) {
      best_eff = eff;
      best = t;
    }
  }
  return best;
}

int strip_shape(const ising_problem* p, int32_t T, int32_t G, StripShape* out) {
  const int sms = num_sms_of(p->device);
  const int smem_max = max_smem_of(p->device);
  if (G == 0) G = p->cfg_group;
  if (G == 0) G = default_group(p, T);
  if (G < 4) G = 4;
  const int groups = (T + G - 1) / G;
  int C = p->cfg_strips;
  if (C == 0) {
    // widest cluster that still gives every CTA its own SM (one 1024-thread
    // CTA per SM), with at least two rows per strip
    C = 1;
    while (C < 8 && groups * (C * 2) <= sms && p->Y / (C * 2) >= 2) C *= 2;
    while (C < 16 && anneal_smem_bytes(p->H, (p->Y + C - 1) / C) > static_cast<size_t>(smem_max) &&
           (C * 2) <= p->Y)
      C *= 2;
  }
  if (C > p->Y) return ISING_ERR_UNSUPPORTED;
  const int Rmax = (p->Y + C - 1) / C;
  if (anneal_smem_bytes(p->H, Rmax) > static_cast<size_t>(smem_max)) return ISING_ERR_UNSUPPORTED;
  if (groups > 65535) return ISING_ERR_UNSUPPORTED;
  int threads = p->cfg_threads;
  if (threads == 0) threads = pick_threads(Rmax * p->H);
  out->G = G;
  out->C = C;
  out->threads = threads;
  out->Rmax = Rmax;
  return ISING_OK;
}

void record_strip_launch(ising_problem* p, int32_t trials, int32_t S, const StripShape& sh) {
  p->last_kernel = 1;
  p->last_group = sh.G;
  p->last_strips = sh.C;
  p->last_threads = sh.threads;
  p->last_grid = sh.C * ((trials + sh.G - 1) / sh.G);
  log_launch(p, trials, S);
}

}  // namespace ising

namespace {

int choose_shape(const ising_problem* p, int32_t T, Shape* out) { return ising::strip_shape(p, T, 0, out); }

// ---------------------------------------------------------------- batches
struct HostBatch {
  std::vector<ising::BatchInst> inst;
  std::vector<ising::BatchUnit> units;
  std::vector<uint32_t> thr;       // all threshold tables, concatenated
  std::vector<size_t> thr_off;     // per instance, in uint32 words
  size_t smem = 0;
  int grid = 0, threads = 0;
  // arena layout (bytes)
  size_t off_inst = 0, off_units = 0, off_counter = 0, off_thr = 0, bytes = 0;
};


// The batched launch's schedule (host only): CTAs per SM and threads, trials
// per work unit of each instance, and the units (instance, group) in the
// order the CTAs take them.  n, H, Y: each instance's spins, words per row and
// rows; blk: its trials per Philox block (4, or 8 in the 16-bit mode).
struct BatchSchedule {
  int per_sm = 0, threads = 0;
  size_t smem = 0;
  std::vector<int> G;
  std::vector<ising::BatchUnit> units;
};

int batch_schedule(int32_t m, const int32_t* n, const int32_t* H, const int32_t* Y, const int32_t* trials,
                   const int32_t* sweeps, const int32_t* blk, int32_t group_trials, int32_t ctas_per_sm, int sms,
                   int smem_max, BatchSchedule* bs) {
  size_t max_smem = 0;
  double total = 0.0;
  for (int32_t q = 0; q < m; ++q) {
    const size_t sb = ising::batched_smem_bytes(H[q], Y[q]);
    if (trials[q] > 0 && sb > max_smem) max_smem = sb;
    total += static_cast<double>(n[q]) * sweeps[q] * trials[q];
  }
  if (max_smem > static_cast<size_t>(smem_max)) return ISING_ERR_UNSUPPORTED;
  // CTAs per SM: one of 1,024 threads when the work-weighted instance has
  // enough site words per half-sweep to give every thread four or more
  // (fewer, larger CTAs also let the units keep 32 trials, see below);
  // otherwise two of 512 threads if shared memory allows.  On the
  // 96-instance batch of {50,100,140,200}x100 tori one CTA per SM measured
  // 1.72 s against 2.17 s for two.
  int per_sm = ctas_per_sm;
  if (per_sm == 0) {
    double wwords = 0.0, wsum = 0.0;
    for (int32_t q = 0; q < m; ++q) {
      const double c = static_cast<double>(n[q]) * sweeps[q] * trials[q];
      wwords += c * (n[q] / 2);
      wsum += c;
    }
    per_sm = (wsum > 0.0 && wwords / wsum >= 4.0 * 1024) ? 1 : 2;
    if (max_smem > 0 && static_cast<size_t>(per_sm) * (max_smem + 1024) > 228 * 1024) per_sm = 1;
  }
  if (max_smem > 0 && static_cast<size_t>(per_sm) * (max_smem + 1024) > 228 * 1024) return ISING_ERR_UNSUPPORTED;
  const int grid = sms * per_sm;
  bs->per_sm = per_sm;
  bs->threads = 1024 / per_sm;
  bs->smem = max_smem;
  // Trials per unit.  A unit's cost is modelled as n (S + 1) (3 + its Philox
  // blocks per site word): the word's own work (field count, loads, store)
  // is about three blocks' worth.  An instance whose 32-trial unit fits in a
  // CTA's average load keeps 32 trials per unit.  The others ("large") share
  // one width G, a multiple of the Philox block from 32 down to one block:
  // the G whose units give the shortest makespan when the CTAs take them
  // longest first (list scheduling, as the kernel's atomic counter does).
  // Ties go to the wider unit.  On 8 instances of 200x100 with 512 trials
  // each, G = 28 gives 152 units for 152 CTAs (18 of 28 trials and one of 8
  // per instance).
  const double per_cta = total / (grid > 0 ? grid : 1);
  std::vector<char> large(static_cast<size_t>(m), 0);
  bool any_large = false;
  int blk_large = 4;
  for (int32_t q = 0; q < m; ++q) {
    const double unit32 = static_cast<double>(n[q]) * sweeps[q] * 32.0;
    if (group_trials == 0 && trials[q] > 0 && unit32 > per_cta && per_cta > 0) {
      large[q] = 1;
      any_large = true;
      if (blk[q] > blk_large) blk_large = blk[q];
    }
  }
  auto unit_cost = [&](int32_t q, int live) {
    return static_cast<double>(n[q]) * (sweeps[q] + 1) * (3.0 + (live + blk[q] - 1) / blk[q]);
  };
  auto widths = [&](int g_large, std::vector<int>& G) {
    G.assign(static_cast<size_t>(m), 32);
    for (int32_t q = 0; q < m; ++q) {
      if (group_trials != 0) G[q] = group_trials;
      else if (large[q]) G[q] = g_large;
    }
  };
  auto units_of = [&](const std::vector<int>& G, std::vector<std::pair<double, ising::BatchUnit>>& order) {
    order.clear();
    for (int32_t q = 0; q < m; ++q) {
      const int groups = (trials[q] + G[q] - 1) / G[q];
      for (int g = 0; g < groups; ++g) order.push_back({unit_cost(q, std::min(G[q], trials[q] - g * G[q])),
                                                        ising::BatchUnit{q, g}});
    }
    std::stable_sort(order.begin(), order.end(),
                     [](const std::pair<double, ising::BatchUnit>& x, const std::pair<double, ising::BatchUnit>& y) {
                       return x.first > y.first;
                     });
  };
  auto makespan = [&](const std::vector<std::pair<double, ising::BatchUnit>>& order) {
    std::vector<double> busy(static_cast<size_t>(grid > 0 ? grid : 1), 0.0);   // min-heap of CTA finish times
    for (const auto& u : order) {
      std::pop_heap(busy.begin(), busy.end(), std::greater<double>());
      busy.back() += u.first;
      std::push_heap(busy.begin(), busy.end(), std::greater<double>());
    }
    return *std::max_element(busy.begin(), busy.end());
  };
  std::vector<std::pair<double, ising::BatchUnit>> order;
  std::vector<int> G;
  int g_best = 32;
  if (any_large) {
    // narrower units only add units: stop before a simulation would take
    // more than ~2^20 of them (such batches keep 32 trials per unit)
    constexpr size_t kMaxSimUnits = size_t(1) << 20;
    double best = 0.0;
    for (int g = 32; g >= blk_large; g -= blk_large) {
      widths(g, G);
      size_t count = 0;
      for (int32_t q = 0; q < m; ++q) count += static_cast<size_t>((trials[q] + G[q] - 1) / G[q]);
      if (count > kMaxSimUnits) break;
      units_of(G, order);
      const double ms = makespan(order);
      if (g == 32 || ms < best) {
        best = ms;
        g_best = g;
      }
    }
  }
  widths(g_best, G);
  units_of(G, order);
  bs->G = G;
  bs->units.resize(order.size());
  for (size_t u = 0; u < order.size(); ++u) bs->units[u] = order[u].second;
  return ISING_OK;
}

int prepare_batch(ising_problem* const* probs, int32_t m, const int32_t* trials, const int32_t* sweeps,
                  const double* const* betas, const uint64_t* seeds, int8_t* const* out_spins,
                  int32_t* const* out_cuts, int32_t group_trials, int32_t ctas_per_sm, HostBatch& hb,
                  const int8_t* const* init_spins = nullptr, uint32_t sweep_offset = 0) {
  if (m < 0 || (m > 0 && (!probs || !trials || !sweeps || !betas || !seeds))) return ISING_ERR_ARG;
  if (group_trials != 0 && (group_trials < 4 || group_trials > 32 || group_trials % 4)) return ISING_ERR_ARG;
  if (ctas_per_sm < 0 || ctas_per_sm > 4) return ISING_ERR_ARG;
  int device = 0;
  for (int32_t q = 0; q < m; ++q) {
    if (!probs[q] || trials[q] < 0 || sweeps[q] < 0 || (sweeps[q] > 0 && !betas[q])) return ISING_ERR_ARG;
    if (probs[q]->graph) return ISING_ERR_UNSUPPORTED;
    if (q == 0) device = probs[q]->device;
    else if (probs[q]->device != device) return ISING_ERR_ARG;
  }
  hb.inst.resize(m);
  hb.thr_off.resize(m);
  std::vector<int32_t> vn(m), vH(m), vY(m), vblk(m);
  for (int32_t q = 0; q < m; ++q) {
    std::vector<uint32_t> t;
    if (probs[q]->draw_bits == 16 && group_trials % 8) return ISING_ERR_ARG;
    const int rc = make_thresholds(betas[q], sweeps[q], t, probs[q]->draw_bits);
    if (rc != ISING_OK) return rc;
    hb.thr_off[q] = hb.thr.size();
    hb.thr.insert(hb.thr.end(), t.begin(), t.end());
    vn[q] = probs[q]->n;
    vH[q] = probs[q]->H;
    vY[q] = probs[q]->Y;
    vblk[q] = probs[q]->draw_bits == 16 ? 8 : 4;   // trials per Philox block
  }
  BatchSchedule bs;
  const int rc = batch_schedule(m, vn.data(), vH.data(), vY.data(), trials, sweeps, vblk.data(), group_trials,
                                ctas_per_sm, num_sms_of(device),
                                max_smem_of(device) - static_cast<int>(ising::batched_static_smem()), &bs);
  if (rc != ISING_OK) return rc;
  hb.grid = num_sms_of(device) * bs.per_sm;
  hb.threads = bs.threads;
  hb.smem = bs.smem;
  for (int32_t q = 0; q < m; ++q) {
    const ising_problem* p = probs[q];
    ising::BatchInst& in = hb.inst[q];
    in.flags = p->d_flags;
    in.thr = nullptr;  // patched once the arena address is known
    in.init = init_spins ? init_spins[q] : nullptr;
    in.k0 = sweep_offset;
    in.out_spins = out_spins ? out_spins[q] : nullptr;
    in.out_cuts = out_cuts ? out_cuts[q] : nullptr;
    in.X = p->X; in.Y = p->Y; in.H = p->H; in.n = p->n;
    in.T = trials[q]; in.S = sweeps[q];
    in.key0 = static_cast<uint32_t>(seeds[q] & 0xFFFFFFFFull);
    in.key1 = static_cast<uint32_t>(seeds[q] >> 32);
    in.neg_edges = p->neg_edges;
    in.G = bs.G[q];
    in.u16 = p->draw_bits == 16 ? 1 : 0;
  }
  hb.units.swap(bs.units);
  hb.off_inst = 0;
  hb.off_units = align256(sizeof(ising::BatchInst) * hb.inst.size());
  hb.off_counter = hb.off_units + align256(sizeof(ising::BatchUnit) * hb.units.size());
  hb.off_thr = hb.off_counter + 256;
  hb.bytes = hb.off_thr + align256(sizeof(uint32_t) * hb.thr.size());
  return ISING_OK;
}

// host image of the arena once its device address is known
std::vector<unsigned char> arena_image(HostBatch& hb, unsigned char* d_arena) {
  std::vector<unsigned char> img(hb.bytes, 0);
  for (size_t q = 0; q < hb.inst.size(); ++q)
    hb.inst[q].thr = reinterpret_cast<const uint32_t*>(d_arena + hb.off_thr) + hb.thr_off[q];
  if (!hb.inst.empty())
    std::memcpy(img.data() + hb.off_inst, hb.inst.data(), sizeof(ising::BatchInst) * hb.inst.size());
  if (!hb.units.empty())
    std::memcpy(img.data() + hb.off_units, hb.units.data(), sizeof(ising::BatchUnit) * hb.units.size());
  if (!hb.thr.empty()) std::memcpy(img.data() + hb.off_thr, hb.thr.data(), sizeof(uint32_t) * hb.thr.size());
  return img;
}

ising::BatchArgs batch_args(const HostBatch& hb, unsigned char* d_arena) {
  ising::BatchArgs a;
  a.inst = reinterpret_cast<const ising::BatchInst*>(d_arena + hb.off_inst);
  a.units = reinterpret_cast<const ising::BatchUnit*>(d_arena + hb.off_units);
  a.n_units = static_cast<int32_t>(hb.units.size());
  a.counter = reinterpret_cast<uint32_t*>(d_arena + hb.off_counter);
  return a;
}

// ---------------------------------------------------------------- flow kernel plan
struct FlowPlan {
  int G = 0, groups = 0, RT = 0, P = 0, LRmax = 0;
  int cap = 0, use_rec = 0;   // items per colour of the largest CTA (multiple of 32); fast-path records
  size_t smem = 0;
  std::vector<int32_t> split;
};

// The persistent kernel's split of the stacked site words (word w = row * H
// + h, rows of all trial groups stacked) over P CTAs: ranges of equal weight,
// a word weighing the Philox blocks of its trial group (weighted) or 1.  A
// range may start and end inside a row: such a row is shared by two CTAs,
// which then read it, and its neighbours, through the global mirror.  With
// whole_rows the ranges end at row boundaries.  Fills split[0..P] and
// returns the largest number of local rows (own rows, plus two halo slots per
// segment that is not a whole trial group) and segments of any CTA.
struct FlowSplit {
  int P = 0, RT = 0, LRmax = 0, max_segments = 0;
  std::vector<int32_t> split;
};

int flow_split(int32_t Y, int32_t H, int32_t T, int32_t G, int32_t blk, int32_t sms, bool weighted,
               bool whole_rows, FlowSplit* fs) {
  if (Y < 1 || H < 1 || T < 1 || G < 1 || blk < 1 || sms < 1) return ISING_ERR_ARG;
  const int groups = (T + G - 1) / G;
  const long long RTl = static_cast<long long>(groups) * Y;
  if (RTl > (1LL << 30) || RTl * H > (1LL << 30)) return ISING_ERR_UNSUPPORTED;
  const int RT = static_cast<int>(RTl);
  const int P = std::min(sms, RT);
  std::vector<long long> cum(static_cast<size_t>(RT) + 1, 0);   // weight of rows before u
  std::vector<int> wrow(static_cast<size_t>(RT));
  for (int u = 0; u < RT; ++u) {
    const int g = u / Y;
    const int live = std::min(G, T - g * G);
    wrow[u] = weighted ? (live + blk - 1) / blk : 1;
    cum[u + 1] = cum[u] + wrow[u];
  }
  const long long total = cum[RT] * H;
  const int W = RT * H;
  std::vector<int32_t> split(static_cast<size_t>(P) + 1);
  split[0] = 0;
  int u = 0;
  for (int j = 1; j < P; ++j) {
    const long long target = (static_cast<long long>(j) * total + P / 2) / P;
    while (u < RT && cum[u + 1] * H <= target) ++u;
    int v = W;
    if (u < RT) {
      const long long rem = target - cum[u] * H;   // weight still needed inside row u
      const long long h = (rem + wrow[u] - 1) / wrow[u];
      v = u * H + static_cast<int>(std::min<long long>(h, H));
    }
    if (whole_rows) v = (v + H - 1) / H * H;
    const int unit = whole_rows ? H : 1;
    if (v <= split[j - 1]) v = split[j - 1] + unit;
    if (v > W - (P - j) * unit) v = W - (P - j) * unit;
    split[j] = v;
  }
  split[P] = W;
  int LRmax = 0, segmax = 0;
  for (int j = 0; j < P; ++j) {
    int lr = 0, nseg = 0;
    for (int w = split[j]; w < split[j + 1];) {
      const int r = w / H, g = r / Y;
      const int wend = std::min(split[j + 1], (g + 1) * Y * H);
      const int n = (wend - 1) / H - r + 1;
      const bool whole = wend - w == Y * H;
      lr += n + (whole ? 0 : 2);
      ++nseg;
      w = wend;
    }
    LRmax = std::max(LRmax, lr);
    segmax = std::max(segmax, nseg);
  }
  fs->P = P;
  fs->RT = RT;
  fs->LRmax = LRmax;
  fs->max_segments = segmax;
  fs->split.swap(split);
  return ISING_OK;
}

// Plans the persistent kernel's launch for T trials: the split above (the
// caller falls back to the unweighted split when a ragged last group would
// pile its light rows onto a few CTAs beyond their shared memory).  In the
// 16-bit draw mode, where a word's own work is cheaper, the extra mirror
// traffic of shared rows costs more than the finer balance gains (measured on
// the 200 x 100 torus with 1,024 trials), so there the ranges end at row
// boundaries.  Fails with ISING_ERR_UNSUPPORTED when a CTA would touch more
// groups than the kernel tracks or its rows would not fit in shared memory.
int plan_flow(const ising_problem* p, int32_t T, FlowPlan* fp, bool weighted = true) {
  const int sms = num_sms_of(p->device);
  const int smem_max = max_smem_of(p->device) - static_cast<int>(ising::flow_static_smem());
  int G = p->cfg_group;
  if (G == 0) G = default_group(p, T);
  const int blk = p->draw_bits == 16 ? 8 : 4;
  const int H = p->H;
  FlowSplit fs;
  const int rc = flow_split(p->Y, H, T, G, blk, sms, weighted, p->draw_bits == 16, &fs);
  if (rc != ISING_OK) return rc;
  if (fs.max_segments > ising::flow_max_segments()) return ISING_ERR_UNSUPPORTED;
  const int LRmax = fs.LRmax;
  const int groups = (T + G - 1) / G;
  const int RT = fs.RT, P = fs.P;
  std::vector<int32_t>& split = fs.split;
  // the kernel's tables hold shared-memory word indices in 16 bits
  if (2LL * LRmax * H + 1 > 0xFFFF) return ISING_ERR_UNSUPPORTED;
  // the kernel's fast path keeps two 16-byte records per item and colour and
  // a 16-bit byte offset of each local row's counter: used when they fit
  int items_max = 0;
  for (int q = 0; q < P; ++q) items_max = std::max(items_max, split[q + 1] - split[q]);
  const int cap = (items_max + 31) / 32 * 32;
  int use_rec = 1;
  size_t smem = ising::flow_smem_bytes(LRmax, p->H, cap, 1);
  if (smem > static_cast<size_t>(smem_max) || 8LL * (LRmax + 2) >= 65536) {
    use_rec = 0;
    smem = ising::flow_smem_bytes(LRmax, p->H, cap, 0);
  }
  if (smem > static_cast<size_t>(smem_max)) return ISING_ERR_UNSUPPORTED;
  fp->G = G;
  fp->groups = groups;
  fp->RT = RT;
  fp->P = P;
  fp->LRmax = LRmax;
  fp->cap = cap;
  fp->use_rec = use_rec;
  fp->smem = smem;
  fp->split.swap(split);
  return ISING_OK;
}

}  // namespace

// A flow-kernel run prepared once for repeated launches: its plan and a
// device arena of (optional) thresholds | split | zeroed before every launch:
// the tagged mirror, cut sums, done, abort.
struct FlowRun {
  ising_problem* p = nullptr;
  FlowPlan fp;
  int32_t trials = 0;
  unsigned char* d = nullptr;
  size_t o_split = 0, o_gm = 0, o_zero = 0, o_acc = 0, o_done = 0, o_abort = 0, bytes = 0;
};

namespace ising {

int flow_run_create(ising_problem* p, int32_t trials, size_t thr_words, FlowRun** out, cudaStream_t st) {
  *out = nullptr;
  FlowRun* r = nullptr;
  try {
    r = new FlowRun();
    int frc = plan_flow(p, trials, &r->fp);
    if (frc == ISING_ERR_UNSUPPORTED) frc = plan_flow(p, trials, &r->fp, false);
    if (frc != ISING_OK) { delete r; return frc; }
  } catch (const std::bad_alloc&) {
    delete r;
    return ISING_ERR_OOM;
  }
  const FlowPlan& fp = r->fp;
  int per_sm = 0;
  cudaError_t e = flow_max_ctas(fp.smem, &per_sm);
  if (e == cudaSuccess && (per_sm < 1 || fp.P > per_sm * num_sms_of(p->device))) {
    delete r;
    return ISING_ERR_UNSUPPORTED;
  }
  r->p = p;
  r->trials = trials;
  r->o_split = align256(thr_words * sizeof(uint32_t));
  r->o_zero = r->o_split + align256(fp.split.size() * sizeof(int32_t));
  r->o_gm = r->o_zero;   // the tagged mirror is zeroed before every launch
  r->o_acc = r->o_gm + align256(static_cast<size_t>(fp.RT) * 2 * p->H * sizeof(unsigned long long));
  r->o_done = r->o_acc + align256(static_cast<size_t>(trials) * sizeof(int32_t));
  r->o_abort = r->o_done + 256;
  r->bytes = r->o_abort + 256;
  if (e == cudaSuccess) e = dev_malloc_async(reinterpret_cast<void**>(&r->d), r->bytes, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(r->d + r->o_split, fp.split.data(), fp.split.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                        st);
  if (e != cudaSuccess) {
    if (r->d) cudaFreeAsync(r->d, st);
    delete r;
    return map_cuda(e);
  }
  *out = r;
  return ISING_OK;
}

uint32_t* flow_run_thresholds(FlowRun* r) { return reinterpret_cast<uint32_t*>(r->d); }

int flow_run_launch(FlowRun* r, const uint32_t* d_thr, int32_t thr_group_stride, int32_t S, uint32_t k0,
                    uint64_t seed, const int8_t* init_spins, int8_t* out_spins, int32_t* out_cuts, cudaStream_t st) {
  ising_problem* p = r->p;
  const FlowPlan& fp = r->fp;
  cudaError_t e = cudaMemsetAsync(r->d + r->o_zero, 0, r->bytes - r->o_zero, st);
  if (e == cudaSuccess) {
    FlowArgs a;
    a.flags = p->d_flags;
    a.thr = d_thr;
    a.thr_group_stride = thr_group_stride;
    a.init = init_spins;
    a.out_spins = out_spins;
    a.out_cuts = out_cuts;
    a.X = p->X; a.Y = p->Y; a.H = p->H; a.n = p->n;
    a.T = r->trials; a.G = fp.G; a.S = S;
    a.k0 = k0;
    a.key0 = static_cast<uint32_t>(seed & 0xFFFFFFFFull);
    a.key1 = static_cast<uint32_t>(seed >> 32);
    for (uint32_t q = 0; q < 10; ++q) {
      a.rk[2 * q] = a.key0 + q * 0x9E3779B9u;
      a.rk[2 * q + 1] = a.key1 + q * 0xBB67AE85u;
    }
    a.RT = fp.RT;
    a.P = fp.P;
    a.LRmax = fp.LRmax;
    a.neg_edges = p->neg_edges;
    a.split = reinterpret_cast<const int32_t*>(r->d + r->o_split);
    a.gm = reinterpret_cast<unsigned long long*>(r->d + r->o_gm);
    a.acc = reinterpret_cast<int32_t*>(r->d + r->o_acc);
    a.done = reinterpret_cast<uint32_t*>(r->d + r->o_done);
    a.abort_flag = reinterpret_cast<uint32_t*>(r->d + r->o_abort);
    a.status = p->d_status;
    a.spin_limit = p->wait_limit > 0 ? p->wait_limit : 4000000000LL;
    a.stall_test = p->stall_test;
    a.u16 = p->draw_bits == 16 ? 1 : 0;
    a.cap = fp.cap;
    a.use_rec = fp.use_rec;
    e = launch_flow(a, st);
  }
  if (e != cudaSuccess) return map_cuda(e);
  p->last_kernel = 2;
  p->last_group = fp.G;
  p->last_strips = 0;
  p->last_threads = flow_threads();
  p->last_grid = fp.P;
  return ISING_OK;
}

void flow_run_destroy(FlowRun* r, cudaStream_t st) {
  if (!r) return;
  if (r->d) cudaFreeAsync(r->d, st);
  delete r;
}

}  // namespace ising

namespace {

int run_flow(ising_problem* p, int32_t trials, const std::vector<uint32_t>& thr, int32_t S, uint64_t seed,
             uint32_t sweep_offset, const int8_t* init_spins, int8_t* out_spins, int32_t* out_cuts, cudaStream_t st) {
  FlowRun* r = nullptr;
  int rc = ising::flow_run_create(p, trials, thr.size(), &r, st);
  if (rc != ISING_OK) return rc;
  cudaError_t e = cudaSuccess;
  if (!thr.empty())
    e = cudaMemcpyAsync(ising::flow_run_thresholds(r), thr.data(), thr.size() * sizeof(uint32_t),
                        cudaMemcpyHostToDevice, st);
  rc = e == cudaSuccess ? ising::flow_run_launch(r, ising::flow_run_thresholds(r), 0, S, sweep_offset, seed,
                                                 init_spins, out_spins, out_cuts, st)
                        : map_cuda(e);
  ising::flow_run_destroy(r, st);
  if (rc == ISING_OK) log_launch(p, trials, S);
  return rc;
}


// ---------------------------------------------------------------- general graphs
// First-fit colouring in index order: site i takes the smallest colour that
// no neighbour j < i holds.  stamp[c] == i + 1 marks colour c as taken for i.
int32_t first_fit(int32_t n, const int64_t* row_ptr, const int32_t* col, std::vector<int32_t>& colour) {
  colour.assign(static_cast<size_t>(n), 0);
  std::vector<int32_t> stamp(16, 0);
  int32_t ncol = 0;
  for (int32_t i = 0; i < n; ++i) {
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
      const int32_t j = col[e];
      if (j >= i) continue;
      const int32_t c = colour[j];
      if (static_cast<size_t>(c) >= stamp.size()) stamp.resize(static_cast<size_t>(c) * 2 + 2, 0);
      stamp[c] = i + 1;
    }
    int32_t c = 0;
    while (static_cast<size_t>(c) < stamp.size() && stamp[c] == i + 1) ++c;
    colour[i] = c;
    ncol = std::max(ncol, c + 1);
  }
  return ncol;
}

ising::GraphArgs graph_args(const ising_problem* p) {
  ising::GraphArgs a{};
  a.nb = p->d_nb;
  a.rowinfo = p->d_rowinfo;
  a.sites = p->d_sites;
  a.colour_off = p->d_colour_off;
  a.n = p->n;
  a.n_pad = (p->n + 3) & ~3;
  a.thr_pad = (p->Dmax + 1 + 3) & ~3;
  a.Dmax = p->Dmax;
  a.planes = p->planes;
  a.ncol = p->ncol;
  return a;
}

int run_graph(ising_problem* p, int32_t trials, const double* betas, int32_t S, uint64_t seed,
              uint32_t sweep_offset, const int8_t* init_spins, int8_t* out_spins, int32_t* out_cuts,
              cudaStream_t st) {
  if (p->draw_bits != 32) return ISING_ERR_UNSUPPORTED;
  // T(dE) = min(floor(exp(-beta dE) 2^32), 2^32 - 1) for dE = 2q, q = 1 .. Dmax
  std::vector<uint32_t> thr;
  try {
    thr.assign(static_cast<size_t>(S) * p->Dmax, 0u);
  } catch (const std::bad_alloc&) {
    return ISING_ERR_OOM;
  }
  for (int32_t k = 0; k < S; ++k) {
    if (!(betas[k] > 0.0)) return ISING_ERR_ARG;
    for (int32_t q = 1; q <= p->Dmax; ++q) {
      const double v = std::floor(std::exp(-(betas[k] * (2.0 * q))) * 4294967296.0);
      thr[static_cast<size_t>(k) * p->Dmax + (q - 1)] = v >= 4294967295.0 ? 0xFFFFFFFFu : static_cast<uint32_t>(v);
    }
  }
  if (trials == 0) return ISING_OK;
  const int sms = num_sms_of(p->device);
  const int groups = (trials + 31) / 32;
  if (groups > 65535) return ISING_ERR_UNSUPPORTED;
  int C = p->cfg_strips;
  if (C == 0) {
    C = 1;
    while (C < 8 && groups * (C * 2) <= sms) C *= 2;
  }
  if (C > 8) return ISING_ERR_UNSUPPORTED;
  uint32_t* d_thr = nullptr;
  const size_t bytes = thr.size() * sizeof(uint32_t);
  if (bytes) {
    cudaError_t e = ising::dev_malloc_async(reinterpret_cast<void**>(&d_thr), bytes, st);
    if (e != cudaSuccess) return map_cuda(e);
    e = cudaMemcpyAsync(d_thr, thr.data(), bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) { cudaFreeAsync(d_thr, st); return map_cuda(e); }
  }
  ising::GraphArgs a = graph_args(p);
  a.thr = d_thr;
  a.init = init_spins;
  a.out_spins = out_spins;
  a.out_cuts = out_cuts;
  a.T = trials;
  a.S = S;
  a.C = C;
  a.k0 = sweep_offset;
  a.key0 = static_cast<uint32_t>(seed & 0xFFFFFFFFull);
  a.key1 = static_cast<uint32_t>(seed >> 32);
  for (uint32_t r = 0; r < 10; ++r) {   // Philox round keys (Weyl sequence)
    a.rk[2 * r] = a.key0 + r * 0x9E3779B9u;
    a.rk[2 * r + 1] = a.key1 + r * 0xBB67AE85u;
  }
  // threads per site word: a team of 8 or 4 when a CTA's share of an average
  // colour class leaves most of its threads idle (small graphs), else 1
  int tpw = p->cfg_graph_tpw;
  if (tpw == 0) {
    const double words = static_cast<double>(p->n) / (p->ncol > 0 ? p->ncol : 1) / C;
    const double slots = 2.0 * ising::graph_threads();
    tpw = words * 8 <= slots ? 8 : (words * 4 <= slots ? 4 : 1);
  }
  a.tpw = tpw;
  cudaError_t e = ising::launch_graph(a, st);
  if (d_thr) {
    const cudaError_t e2 = cudaFreeAsync(d_thr, st);
    if (e == cudaSuccess) e = e2;
  }
  if (e != cudaSuccess) return map_cuda(e);
  p->last_kernel = 3;
  p->last_group = 32;
  p->last_strips = C;
  p->last_threads = ising::graph_threads();
  p->last_grid = C * groups;
  log_launch(p, trials, S);
  return ISING_OK;
}
}  // namespace

extern "C" {

const char* ising_strerror(int code) {
  switch (code) {
    case ISING_OK: return "ok";
    case ISING_ERR_ARG: return "invalid argument";
    case ISING_ERR_NOT_TORUS: return "CSR is not a symmetric 4-neighbour torus of the given shape";
    case ISING_ERR_ODD_DIM: return "torus width and height must be even";
    case ISING_ERR_H_UNSUPPORTED: return "non-zero local fields h are not supported";
    case ISING_ERR_OOM: return "out of memory";
    case ISING_ERR_CUDA: return "CUDA error";
    case ISING_ERR_TIMEOUT: return "bounded device wait timed out";
    case ISING_ERR_UNSUPPORTED: return "valid input outside what this library supports";
    default: return "unknown status code";
  }
}

int ising_create(int32_t n, const int64_t* row_ptr, const int32_t* col_idx, const int8_t* J,
                 const int8_t* h, int32_t X, int32_t Y, ising_problem** out) {
  if (!row_ptr || !col_idx || !J || !out) return ISING_ERR_ARG;
  if (X < 4 || Y < 4) return ISING_ERR_ARG;
  if ((X & 1) || (Y & 1)) return ISING_ERR_ODD_DIM;
  if (static_cast<int64_t>(X) * Y != n || n > (1 << 28)) return ISING_ERR_ARG;
  if (row_ptr[0] != 0) return ISING_ERR_NOT_TORUS;
  for (int32_t i = 0; i < n; ++i)
    if (row_ptr[i + 1] - row_ptr[i] != 4) return ISING_ERR_NOT_TORUS;
  if (h) {
    for (int32_t i = 0; i < n; ++i)
      if (h[i] != 0) return ISING_ERR_H_UNSUPPORTED;
  }
  // J of each site towards left, right, up, down
  std::vector<int8_t> jl, jr, ju, jd;
  try {
    jl.resize(n); jr.resize(n); ju.resize(n); jd.resize(n);
  } catch (const std::bad_alloc&) {
    return ISING_ERR_OOM;
  }
  for (int32_t y = 0; y < Y; ++y) {
    for (int32_t x = 0; x < X; ++x) {
      const int32_t i = y * X + x;
      const int32_t want[4] = {y * X + (x + X - 1) % X, y * X + (x + 1) % X, ((y + Y - 1) % Y) * X + x,
                               ((y + 1) % Y) * X + x};
      bool seen[4] = {false, false, false, false};
      int8_t val[4] = {0, 0, 0, 0};
      for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
        const int8_t v = J[e];
        if (v != 1 && v != -1) return ISING_ERR_ARG;
        int which = -1;
        for (int d = 0; d < 4; ++d)
          if (col_idx[e] == want[d]) which = d;
        if (which < 0 || seen[which]) return ISING_ERR_NOT_TORUS;
        seen[which] = true;
        val[which] = v;
      }
      jl[i] = val[0]; jr[i] = val[1]; ju[i] = val[2]; jd[i] = val[3];
    }
  }
  // symmetry J_ij = J_ji
  for (int32_t y = 0; y < Y; ++y)
    for (int32_t x = 0; x < X; ++x) {
      const int32_t i = y * X + x;
      if (jr[i] != jl[y * X + (x + 1) % X]) return ISING_ERR_NOT_TORUS;
      if (jd[i] != ju[((y + 1) % Y) * X + x]) return ISING_ERR_NOT_TORUS;
    }
  // pack: w = -J, flag bit set where w = -1, i.e. J = +1
  const int32_t H = X / 2;
  std::vector<uint8_t> flags(n), eflags(n);
  int32_t neg = 0;
  for (int32_t y = 0; y < Y; ++y)
    for (int32_t x = 0; x < X; ++x) {
      const int32_t i = y * X + x;
      const int c = (x + y) & 1;
      const uint8_t f = static_cast<uint8_t>((jl[i] == 1 ? 1 : 0) | (jr[i] == 1 ? 2 : 0) | (ju[i] == 1 ? 4 : 0) |
                                             (jd[i] == 1 ? 8 : 0));
      flags[(static_cast<size_t>(c) * Y + y) * H + (x >> 1)] = f;
      eflags[i] = static_cast<uint8_t>((jr[i] == 1 ? 1 : 0) | (jd[i] == 1 ? 2 : 0));
      neg += (jr[i] == 1) + (jd[i] == 1);
    }
  ising_problem* p = new (std::nothrow) ising_problem();
  if (!p) return ISING_ERR_OOM;
  p->X = X; p->Y = Y; p->n = n; p->H = H;
  p->neg_edges = neg;
  p->weight_sum = 2 * n - 2 * neg;
  if (cudaGetDevice(&p->device) != cudaSuccess) { delete p; return ISING_ERR_CUDA; }
  cudaError_t e = ising::dev_malloc(&p->d_flags, n);
  if (e == cudaSuccess) e = ising::dev_malloc(&p->d_eflags, n);
  if (e == cudaSuccess) e = ising::dev_malloc(reinterpret_cast<void**>(&p->d_status), sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemset(p->d_status, 0, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemcpy(p->d_flags, flags.data(), n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_eflags, eflags.data(), n, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(p->d_flags);
    cudaFree(p->d_eflags);
    cudaFree(p->d_status);
    delete p;
    return map_cuda(e);
  }
  *out = p;
  return ISING_OK;
}

void ising_destroy(ising_problem* p) {
  if (!p) return;
  cudaFree(p->d_flags);
  cudaFree(p->d_eflags);
  cudaFree(p->d_status);
  cudaFree(p->d_nb);
  cudaFree(p->d_rowinfo);
  cudaFree(p->d_sites);
  cudaFree(p->d_colour_off);
  delete p;
}

int ising_set_launch(ising_problem* p, int32_t group_trials, int32_t strips, int32_t threads) {
  if (!p) return ISING_ERR_ARG;
  if (group_trials != 0 && (group_trials < 4 || group_trials > 32 || group_trials % 4)) return ISING_ERR_ARG;
  if (strips != 0 && (strips < 1 || strips > 16 || (p->graph ? strips > 8 : strips > p->Y))) return ISING_ERR_ARG;
  if (threads != 0 && (threads < 64 || threads > 1024 || threads % 32)) return ISING_ERR_ARG;
  p->cfg_group = group_trials;
  p->cfg_strips = strips;
  p->cfg_threads = threads;
  return ISING_OK;
}

int ising_last_launch(const ising_problem* p, int32_t* group_trials, int32_t* strips, int32_t* threads,
                      int32_t* grid_ctas) {
  if (!p) return ISING_ERR_ARG;
  if (group_trials) *group_trials = p->last_group;
  if (strips) *strips = p->last_strips;
  if (threads) *threads = p->last_threads;
  if (grid_ctas) *grid_ctas = p->last_grid;
  return ISING_OK;
}

int ising_set_draw_bits(ising_problem* p, int32_t bits) {
  if (!p || (bits != 32 && bits != 16)) return ISING_ERR_ARG;
  p->draw_bits = bits;
  return ISING_OK;
}

int ising_batch_schedule(int32_t m, const int32_t* X, const int32_t* Y, const int32_t* trials, const int32_t* sweeps,
                         int32_t draw_bits, int32_t group_trials, int32_t ctas_per_sm, int32_t sms,
                         int32_t smem_per_cta_max, int32_t* per_sm, int32_t* threads, int32_t* G, int32_t* units,
                         int32_t cap, int32_t* nunits) {
  if (m < 0 || (m > 0 && (!X || !Y || !trials || !sweeps || !G)) || !per_sm || !threads || !nunits ||
      !(draw_bits == 32 || draw_bits == 16) || sms < 1 || ctas_per_sm < 0 || ctas_per_sm > 4)
    return ISING_ERR_ARG;
  if (group_trials != 0 && (group_trials < 4 || group_trials > 32 || group_trials % (draw_bits == 16 ? 8 : 4)))
    return ISING_ERR_ARG;
  std::vector<int32_t> n(m), H(m), blk(m, draw_bits == 16 ? 8 : 4);
  for (int32_t q = 0; q < m; ++q) {
    if (X[q] < 4 || Y[q] < 4 || X[q] % 2 || Y[q] % 2 || trials[q] < 0 || sweeps[q] < 0) return ISING_ERR_ARG;
    n[q] = X[q] * Y[q];
    H[q] = X[q] / 2;
  }
  BatchSchedule bs;
  int rc;
  try {
    rc = batch_schedule(m, n.data(), H.data(), Y, trials, sweeps, blk.data(), group_trials, ctas_per_sm, sms,
                        smem_per_cta_max > 0 ? smem_per_cta_max : 227 * 1024, &bs);
  } catch (const std::bad_alloc&) {
    return ISING_ERR_OOM;
  }
  if (rc != ISING_OK) return rc;
  *per_sm = bs.per_sm;
  *threads = bs.threads;
  for (int32_t q = 0; q < m; ++q) G[q] = bs.G[q];
  *nunits = static_cast<int32_t>(bs.units.size());
  if (units) {
    if (cap < *nunits) return ISING_ERR_ARG;
    for (size_t u = 0; u < bs.units.size(); ++u) {
      units[2 * u] = bs.units[u].inst;
      units[2 * u + 1] = bs.units[u].group;
    }
  }
  return ISING_OK;
}

int ising_thresholds(const double* betas, int32_t S, int32_t draw_bits, uint32_t* out) {
  if (S < 0 || (S > 0 && (!betas || !out)) || (draw_bits != 32 && draw_bits != 16)) return ISING_ERR_ARG;
  std::vector<uint32_t> t;
  try {
    const int rc = make_thresholds(betas, S, t, draw_bits);
    if (rc != ISING_OK) return rc;
  } catch (const std::bad_alloc&) {
    return ISING_ERR_OOM;
  }
  if (!t.empty()) std::memcpy(out, t.data(), t.size() * sizeof(uint32_t));
  return ISING_OK;
}

int ising_flow_split(int32_t Y, int32_t H, int32_t trials, int32_t group_trials, int32_t draw_bits, int32_t sms,
                     int32_t weighted, int32_t* split_out, int32_t cap, int32_t* ctas, int32_t* local_rows_max,
                     int32_t* segments_max) {
  if (!(draw_bits == 32 || draw_bits == 16) || group_trials < 1 || group_trials > 32 || !split_out || !ctas)
    return ISING_ERR_ARG;
  FlowSplit fs;
  int rc;
  try {
    rc = flow_split(Y, H, trials, group_trials, draw_bits == 16 ? 8 : 4, sms, weighted != 0, draw_bits == 16, &fs);
  } catch (const std::bad_alloc&) {
    return ISING_ERR_OOM;
  }
  if (rc != ISING_OK) return rc;
  if (cap < fs.P + 1) return ISING_ERR_ARG;
  std::memcpy(split_out, fs.split.data(), sizeof(int32_t) * (fs.P + 1));
  *ctas = fs.P;
  if (local_rows_max) *local_rows_max = fs.LRmax;
  if (segments_max) *segments_max = fs.max_segments;
  return ISING_OK;
}

int ising_set_graph_threads_per_site(ising_problem* p, int32_t threads_per_site) {
  if (!p || !(threads_per_site == 0 || threads_per_site == 1 || threads_per_site == 4 || threads_per_site == 8))
    return ISING_ERR_ARG;
  p->cfg_graph_tpw = threads_per_site;
  return ISING_OK;
}

int ising_set_kernel(ising_problem* p, int32_t kind) {
  if (!p || kind < 0 || kind > 2) return ISING_ERR_ARG;
  p->cfg_kernel = kind;
  return ISING_OK;
}

int ising_last_kernel(const ising_problem* p, int32_t* kind) {
  if (!p || !kind) return ISING_ERR_ARG;
  *kind = p->last_kernel;
  return ISING_OK;
}

int ising_get_status(ising_problem* p, void* cuda_stream, int32_t* code) {
  if (!p || !code) return ISING_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (const int crc = ising::refuse_capture(st)) return crc;
  int32_t v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, p->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->d_status, 0, sizeof(int32_t), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return map_cuda(e);
  *code = v;
  return ISING_OK;
}

int ising_set_wait_limit(ising_problem* p, int64_t cycles, int32_t stall_test) {
  if (!p || cycles < 0 || stall_test < 0 || stall_test > 1) return ISING_ERR_ARG;
  p->wait_limit = cycles;
  p->stall_test = stall_test;
  return ISING_OK;
}

int ising_problem_info(const ising_problem* p, int32_t* X, int32_t* Y, int32_t* weight_sum) {
  if (!p) return ISING_ERR_ARG;
  if (X) *X = p->X;
  if (Y) *Y = p->Y;
  if (weight_sum) *weight_sum = p->weight_sum;
  return ISING_OK;
}

int ising_anneal(ising_problem* p, int32_t trials, const double* betas, int32_t S, uint64_t seed,
                 uint32_t sweep_offset, const int8_t* init_spins, int8_t* out_spins, int32_t* out_cuts,
                 void* cuda_stream) {
  if (!p || trials < 0 || S < 0 || (S > 0 && !betas)) return ISING_ERR_ARG;
  if (const int crc = ising::refuse_capture(static_cast<cudaStream_t>(cuda_stream))) return crc;
  if (p->graph)
    return run_graph(p, trials, betas, S, seed, sweep_offset, init_spins, out_spins, out_cuts,
                     static_cast<cudaStream_t>(cuda_stream));
  if (p->draw_bits == 16 && p->cfg_group % 8) return ISING_ERR_ARG;
  std::vector<uint32_t> thr;
  try {
    const int rc = make_thresholds(betas, S, thr, p->draw_bits);
    if (rc != ISING_OK) return rc;
  } catch (const std::bad_alloc&) {
    return ISING_ERR_OOM;
  }
  if (trials == 0) return ISING_OK;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // kernel: the persistent flow kernel when the instance is large enough and
  // its stacked rows give every SM at least four (unless the handle fixes a
  // kernel or a strip shape), else the cluster-strip kernel
  int kind = p->cfg_kernel;
  if (kind == 0) {
    const long long rows = static_cast<long long>((trials + 31) / 32) * p->Y;
    kind = (p->cfg_strips == 0 && p->n >= 2048 && rows >= 4LL * num_sms_of(p->device)) ? 2 : 1;
  }
  if (kind == 2) {
    const int frc = run_flow(p, trials, thr, S, seed, sweep_offset, init_spins, out_spins, out_cuts, st);
    if (frc != ISING_ERR_UNSUPPORTED || p->cfg_kernel == 2) return frc;
  }
  Shape sh;
  const int rc = choose_shape(p, trials, &sh);
  if (rc != ISING_OK) return rc;
  uint32_t* d_thr = nullptr;
  const size_t thr_bytes = thr.size() * sizeof(uint32_t);
  if (thr_bytes) {
    cudaError_t e = ising::dev_malloc_async(reinterpret_cast<void**>(&d_thr), thr_bytes, st);
    if (e != cudaSuccess) return map_cuda(e);
    e = cudaMemcpyAsync(d_thr, thr.data(), thr_bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) { cudaFreeAsync(d_thr, st); return map_cuda(e); }
  }
  ising::AnnealArgs a{};
  a.flags = p->d_flags;
  a.thr = d_thr;
  a.init = init_spins;
  a.out_spins = out_spins;
  a.out_cuts = out_cuts;
  a.X = p->X; a.Y = p->Y; a.H = p->H; a.n = p->n;
  a.T = trials;
  a.G = sh.G;
  a.S = S;
  a.k0 = sweep_offset;
  a.key0 = static_cast<uint32_t>(seed & 0xFFFFFFFFull);
  a.key1 = static_cast<uint32_t>(seed >> 32);
  for (uint32_t r = 0; r < 10; ++r) {   // Philox round keys (Weyl sequence)
    a.rk[2 * r] = a.key0 + r * 0x9E3779B9u;
    a.rk[2 * r + 1] = a.key1 + r * 0xBB67AE85u;
  }
  a.C = sh.C;
  a.Rmax = sh.Rmax;
  a.neg_edges = p->neg_edges;
  a.u16 = p->draw_bits == 16 ? 1 : 0;
  cudaError_t e = ising::launch_anneal(a, sh.threads, st);
  if (d_thr) {
    const cudaError_t e2 = cudaFreeAsync(d_thr, st);
    if (e == cudaSuccess) e = e2;
  }
  if (e != cudaSuccess) return map_cuda(e);
  ising::record_strip_launch(p, trials, S, sh);
  return ISING_OK;
}

int ising_cut(const ising_problem* p, const int8_t* spins, int32_t k, int32_t* out_cuts, void* cuda_stream) {
  if (!p || k < 0 || (k > 0 && (!spins || !out_cuts))) return ISING_ERR_ARG;
  if (p->graph)
    return map_cuda(ising::launch_graph_measure(graph_args(p), spins, k, out_cuts, nullptr,
                                                static_cast<cudaStream_t>(cuda_stream)));
  return map_cuda(ising::launch_cut(p, spins, k, out_cuts, static_cast<cudaStream_t>(cuda_stream)));
}

int ising_anneal_batched(ising_problem* const* probs, int32_t m, const int32_t* trials, const int32_t* sweeps,
                         const double* const* betas, const uint64_t* seeds, int8_t* const* out_spins,
                         int32_t* const* out_cuts, void* cuda_stream) {
  if (const int crc = ising::refuse_capture(static_cast<cudaStream_t>(cuda_stream))) return crc;
  HostBatch hb;
  try {
    const int rc = prepare_batch(probs, m, trials, sweeps, betas, seeds, out_spins, out_cuts, 0, 0, hb);
    if (rc != ISING_OK) return rc;
  } catch (const std::bad_alloc&) {
    return ISING_ERR_OOM;
  }
  if (hb.units.empty()) return ISING_OK;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  unsigned char* d_arena = nullptr;
  cudaError_t e = ising::batched_prepare(hb.smem);
  if (e != cudaSuccess) return map_cuda(e);
  e = ising::dev_malloc_async(reinterpret_cast<void**>(&d_arena), hb.bytes, st);
  if (e != cudaSuccess) return map_cuda(e);
  std::vector<unsigned char> img;
  try {
    img = arena_image(hb, d_arena);
  } catch (const std::bad_alloc&) {
    cudaFreeAsync(d_arena, st);
    return ISING_ERR_OOM;
  }
  e = cudaMemcpyAsync(d_arena, img.data(), hb.bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = ising::launch_batched(batch_args(hb, d_arena), hb.grid, hb.threads, hb.smem, st);
  const cudaError_t e2 = cudaFreeAsync(d_arena, st);
  if (e == cudaSuccess) e = e2;
  return map_cuda(e);
}

struct ising_batch {
  unsigned char* d_arena = nullptr;
  cudaStream_t capture = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t done = nullptr;
};

void ising_batch_destroy(ising_batch* b) {
  if (!b) return;
  if (b->done) cudaEventSynchronize(b->done);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->done) cudaEventDestroy(b->done);
  if (b->capture) cudaStreamDestroy(b->capture);
  if (b->d_arena) cudaFree(b->d_arena);
  delete b;
}

int ising_batch_create(ising_problem* const* probs, int32_t m, const int32_t* trials, const int32_t* sweeps,
                       const double* const* betas, const uint64_t* seeds, int8_t* const* out_spins,
                       int32_t* const* out_cuts, int32_t group_trials, int32_t ctas_per_sm, void* cuda_stream,
                       ising_batch** out) {
  if (!out) return ISING_ERR_ARG;
  if (const int crc = ising::refuse_capture(static_cast<cudaStream_t>(cuda_stream))) return crc;
  HostBatch hb;
  try {
    const int rc = prepare_batch(probs, m, trials, sweeps, betas, seeds, out_spins, out_cuts, group_trials,
                                 ctas_per_sm, hb);
    if (rc != ISING_OK) return rc;
  } catch (const std::bad_alloc&) {
    return ISING_ERR_OOM;
  }
  ising_batch* b = new (std::nothrow) ising_batch();
  if (!b) return ISING_ERR_OOM;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = ising::dev_malloc(reinterpret_cast<void**>(&b->d_arena), hb.bytes);
  std::vector<unsigned char> img;
  if (e == cudaSuccess) {
    try {
      img = arena_image(hb, b->d_arena);
    } catch (const std::bad_alloc&) {
      ising_batch_destroy(b);
      return ISING_ERR_OOM;
    }
    e = cudaMemcpyAsync(b->d_arena, img.data(), hb.bytes, cudaMemcpyHostToDevice, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = ising::batched_prepare(hb.smem);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    const ising::BatchArgs a = batch_args(hb, b->d_arena);
    cudaError_t ec = cudaMemsetAsync(a.counter, 0, sizeof(uint32_t), b->capture);
    if (ec == cudaSuccess) ec = ising::launch_batched(a, hb.grid, hb.threads, hb.smem, b->capture);
    e = cudaStreamEndCapture(b->capture, &b->graph);
    if (e == cudaSuccess) e = ec;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e != cudaSuccess) {
    ising_batch_destroy(b);
    return map_cuda(e);
  }
  *out = b;
  return ISING_OK;
}

int ising_batch_launch(ising_batch* b, void* cuda_stream) {
  if (!b || !b->exec) return ISING_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaGraphLaunch(b->exec, st);
  if (e == cudaSuccess) e = cudaEventRecord(b->done, st);
  return map_cuda(e);
}

// ---------------------------------------------------------------- learned form as one graph
struct ising_learned {
  unsigned char* d_arena = nullptr;   // the batch arenas of every annealing launch
  int8_t* d_other = nullptr;          // second state buffer of the partner moves
  cudaStream_t capture = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

void ising_learned_destroy(ising_learned* L) {
  if (!L) return;
  if (L->exec) cudaGraphExecDestroy(L->exec);
  if (L->graph) cudaGraphDestroy(L->graph);
  if (L->capture) cudaStreamDestroy(L->capture);
  if (L->d_arena) cudaFree(L->d_arena);
  if (L->d_other) cudaFree(L->d_other);
  delete L;
}

int ising_learned_create(ising_problem* const* probs, int32_t m, int32_t trials, const double* betas, int32_t S,
                         const uint64_t* seeds, int32_t k_first, int32_t every, const ising_cnn* net,
                         int32_t partner_period, int32_t warm, int8_t* spins, int32_t* cuts, int32_t* accepted,
                         float* logits, void* ws, size_t ws_bytes, void* cuda_stream, ising_learned** out) {
  if (!out || !probs || m < 1 || m > 16 || trials < 1 || S < 0 || (S > 0 && !betas) || !seeds || k_first < 0 ||
      k_first > S || every < 1 || partner_period < 0 || warm < 0 || warm > 1 || (warm && !net) || !spins || !cuts ||
      (net && (!logits || !ws)))
    return ISING_ERR_ARG;
  if (const int crc = ising::refuse_capture(static_cast<cudaStream_t>(cuda_stream))) return crc;
  for (int32_t q = 0; q < m; ++q) {
    if (!probs[q]) return ISING_ERR_ARG;
    if (probs[q]->graph) return ISING_ERR_UNSUPPORTED;
    if (probs[q]->X != probs[0]->X || probs[q]->Y != probs[0]->Y || probs[q]->device != probs[0]->device)
      return ISING_ERR_ARG;
  }
  *out = nullptr;
  const size_t n = static_cast<size_t>(probs[0]->n);
  const size_t state_bytes = static_cast<size_t>(m) * trials * n;
  ising_learned* L = new (std::nothrow) ising_learned();
  if (!L) return ISING_ERR_OOM;
  cudaError_t e = cudaSuccess;
  if (partner_period > 0) e = ising::dev_malloc(reinterpret_cast<void**>(&L->d_other), state_bytes);
  if (e != cudaSuccess) {
    ising_learned_destroy(L);
    return map_cuda(e);
  }
  int8_t* A = spins;
  int8_t* B2 = L->d_other;
  // the annealing launches: the start (warm: its sweeps follow the warm
  // start as a second launch), then one per window chunk [k, k + len),
  // resumed at global sweep k from the state of the previous step (after a
  // partner move that is the second buffer)
  struct Step {
    int32_t k0, len;
    const int8_t* init;   // null: the Philox start
    bool chunk;           // a window chunk: proposals follow
  };
  std::vector<Step> steps;
  if (warm) {
    steps.push_back({0, 0, nullptr, false});
    if (k_first > 0) steps.push_back({0, k_first, A, false});
  } else {
    steps.push_back({0, k_first, nullptr, false});
  }
  {
    int32_t j = 0;
    for (int32_t k = k_first; k < S; k += every, ++j)
      steps.push_back({k, std::min(every, S - k), (partner_period > 0 && j > 0) ? B2 : A, true});
  }
  std::vector<HostBatch> batches(steps.size());
  std::vector<size_t> base(steps.size());
  size_t total = 0;
  try {
    std::vector<int8_t*> outs(m);
    std::vector<const int8_t*> inits(m);
    const std::vector<int32_t> vt(m, trials);
    for (size_t c = 0; c < steps.size(); ++c) {
      for (int32_t q = 0; q < m; ++q) {
        outs[q] = A + static_cast<size_t>(q) * trials * n;
        inits[q] = steps[c].init ? steps[c].init + static_cast<size_t>(q) * trials * n : nullptr;
      }
      const std::vector<int32_t> vs(m, steps[c].len);
      const std::vector<const double*> vb(m, betas ? betas + steps[c].k0 : nullptr);
      const int rc = prepare_batch(probs, m, vt.data(), vs.data(), vb.data(), seeds, outs.data(), nullptr, 0, 0,
                                   batches[c], steps[c].init ? inits.data() : nullptr,
                                   static_cast<uint32_t>(steps[c].k0));
      if (rc != ISING_OK) {
        ising_learned_destroy(L);
        return rc;
      }
      base[c] = total;
      total += align256(batches[c].bytes);
    }
  } catch (const std::bad_alloc&) {
    ising_learned_destroy(L);
    return ISING_ERR_OOM;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  e = ising::dev_malloc(reinterpret_cast<void**>(&L->d_arena), total);
  try {
    for (size_t c = 0; c < batches.size() && e == cudaSuccess; ++c) {
      const std::vector<unsigned char> img = arena_image(batches[c], L->d_arena + base[c]);
      e = cudaMemcpy(L->d_arena + base[c], img.data(), batches[c].bytes, cudaMemcpyHostToDevice);
    }
  } catch (const std::bad_alloc&) {
    ising_learned_destroy(L);
    return ISING_ERR_OOM;
  }
  if (e == cudaSuccess) e = ising::batched_prepare(batches[0].smem);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    ising_learned_destroy(L);
    return map_cuda(e);
  }
  // the whole learned anneal as one graph
  int rc = ISING_OK;
  e = cudaStreamCreateWithFlags(&L->capture, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(L->capture, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaStream_t cs = L->capture;
    cudaError_t ec = accepted ? cudaMemsetAsync(accepted, 0, sizeof(int32_t) * m * trials, cs) : cudaSuccess;
    auto logits_of = [&](int32_t q) {
      for (int32_t r = q; r < q + 1 && rc == ISING_OK; ++r)
        rc = ising::cnn_forward_ws(net, probs[r], A + static_cast<size_t>(r) * trials * n, trials,
                                   logits + static_cast<size_t>(r) * trials * n, ws, ws_bytes, cs);
    };
    int32_t j = 0;
    for (size_t c = 0; c < steps.size() && ec == cudaSuccess && rc == ISING_OK; ++c) {
      const ising::BatchArgs a = batch_args(batches[c], L->d_arena + base[c]);
      ec = cudaMemsetAsync(a.counter, 0, sizeof(uint32_t), cs);
      if (ec == cudaSuccess)
        ec = ising::launch_batched(a, batches[c].grid, batches[c].threads, batches[c].smem, cs);
      if (ec != cudaSuccess) break;
      if (warm && c == 0) {   // warm start: the network's whole-lattice proposal on the start state
        for (int32_t q = 0; q < m && rc == ISING_OK; ++q) {
          logits_of(q);
          if (rc == ISING_OK)
            rc = ising_propose(probs[q], A + static_cast<size_t>(q) * trials * n, trials,
                               logits + static_cast<size_t>(q) * trials * n, 0, nullptr, cs);
        }
        continue;
      }
      if (!steps[c].chunk) continue;
      if (net) {   // the network's logits per instance, then its block flips over all
        for (int32_t q = 0; q < m && rc == ISING_OK; ++q) logits_of(q);
        if (rc == ISING_OK) rc = ising::propose_clusters_launch(probs, m, A, trials, logits, accepted, 1, cs);
      }
      if (partner_period > 0 && rc == ISING_OK)   // partner moves into the second buffer
        rc = ising::transcribe_launch(probs, m, A, B2, trials, 1 + j % partner_period, accepted, 1, cs);
      ++j;
    }
    if (ec == cudaSuccess && rc == ISING_OK && partner_period > 0 && j > 0)
      ec = cudaMemcpyAsync(A, B2, state_bytes, cudaMemcpyDeviceToDevice, cs);
    for (int32_t q = 0; q < m && ec == cudaSuccess && rc == ISING_OK; ++q)
      ec = ising::launch_cut(probs[q], A + static_cast<size_t>(q) * trials * n, trials,
                             cuts + static_cast<size_t>(q) * trials, cs);
    e = cudaStreamEndCapture(cs, &L->graph);
    if (e == cudaSuccess) e = ec;
  }
  if (e == cudaSuccess && rc == ISING_OK) e = cudaGraphInstantiate(&L->exec, L->graph, 0);
  if (e != cudaSuccess || rc != ISING_OK) {
    ising_learned_destroy(L);
    return rc != ISING_OK ? rc : map_cuda(e);
  }
  *out = L;
  return ISING_OK;
}

int ising_learned_launch(ising_learned* L, void* cuda_stream) {
  if (!L || !L->exec) return ISING_ERR_ARG;
  return map_cuda(cudaGraphLaunch(L->exec, static_cast<cudaStream_t>(cuda_stream)));
}

int ising_greedy_colouring(int32_t n, const int64_t* row_ptr, const int32_t* col_idx, int32_t* colour,
                           int32_t* ncol) {
  if (n < 0 || (n > 0 && (!row_ptr || !col_idx || !colour)) || !ncol) return ISING_ERR_ARG;
  std::vector<int32_t> c;
  try {
    *ncol = first_fit(n, row_ptr, col_idx, c);
  } catch (const std::bad_alloc&) {
    return ISING_ERR_OOM;
  }
  if (n > 0) std::memcpy(colour, c.data(), sizeof(int32_t) * static_cast<size_t>(n));
  return ISING_OK;
}

int ising_graph_create(int32_t n, const int64_t* row_ptr, const int32_t* col_idx, const int8_t* J,
                       const int8_t* h, ising_problem** out) {
  if (!row_ptr || !col_idx || !J || !out || n <= 0) return ISING_ERR_ARG;
  if (n > (1 << 24)) return ISING_ERR_UNSUPPORTED;
  if (row_ptr[0] != 0) return ISING_ERR_ARG;
  for (int32_t i = 0; i < n; ++i)
    if (row_ptr[i + 1] < row_ptr[i]) return ISING_ERR_ARG;
  const int64_t nnz = row_ptr[n];
  if (nnz > (int64_t(1) << 31)) return ISING_ERR_UNSUPPORTED;
  std::vector<uint32_t> nb;
  std::vector<int4> rowinfo;
  std::vector<int32_t> colour, sites, off;
  int32_t Dmax = 0, ncol = 0;
  int64_t wsum = 0;
  try {
    nb.resize(static_cast<size_t>(nnz));
    rowinfo.resize(static_cast<size_t>(n));
    // entries, self loops, repeats; per-row sorted copies for the symmetry test
    std::vector<std::pair<int32_t, int8_t>> rows(static_cast<size_t>(nnz));
    for (int32_t i = 0; i < n; ++i) {
      int32_t D = 0;
      for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
        const int32_t j = col_idx[e];
        const int8_t v = J[e];
        if (j < 0 || j >= n || j == i || v == 0 || v == -128) return ISING_ERR_ARG;
        rows[e] = {j, v};
        const int32_t mag = v < 0 ? -v : v;
        D += mag;
        nb[e] = static_cast<uint32_t>(j) | (v < 0 ? (1u << 24) : 0u) | (static_cast<uint32_t>(mag - 1) << 25);
        if (j > i) wsum -= v;
      }
      std::sort(rows.begin() + row_ptr[i], rows.begin() + row_ptr[i + 1]);
      for (int64_t e = row_ptr[i] + 1; e < row_ptr[i + 1]; ++e)
        if (rows[e].first == rows[e - 1].first) return ISING_ERR_ARG;
      int32_t hv = 0;
      if (h) {
        if (h[i] == -128) return ISING_ERR_ARG;
        hv = h[i];
      }
      D += hv < 0 ? -hv : hv;
      if (D > 255) return ISING_ERR_UNSUPPORTED;
      Dmax = std::max(Dmax, D);
      rowinfo[i] = make_int4(static_cast<int>(row_ptr[i]), static_cast<int>(row_ptr[i + 1] - row_ptr[i]), hv, D);
    }
    for (int32_t i = 0; i < n; ++i)
      for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
        const int32_t j = rows[e].first;
        const auto b = rows.begin() + row_ptr[j], en = rows.begin() + row_ptr[j + 1];
        const auto it = std::lower_bound(b, en, std::make_pair(i, static_cast<int8_t>(-128)));
        if (it == en || it->first != i || it->second != rows[e].second) return ISING_ERR_ARG;
      }
    ncol = first_fit(n, row_ptr, col_idx, colour);
    off.assign(static_cast<size_t>(ncol) + 1, 0);
    for (int32_t i = 0; i < n; ++i) ++off[colour[i] + 1];
    for (int32_t c = 0; c < ncol; ++c) off[c + 1] += off[c];
    sites.resize(static_cast<size_t>(n));
    std::vector<int32_t> fill(off.begin(), off.end() - 1);
    for (int32_t i = 0; i < n; ++i) sites[fill[colour[i]]++] = i;
  } catch (const std::bad_alloc&) {
    return ISING_ERR_OOM;
  }
  int planes = 1;
  while ((1 << planes) <= Dmax) ++planes;
  ising_problem* p = new (std::nothrow) ising_problem();
  if (!p) return ISING_ERR_OOM;
  p->graph = 1;
  p->n = n;
  p->nnz = nnz;
  p->ncol = ncol;
  p->Dmax = Dmax;
  p->planes = planes;
  p->weight_sum = static_cast<int32_t>(wsum);
  if (cudaGetDevice(&p->device) != cudaSuccess) { delete p; return ISING_ERR_CUDA; }
  if (ising::graph_smem_bytes(n, Dmax) > static_cast<size_t>(max_smem_of(p->device))) {
    delete p;
    return ISING_ERR_UNSUPPORTED;
  }
  cudaError_t e = ising::dev_malloc(reinterpret_cast<void**>(&p->d_status), sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemset(p->d_status, 0, sizeof(int32_t));
  if (e == cudaSuccess && nnz) e = ising::dev_malloc(reinterpret_cast<void**>(&p->d_nb), sizeof(uint32_t) * nnz);
  if (e == cudaSuccess) e = ising::dev_malloc(reinterpret_cast<void**>(&p->d_rowinfo), sizeof(int4) * n);
  if (e == cudaSuccess) e = ising::dev_malloc(reinterpret_cast<void**>(&p->d_sites), sizeof(int32_t) * n);
  if (e == cudaSuccess) e = ising::dev_malloc(reinterpret_cast<void**>(&p->d_colour_off), sizeof(int32_t) * (ncol + 1));
  if (e == cudaSuccess && nnz)
    e = cudaMemcpy(p->d_nb, nb.data(), sizeof(uint32_t) * nnz, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_rowinfo, rowinfo.data(), sizeof(int4) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_sites, sites.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(p->d_colour_off, off.data(), sizeof(int32_t) * (ncol + 1), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    ising_destroy(p);
    return map_cuda(e);
  }
  *out = p;
  return ISING_OK;
}

int ising_graph_info(const ising_problem* p, int32_t* n, int32_t* ncol, int32_t* Dmax) {
  if (!p || !p->graph) return ISING_ERR_ARG;
  if (n) *n = p->n;
  if (ncol) *ncol = p->ncol;
  if (Dmax) *Dmax = p->Dmax;
  return ISING_OK;
}

int ising_energy(const ising_problem* p, const int8_t* spins, int32_t k, int64_t* out_energies, void* cuda_stream) {
  if (!p || k < 0 || (k > 0 && (!spins || !out_energies))) return ISING_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (p->graph)
    return map_cuda(ising::launch_graph_measure(graph_args(p), spins, k, nullptr,
                                                reinterpret_cast<long long*>(out_energies), st));
  // torus (h = 0): H = W - 2 cut
  if (k == 0) return ISING_OK;
  int32_t* tmp = nullptr;
  cudaError_t e = ising::dev_malloc_async(reinterpret_cast<void**>(&tmp), sizeof(int32_t) * k, st);
  if (e != cudaSuccess) return map_cuda(e);
  e = ising::launch_cut(p, spins, k, tmp, st);
  if (e == cudaSuccess) e = ising::launch_energy_from_cut(tmp, p->weight_sum, k, out_energies, st);
  const cudaError_t e2 = cudaFreeAsync(tmp, st);
  if (e == cudaSuccess) e = e2;
  return map_cuda(e);
}

}  // extern "C"

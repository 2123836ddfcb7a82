"""Benchmark: spin-updates/s and time-to-99.9%-cut of the plain GPU annealer.

Workload (one "step"): the 200x100 toroidal +-1 instance (20,000 spins,
instance seed 2), 1,024 trials x 10,000 Metropolis sweeps, beta linear
0.1 -> 3.0, Philox seed 1002 + step; spins and exact cuts of every trial are
produced on the device.  A step is T*S*n = 2.048e11 spin updates.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
    python bench.py --leg NAME [leg options]      # one secondary workload alone

N > 1 (torchrun): every rank runs the full workload with its own seeds
(independent trials, weak scaling), no collective on the data path.

Output (rank 0): one JSON line per secondary workload ("leg": draw16,
batched, graph, pt, campaign, learned), each with its full detail, then the
headline as the LAST line: a compact object with the metric, the roofline,
the CPU baseline, the clocks and a one-number summary of every leg.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "spin-updates/s; time-to-99.9%-cut on 200x100 +-1 torus, learned vs plain"
WORKLOAD = {"X": 200, "Y": 100, "inst_seed": 2, "trials": 1024, "sweeps": 10000, "beta0": 0.1, "beta1": 3.0,
            "seed": 1002}
WORKLOAD_NAME = "plain annealer, 200x100 +-1 torus (20,000 spins), 1,024 trials x 10,000 sweeps, beta 0.1->3.0"
# the small 50x50 workload (64 trials x 1,000 sweeps, instance seed 1, seed 1001)
SMALL = {"X": 50, "Y": 50, "inst_seed": 1, "trials": 64, "sweeps": 1000, "beta0": 0.1, "beta1": 3.0,
         "seed": 1001}
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
PEAK_HBM_GBS = float(json.load(open(PEAKS_FILE)).get("hbm_gbs", 6800.0)) if os.path.exists(PEAKS_FILE) else 6800.0
# Integer multiply lanes per SM per clock (32-bit IMAD; a 32x32->64 multiply
# counts as two): 4 sub-partitions x 16 lanes.  The integer-pipe probe
# (tests/alu_peak.cu, run by tests/test_gpu_alu_peak.py) measured 64.07
# mad.lo per clock per SM on the GB300.
IMAD_LANES_PER_SM = 64
# Philox4x32-10 multiplies per spin update: 10 rounds x 2 products x 2 halves / 4 draws
IMAD_OPS_PER_UPDATE = 10
# DRAM bytes (read + write) of one launch of the persistent annealing kernel
# on this workload (the timed launch, after the L2 flush), from an ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum, --clock-control none) of the
# same launch configuration: 3,113,472 + 176,896 bytes
FLOW_TRAFFIC_BYTES = 3113472 + 176896
# the headline line stays well inside what a log tail keeps
HEADLINE_MAX_BYTES = 6144
HEADLINE_KEYS = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                 "scaling", "vs_baseline", "dtype", "data", "config", "e2e", "gpu_launches", "roofline",
                 "cpu_baseline", "clocks")

CNN_FLOP_PER_SITE = 2 * 9 * (3 * 32 + 32 * 32 * 2 + 32 * 1)
CNN_BYTES_PER_SITE = 1 + 3 * 2 * 64 + 4   # spins in, three BF16 maps written and read, FP32 logits out
PROPOSE_BYTES_PER_SITE = 1 + 4 + 1        # spins read and written, FP32 logits read


def updates_per_step(w):
    return w["trials"] * w["sweeps"] * w["X"] * w["Y"]


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.proc = None
        self.path = None
        self.device_index = device_index

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device_index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[4], f[5], f[6], f[7], f[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        sm = sorted(r[0] for r in rows)
        reasons = set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            for nm, v in zip(names, r[3:]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r[1] for r in rows), "reasons": sorted(reasons),
                "samples": len(rows)}


def _cuda_time(fn, reps=1):
    """Milliseconds per call of fn(), CUDA events on the current stream."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


# ------------------------------------------------------------------ CPU oracle
def _oracle_job(args):
    import oracle  # test infrastructure: the CPU baseline legs only
    inst, betas, seed, t_begin, t_count, sweep_offset = args
    t = time.perf_counter()
    _, cuts = oracle.anneal(inst, betas, seed, t_begin=t_begin, t_count=t_count, sweep_offset=sweep_offset)
    return time.perf_counter() - t, cuts


def _oracle_pool(jobs, procs):
    """Run oracle jobs in `procs` spawned processes; (wall seconds, results)."""
    import multiprocessing as mp
    import oracle
    oracle.lib()  # build before starting workers
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(procs) as pool:
        res = pool.map(_oracle_job, jobs)
    return time.perf_counter() - t0, res


def oracle_sample_jobs(w, inst, procs, sweeps):
    """A bounded, stratified sample of the workload: process p runs trial p
    over `sweeps` consecutive sweeps of the schedule starting at sweep
    p * S / procs (from that trial's start spins), so that the sample covers
    the whole temperature range."""
    betas = synth.linear_betas(w["beta0"], w["beta1"], w["sweeps"])
    jobs = []
    for p in range(procs):
        k0 = min(w["sweeps"] - sweeps, (p * w["sweeps"]) // procs)
        jobs.append((inst, betas[k0:k0 + sweeps], w["seed"], p, 1, k0))
    return jobs


def oracle_throughput(w, inst, sweeps=2000, procs=None):
    """The CPU oracle, as it stands, on a bounded sample of the workload
    (oracle_sample_jobs), one spawned process per host core."""
    procs = procs or os.cpu_count() or 1
    jobs = oracle_sample_jobs(w, inst, procs, sweeps)
    wall, res = _oracle_pool(jobs, procs)
    if procs == 1:          # one core: the worker's own time, without the process start-up
        wall = res[0][0]
    ups = procs * sweeps * w["X"] * w["Y"]
    return {"value": ups / wall, "unit": "spin-updates/s", "cores": procs, "kind": "oracle", "updates": ups,
            "wall_s": wall,
            "sample": f"{procs} processes x 1 trial x {sweeps} sweeps of the {w['X']}x{w['Y']} workload, "
                      f"process p from sweep p*{w['sweeps']}/{procs} ({ups:.3g} updates)"}


def oracle_ttt(w, inst, seed, procs, trials=None, target=None, r_gpu=None):
    """Time-to-target of the oracle on the host cores (Eq. 3-5): `trials`
    whole trials (default: all of the workload's) of the full schedule with
    seed `seed`, split over `procs` spawned processes.  t_trial = wall /
    trials (throughput form).  Without a target the oracle's own best cut
    sets it; with one (from the GPU run of the same seed), the repetitions r
    come from the GPU's full distribution, which the oracle's trials
    reproduce bit for bit (their cuts are returned for that check)."""
    from paper_2505_18508_gb300 import stats
    trials = trials or w["trials"]
    procs = min(procs, trials)
    betas = synth.linear_betas(w["beta0"], w["beta1"], w["sweeps"])
    per = [trials // procs + (1 if p < trials % procs else 0) for p in range(procs)]
    jobs, t0 = [], 0
    for c in per:
        jobs.append((inst, betas, seed, t0, c, 0))
        t0 += c
    wall, res = _oracle_pool(jobs, procs)
    cuts = np.concatenate([c for _, c in res])
    if target is None:
        target = stats.target_cut(int(cuts.max()))
        Ps = stats.success_probability(cuts, target)
        r = stats.repetitions(Ps)
    else:
        r = r_gpu
    t_trial = wall / trials
    return {"trials": trials, "processes": procs, "wall_s": wall, "t_trial_s": t_trial, "target": int(target),
            "r": r, "TTT_s": t_trial * r if math.isfinite(r) else None}, cuts


# ------------------------------------------------------------------ helpers
def ttt_stats(cuts, t_step_s, trials, sweeps, quality=0.999):
    from paper_2505_18508_gb300 import stats  # Eq. 3-5
    best = int(cuts.max())
    target = stats.target_cut(best, quality)
    Ps = stats.success_probability(cuts, target)
    r = stats.repetitions(Ps)
    t_trial = t_step_s / trials
    return {"best_cut": best, "target": target, "P_s": Ps, "r": r, "STT_sweeps": sweeps * r,
            "TTT_s_throughput_form": t_trial * r,
            "TTT_s_latency_form": t_step_s * math.ceil(r / trials) if math.isfinite(r) else None,
            "cut_mean": float(cuts.mean()), "cut_min": int(cuts.min())}


def _round(v, nd=4):
    if isinstance(v, float):
        if not math.isfinite(v):
            return None
        return float(f"{v:.{nd}g}")
    if isinstance(v, dict):
        return {k: _round(x, nd) for k, x in v.items()}
    if isinstance(v, (list, tuple)):
        return [_round(x, nd) for x in v]
    return v


# ------------------------------------------------------------------ secondary legs
def draw16_leg(args, prob=None, inst=None):
    """The headline workload in the 16-bit draw mode (one Philox block per
    eight trials), 3 timed steps with an L2 flush between them."""
    import torch
    import paper_2505_18508_gb300 as ia
    w = dict(WORKLOAD)
    own = prob is None
    if own:
        inst = synth.torus_instance(w["X"], w["Y"], w["inst_seed"])
        prob = ia.Problem.from_instance(inst)
    T, S, n = w["trials"], w["sweeps"], inst["n"]
    betas = synth.linear_betas(w["beta0"], w["beta1"], S)
    spins = torch.empty((T, n), dtype=torch.int8, device="cuda")
    cuts = torch.empty((T,), dtype=torch.int32, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")
    prob.set_draw_bits(16)
    for i in range(2):
        ia.anneal(prob, T, betas, 3000 + i, out_spins=spins, out_cuts=cuts)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(3)]
    stream = torch.cuda.current_stream()
    for i, (e0, e1) in enumerate(ev):
        flush.zero_()
        e0.record(stream)
        ia.anneal(prob, T, betas, 3100 + i, out_spins=spins, out_cuts=cuts)
        e1.record(stream)
    torch.cuda.synchronize()
    prob.set_draw_bits(32)
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    ups = updates_per_step(w)
    peak = _imad_peak_tops()
    a16 = ups * (IMAD_OPS_PER_UPDATE / 2) / (ms / 1e3) / 1e12
    if own:
        prob.destroy()
    return {"workload": "the headline workload with 16-bit draws (the 16-bit decision stream)",
            "value": ups / (ms / 1e3), "unit": "spin-updates/s", "ms_per_step": ms,
            "roofline": {"bound": "alu", "achieved": a16, "peak": peak, "frac": a16 / peak,
                         "unit": "Tops/s (32-bit IMAD)", "ops_per_update": IMAD_OPS_PER_UPDATE / 2}}


def batched_leg(args):
    """The 96-instance uneven batch ({50,100,140,200}x100, 32-512 trials,
    2,000-20,000 sweeps, each sweep count times --scale) as one graph-replayed
    persistent launch."""
    import paper_2505_18508_gb300 as ia
    cfg = synth.batched_config()
    insts = [synth.torus_instance(c["X"], c["Y"], c["inst_seed"]) for c in cfg]
    probs = [ia.Problem.from_instance(i) for i in insts]
    trials = [c["trials"] for c in cfg]
    sweeps = [max(1, int(c["sweeps"] * args.scale)) for c in cfg]
    betas = [synth.linear_betas(0.1, 3.0, S) for S in sweeps]
    seeds = [c["seed"] for c in cfg]
    plan = ia.BatchPlan(probs, trials, sweeps, betas, seeds, group_trials=args.group_trials,
                        ctas_per_sm=args.ctas_per_sm)
    plan.launch()
    ms = _cuda_time(plan.launch, args.reps)
    ups = sum(t * s * i["n"] for t, s, i in zip(trials, sweeps, insts))
    plan.destroy()
    for p in probs:
        p.destroy()
    return {"workload": "96 tori {50,100,140,200}x100, 32-512 trials, 2,000-20,000 sweeps"
                        + (f" x {args.scale}" if args.scale != 1.0 else "") + ", one CUDA-graph replay",
            "updates": ups, "ms_per_replay": ms, "value": ups / (ms / 1e3), "unit": "spin-updates/s"}


GRAPHS = ("g22", "r20k", "torus")


def _graph_case(name):
    if name == "g22":
        return "random_2000v_19990e_w1", synth.random_graph(2000, 19990, 22, weights="one")
    if name == "r20k":
        return "random_20000v_40000e_pm1", synth.random_graph(20000, 40000, 81, weights="pm1")
    inst = synth.torus_instance(200, 100, 2)
    return "torus_200x100_as_graph", {"n": inst["n"], "row_ptr": inst["row_ptr"], "col": inst["col"],
                                      "J": inst["J"], "h": None}


def graph_leg(args):
    """General sparse graphs through the general-graph kernel (spins in
    shared memory, colour classes in order): a G22-like random graph (2,000
    vertices, 19,990 edges, w = +1), a random graph of the headline's size
    (20,000 vertices, 40,000 edges, w = +-1) and the headline torus given as a
    general graph."""
    import torch
    import paper_2505_18508_gb300 as ia
    out = {}
    betas = synth.linear_betas(0.1, 3.0, args.sweeps)
    for gname in ([args.graph] if args.graph != "all" else GRAPHS):
        name, g = _graph_case(gname)
        prob = ia.Problem.from_graph(g)
        prob.set_graph_threads_per_site(args.threads_per_site)
        prob.set_launch(strips=args.strips)
        cuts = torch.empty(args.trials, dtype=torch.int32, device="cuda")
        ia.anneal(prob, args.trials, betas, 1, want_spins=False, out_cuts=cuts)
        torch.cuda.synchronize()
        ms = _cuda_time(lambda: ia.anneal(prob, args.trials, betas, 2, want_spins=False, out_cuts=cuts), args.reps)
        info = prob.graph_info()
        ups = args.trials * args.sweeps * g["n"]
        out[name] = {"n": g["n"], "edges": int(len(g["col"]) // 2), "colours": info["colours"], "Dmax": info["Dmax"],
                     "trials": args.trials, "sweeps": args.sweeps, "ms": ms, "value": ups / (ms / 1e3),
                     "unit": "spin-updates/s", "best_cut": int(cuts.max().item()),
                     "mean_cut": float(cuts.double().mean().item())}
        prob.destroy()
    return out


def pt_leg(args, temps=8, chains=128):
    """Replica exchange on the headline instance at the headline's update
    budget (temps x chains = 1,024 slots, rounds x sweeps = 10,000 sweeps):
    throughput, and the coldest temperature's cuts."""
    import torch
    import paper_2505_18508_gb300 as ia
    inst = synth.torus_instance(200, 100, 2)
    prob = ia.Problem.from_instance(inst)
    betas = np.geomspace(0.5, 3.0, temps)
    ia.anneal_pt(prob, betas, chains, 2, args.sweeps_per_round, 1)
    torch.cuda.synchronize()
    res = {}

    def run():
        res["out"] = ia.anneal_pt(prob, betas, chains, args.rounds, args.sweeps_per_round, 1002)
    ms = _cuda_time(run)
    _, cuts, swaps = res["out"]
    cold = cuts[(temps - 1) * chains:].cpu().numpy()
    ups = temps * chains * args.rounds * args.sweeps_per_round * inst["n"]
    out = {"workload": f"200x100 torus, {temps} temperatures (geometric 0.5..3.0) x {chains} chains, "
                       f"{args.rounds} rounds x {args.sweeps_per_round} sweeps", "ms": ms, "value": ups / (ms / 1e3),
           "unit": "spin-updates/s", "swaps": int(swaps.item()), "kernel": prob.last_kernel(),
           "coldest": {"best_cut": int(cold.max()), "mean_cut": float(cold.mean())}}
    prob.destroy()
    return out


def trace_leg(args):
    """The headline workload read out along the trajectory (every trial's cut
    after every --trace-every sweeps, best-so-far cut and configuration)
    against the same anneal read out at the end only."""
    import paper_2505_18508_gb300 as ia
    w = WORKLOAD
    inst = synth.torus_instance(w["X"], w["Y"], w["inst_seed"])
    prob = ia.Problem.from_instance(inst)
    betas = synth.linear_betas(w["beta0"], w["beta1"], w["sweeps"])
    ups = updates_per_step(w)
    T = w["trials"]
    ia.anneal(prob, T, betas, 1)
    ia.anneal_trace(prob, T, betas, 1, args.trace_every)
    ms_plain = _cuda_time(lambda: ia.anneal(prob, T, betas, 1002), args.reps)
    ms_trace = _cuda_time(lambda: ia.anneal_trace(prob, T, betas, 1002, args.trace_every), args.reps)
    prob.destroy()
    return {"trace_every": args.trace_every, "ms_plain": ms_plain, "ms_trace": ms_trace,
            "value": ups / (ms_trace * 1e-3), "unit": "spin-updates/s", "overhead": ms_trace / ms_plain - 1.0}


def cnn_leg(args):
    """The learned stage's network on --batch seeded random configurations of
    an --X x --Y torus: one forward pass (logits), one gradient (forward,
    loss, input and weight gradients) and the tile proposals on those logits
    (10 x 10 tiles, exact dE <= 0 acceptance), through the C ABI.  Forward:
    2 * 9 * (3*32 + 32*32*2 + 32*1) useful flops and 389 algorithmic HBM bytes
    per site (spins in, three BF16 activation maps written and read, FP32
    logits out); proposals: 6 bytes per site."""
    import torch
    import paper_2505_18508_gb300 as ia
    X, Y, B = args.X, args.Y, args.batch
    prob = ia.Problem.from_instance(synth.torus_instance(X, Y, 3))
    net = ia.CNN(synth.cnn_init_params(1, scale=0.7))
    s = torch.from_numpy(synth.random_spins(B, X * Y, 5)).cuda()
    y = torch.from_numpy(synth.random_spins(B, X * Y, 6)).cuda().gt(0).to(torch.uint8)
    z = torch.empty((B, X * Y), dtype=torch.float32, device="cuda")

    def timed(fn, reps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        return _cuda_time(fn, reps)

    fwd_ms = timed(lambda: net.forward(prob, s, out=z), args.reps)
    grad_ms = timed(lambda: net.grad(prob, s, y), max(1, args.reps // 4))
    prop_ms = timed(lambda: ia.propose(prob, s, z, 10), args.reps)
    sites = B * X * Y
    fwd_gbs = CNN_BYTES_PER_SITE * sites / (fwd_ms * 1e-3) / 1e9
    out = {"workload": f"{B} x {X}x{Y} spin configurations", "forward_ms": fwd_ms,
           "forward_tflops": CNN_FLOP_PER_SITE * sites / (fwd_ms * 1e-3) / 1e12,
           "forward_gbs": fwd_gbs, "forward_hbm_frac": fwd_gbs / PEAK_HBM_GBS,
           "grad_ms": grad_ms, "grad_status": prob.get_status(), "propose_ms": prop_ms,
           "propose_gbs": PROPOSE_BYTES_PER_SITE * sites / (prop_ms * 1e-3) / 1e9}
    net.destroy()
    prob.destroy()
    return out


def campaign_leg(args):
    """Fig. 1 style ladder on the headline instance: --campaign-trials trials
    per budget, beta 0.1 -> 3.0 over S sweeps, one anneal per budget."""
    import paper_2505_18508_gb300 as ia
    from paper_2505_18508_gb300.campaign import run_campaign
    inst = synth.torus_instance(200, 100, 2)
    prob = ia.Problem.from_instance(inst)
    budgets = [int(float(b)) for b in args.budgets.split(",")]
    out = run_campaign(prob, budgets, args.campaign_trials, 4242)
    prob.destroy()
    out["workload"] = (f"Fig. 1 style ladder on the 200x100 instance (seed 2): {args.campaign_trials} trials per "
                       "budget, beta 0.1->3.0 over S sweeps, one anneal per budget")
    return out


def _train_droplet_net(X, Y, seeds, trials, S_train, steps, init_seed=3):
    """The network trained on droplet targets: `trials` plain anneals of each
    held-out instance (seeds), targets = the improving components of each
    final state's disagreement with the instance's best state."""
    import torch
    import paper_2505_18508_gb300 as ia
    from paper_2505_18508_gb300 import learned
    t0 = time.perf_counter()
    probs = [ia.Problem.from_instance(synth.torus_instance(X, Y, sd)) for sd in seeds]
    data = learned.droplet_dataset(probs, trials, synth.linear_betas(0.1, 3.0, S_train))
    pos = float(np.mean([float(y.float().mean().item()) for _, _, y, _ in data]))
    net = ia.CNN(synth.cnn_init_params(init_seed, scale=0.7))
    losses = learned.train(net, data, steps, batch=16, lr=2e-3, log_every=max(1, steps // 4))
    torch.cuda.synchronize()
    for p in probs:
        p.destroy()
    p_hat = min(max(pos, 1e-9), 1 - 1e-9)
    return net, {"instances": len(seeds), "trials": trials, "sweeps": S_train, "steps": steps,
                 "target_positive_fraction": pos, "loss": losses,
                 "base_rate_entropy": -(p_hat * math.log(p_hat) + (1 - p_hat) * math.log(1 - p_hat)),
                 "seconds": time.perf_counter() - t0}


# The proposal schedule of the learned plans: network block flips and partner
# moves after every PROPOSAL_EVERY-sweep chunk of the second half of the
# schedule (the last PROPOSAL_WINDOW x S sweeps), chunk j's partner at offset
# 1 + j mod PARTNER_PERIOD.  Chosen on 8 config-5 instances (seeds 30000-30007)
# among windows of 1,000 / 3,000 / 0.3 S / 0.5 S / S sweeps, chunks of 25-200
# sweeps and offset cycles of 3-255: it reaches 99.9 % of the best cut with
# every trial from 3,000 sweeps on, against a median time-to-target 20 times
# longer for the last 1,000 sweeps in 100-sweep chunks with 7 offsets.
PROPOSAL_EVERY, PROPOSAL_WINDOW, PARTNER_PERIOD = 50, 0.5, 31


def _run_forms(X, Y, eval_seeds, seed0, T, budgets, forms, warm=False):
    """Every form on every evaluation instance and budget, 8 instances per
    launch (one CUDA graph per form and budget).  forms: name -> (net or
    None, partner period) or None for the plain annealer.  Returns
    {(S, instance seed): {form: (cuts, wall ms per instance, accepted)}}."""
    import torch
    import paper_2505_18508_gb300 as ia
    res = {}
    for g0 in range(0, len(eval_seeds), 8):
        group = eval_seeds[g0:g0 + 8]
        probs = [ia.Problem.from_instance(synth.torus_instance(X, Y, sd)) for sd in group]
        seeds = [seed0 + sd for sd in group]
        m = len(group)
        for S in budgets:
            betas = synth.linear_betas(0.1, 3.0, S)
            kf = max(0, S - int(round(PROPOSAL_WINDOW * S)))
            for name, spec in forms.items():
                if spec is None:
                    plan = ia.BatchPlan(probs, [T] * m, [S] * m, [betas] * m, seeds, want_spins=False)
                else:
                    net, period = spec
                    plan = ia.LearnedPlan(probs, net, T, betas, seeds, k_first=kf, every=PROPOSAL_EVERY, partner_period=period,
                                          warm=warm and net is not None)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                out = plan.launch()
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                if spec is None:
                    cuts, acc = torch.cat(out[1]).cpu().numpy().reshape(m, T), None
                else:
                    cuts = out[1].cpu().numpy().reshape(m, T)
                    acc = out[2].double().reshape(m, T).mean(dim=1).cpu().numpy()
                for q, sd in enumerate(group):
                    res.setdefault((S, sd), {})[name] = (cuts[q], ms / m, None if acc is None else float(acc[q]))
                plan.destroy()
        for p in probs:
            p.destroy()
    return res


def _form_stats(res, names, T):
    """Per instance: target = ceil(0.999 best) over the forms `names` and every
    budget (Eq. 3-5 with the paper's 99.9 % style); per form and budget the
    mean and standard error over instances of P_s, and per instance the
    form's best time-to-target over the budgets (TTT = wall per trial x r)."""
    from paper_2505_18508_gb300 import stats
    budgets = sorted({S for S, _ in res})
    insts = sorted({sd for _, sd in res})
    ps = {(f, S): [] for f in names for S in budgets}
    ttt = {f: [] for f in names}
    for sd in insts:
        best = max(int(res[(S, sd)][f][0].max()) for S in budgets for f in names)
        tgt = stats.target_cut(best)
        best_t = {f: math.inf for f in names}
        for S in budgets:
            for f in names:
                cuts, ms, _ = res[(S, sd)][f]
                P = stats.success_probability(cuts, tgt)
                ps[(f, S)].append(P)
                r = stats.repetitions(P)
                if math.isfinite(r):
                    best_t[f] = min(best_t[f], ms / 1e3 / T * r)
        for f in names:
            ttt[f].append(best_t[f])
    k = len(insts)
    out = {"P_s": {f"{f}@{S}": [float(np.mean(v)), float(np.std(v, ddof=1) / math.sqrt(k)) if k > 1 else 0.0]
                   for (f, S), v in ps.items()}}
    out["TTT_s"] = {}
    for f, v in ttt.items():
        fin = [x for x in v if math.isfinite(x)]
        out["TTT_s"][f] = {"median": float(np.median(v)) if len(fin) * 2 > k else None, "reached": len(fin),
                           "mean_reached": float(np.mean(fin)) if fin else None,
                           "se_reached": float(np.std(fin, ddof=1) / math.sqrt(len(fin))) if len(fin) > 1 else None}
    return out


def _cut_stats(res, names):
    budgets = sorted({S for S, _ in res})
    return {f"{f}@{S}": {"mean_cut": float(np.mean([res[k][f][0].mean() for k in res if k[0] == S])),
                         "best_cut_mean": float(np.mean([res[k][f][0].max() for k in res if k[0] == S])),
                         "wall_ms_per_instance": float(np.mean([res[k][f][1] for k in res if k[0] == S])),
                         "accepted_per_trial": (float(np.mean([res[k][f][2] for k in res if k[0] == S]))
                                                if res[next(iter(res))][f][2] is not None else None)}
            for f in names for S in budgets}


def learned_leg(args):
    """Config 5 of the workload set: 200x100 tori, 16 evaluation instances
    (seeds 30000-30015) x 512 trials, beta 0.1 -> 3.0 over S sweeps on a
    budget ladder; the network trained on droplet targets of 20,000-spin
    instances (seeds 40000-40255).  Forms, each one CUDA graph over 8
    instances: the plain annealer; the network's cluster block flips after
    every PROPOSAL_EVERY-sweep chunk of the second half of the schedule
    (trained, and untrained for what training adds); partner moves in the
    same chunks; both.
    Statistics per instance against 99.9 % of the best cut any form found."""
    X, Y, T = 200, 100, 512
    net, train = _train_droplet_net(X, Y, list(range(40000, 40000 + args.learned_train)), 16, 10000, 800)
    import paper_2505_18508_gb300 as ia
    untrained = ia.CNN(synth.cnn_init_params(3, scale=0.7))
    budgets = [int(b) for b in args.learned_budgets.split(",")]
    forms = {"plain": None, "learned": (net, 0), "untrained": (untrained, 0), "partner": (None, PARTNER_PERIOD),
             "learned_partner": (net, PARTNER_PERIOD)}
    res = _run_forms(X, Y, list(range(30000, 30000 + args.learned_seeds)), 40000, T, budgets, forms)
    net.destroy()
    untrained.destroy()
    names = list(forms)
    all_forms = _form_stats(res, names, T)
    net_only = _form_stats(res, ["plain", "learned", "untrained"], T)
    top = str(max(budgets))
    return {"summary": {"P_s@" + top: {f: all_forms["P_s"][f"{f}@{top}"] for f in names},
                        "median_TTT_s": {f: all_forms["TTT_s"][f]["median"] for f in names},
                        "TTT_reached": {f: all_forms["TTT_s"][f]["reached"] for f in names},
                        "network_only_P_s@" + top: {f: net_only["P_s"][f"{f}@{top}"]
                                                    for f in ("plain", "learned", "untrained")},
                        "instances": len({sd for _, sd in res})},
            "workload": f"200x100 tori, instance seeds 30000-{30000 + args.learned_seeds - 1}, 512 trials each, "
                        f"beta 0.1->3.0 over S sweeps, S in {budgets}; proposals after every {PROPOSAL_EVERY}-sweep "
                        f"chunk of the last {PROPOSAL_WINDOW} S sweeps, partner offsets 1..{PARTNER_PERIOD}; each "
                        "form one CUDA graph over 8 instances (wall time shared by 8 x 512 trials)",
            "train": train, "targets_all_forms": all_forms, "targets_plain_and_network": net_only,
            "cuts": _cut_stats(res, names)}


def partner_leg(args):
    """The cost of the partner moves inside the plan: 8 tori 200x100 x 512
    trials, beta 0.1 -> 3.0 over --leg-sweeps sweeps, the plain annealer
    (one batched graph) against the same with partner moves on the learned
    legs' schedule (one learned-plan graph), each replayed --reps times after
    one warm-up replay (CUDA events)."""
    import torch
    import paper_2505_18508_gb300 as ia
    X, Y, T, S = 200, 100, 512, args.leg_sweeps
    probs = [ia.Problem.from_instance(synth.torus_instance(X, Y, 30000 + q)) for q in range(8)]
    seeds = [70000 + q for q in range(8)]
    betas = synth.linear_betas(0.1, 3.0, S)
    plans = {"plain": ia.BatchPlan(probs, [T] * 8, [S] * 8, [betas] * 8, seeds, want_spins=False),
             "partner": ia.LearnedPlan(probs, None, T, betas, seeds, k_first=max(0, S - int(round(PROPOSAL_WINDOW * S))),
                                       every=PROPOSAL_EVERY, partner_period=PARTNER_PERIOD)}
    out = {"workload": f"8 tori 200x100, 512 trials, {S} sweeps; partner moves after every {PROPOSAL_EVERY}-sweep "
                       f"chunk of the last {PROPOSAL_WINDOW} S sweeps, offsets 1..{PARTNER_PERIOD}"}
    for name, plan in plans.items():
        plan.launch()
        torch.cuda.synchronize()
        ms = _cuda_time(plan.launch, args.reps)
        res = plan.launch()
        torch.cuda.synchronize()
        cuts = torch.cat(res[1]) if name == "plain" else res[1]
        out[name] = {"ms_per_replay": ms, "mean_cut": float(cuts.double().mean().item()),
                     "best_cut_mean": float(cuts.reshape(8, T).max(dim=1).values.double().mean().item())}
        if name == "partner":
            out[name]["components_per_trial"] = float(res[2].double().mean().item())
        plan.destroy()
    out["overhead"] = out["partner"]["ms_per_replay"] / out["plain"]["ms_per_replay"] - 1.0
    for p in probs:
        p.destroy()
    return out


def learned100_leg(args):
    """Config 4 of the workload set: 100x100 tori, 8 evaluation instances
    (seeds 20000-20007) x 512 trials; the network trained on droplet targets
    of 256 held-out instances (seeds 10000-10255); the learned form with a
    warm start (the network's whole-lattice proposal on the start state) and
    cluster block flips on the learned legs' schedule, against the plain
    annealer and partner moves."""
    X, Y, T = 100, 100, 512
    net, train = _train_droplet_net(X, Y, list(range(10000, 10256)), 8, 3000, 600, init_seed=5)
    budgets = [1000, 3000, 10000]
    forms = {"plain": None, "learned": (net, 0), "partner": (None, PARTNER_PERIOD),
             "learned_partner": (net, PARTNER_PERIOD)}
    res = _run_forms(X, Y, list(range(20000, 20008)), 20000, T, budgets, forms, warm=True)
    net.destroy()
    names = list(forms)
    st = _form_stats(res, names, T)
    return {"summary": {"P_s@10000": {f: st["P_s"][f"{f}@10000"] for f in names},
                        "median_TTT_s": {f: st["TTT_s"][f]["median"] for f in names},
                        "TTT_reached": {f: st["TTT_s"][f]["reached"] for f in names}},
            "workload": "100x100 tori, instance seeds 20000-20007, 512 trials each, beta 0.1->3.0 over S sweeps, "
                        f"S in {budgets}; warm start plus cluster block flips after every {PROPOSAL_EVERY}-sweep "
                        f"chunk of the last {PROPOSAL_WINDOW} S sweeps, partner offsets 1..{PARTNER_PERIOD}",
            "train": train, "stats": st, "cuts": _cut_stats(res, names)}


LEGS = {"draw16": draw16_leg, "batched": batched_leg, "graph": graph_leg, "pt": pt_leg, "trace": trace_leg,
        "cnn": cnn_leg, "campaign": campaign_leg, "learned": learned_leg, "learned100": learned100_leg,
        "partner": partner_leg}
# legs the default run adds after the headline's timed region
DEFAULT_LEGS = ("draw16", "batched", "graph", "pt", "campaign", "learned", "learned100")


def leg_summary(name, d):
    """One or two numbers per leg for the headline line."""
    if d is None:
        return None
    if "error" in d:
        return {"error": d["error"][:200]}
    if name == "draw16":
        return {"value": d["value"], "frac": d["roofline"]["frac"]}
    if name in ("batched", "trace"):
        return {"value": d["value"]}
    if name == "partner":
        return {"overhead": d["overhead"]}
    if name == "pt":
        return {"value": d["value"], "coldest_best_cut": d["coldest"]["best_cut"]}
    if name == "graph":
        return {k: v["value"] for k, v in d.items()}
    if name == "campaign":
        return {"sweeps": [b["sweeps"] for b in d["budgets"]], "highest": [b["highest"] for b in d["budgets"]]}
    if name in ("learned", "learned100"):
        return d.get("summary")
    if name == "cnn":
        return {"forward_ms": d["forward_ms"], "forward_hbm_frac": d["forward_hbm_frac"]}
    return None


def headline_line(base, legs):
    """The last stdout line: the contract's keys, with every number rounded,
    and a one-number summary per leg.  Leg summaries are dropped, largest
    first, while the line is longer than HEADLINE_MAX_BYTES; a line whose
    contract keys alone are too long raises, as does a missing key."""
    line = {k: base[k] for k in HEADLINE_KEYS}
    for k in ("ttt_99_9",):
        if k in base:
            line[k] = base[k]
    line["legs"] = {name: leg_summary(name, d) for name, d in legs.items()}
    line = _round(line)
    text = json.dumps(line, separators=(",", ":"))
    while len(text) > HEADLINE_MAX_BYTES and any(v is not None and v != "on its own line"
                                                 for v in line["legs"].values()):
        big = max((k for k, v in line["legs"].items() if v is not None and v != "on its own line"),
                  key=lambda k: len(json.dumps(line["legs"][k])))
        line["legs"][big] = "on its own line"
        text = json.dumps(line, separators=(",", ":"))
    if len(text) > HEADLINE_MAX_BYTES:
        raise ValueError(f"headline line is {len(text)} bytes (limit {HEADLINE_MAX_BYTES})")
    return text


def dist_env():
    from paper_2505_18508_gb300 import replicas
    return replicas.env()


def _imad_peak_tops(sms=None):
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    if sms is None:
        import torch
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    clk_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    return sms * IMAD_LANES_PER_SM * clk_mhz * 1e6 / 1e12


# ------------------------------------------------------------------ reference arm
def reference_arm(args):
    """The oracle as it stands on the host cores: each step is the bounded,
    stratified sample of the headline workload that oracle_sample_jobs
    describes; the line states that sample and its own updates per step."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    w = dict(WORKLOAD)
    inst = synth.torus_instance(w["X"], w["Y"], w["inst_seed"])
    sweeps = 1000
    for _ in range(args.warmup):
        oracle_throughput(w, inst, sweeps=sweeps)
    vals = [oracle_throughput(w, inst, sweeps=sweeps) for _ in range(args.steps)]
    wall = float(np.mean([x["wall_s"] for x in vals]))
    step_ups = vals[-1]["updates"]
    v = step_ups / wall
    cb = {k: vals[-1][k] for k in ("unit", "cores", "kind", "sample")}
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "spin-updates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, **w, "updates_per_step": step_ups,
                       "sample": vals[-1]["sample"],
                       "note": "each step is the stated sample of the workload, not all of its 2.048e11 updates"},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": "spin-updates/s", "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(_round(line, 6)), flush=True)
    return 0


# ------------------------------------------------------------------ main arm
def _parser():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--sweeps", type=int, default=None, help="override (profiling runs only)")
    ap.add_argument("--trials", type=int, default=None, help="override (profiling runs only)")
    ap.add_argument("--launch", default=None, help="G,C,threads launch shape (default: automatic)")
    ap.add_argument("--legs", default=",".join(DEFAULT_LEGS), help="secondary legs after the headline ('' = none)")
    ap.add_argument("--leg", default=None, choices=sorted(LEGS), help="run one secondary leg alone and exit")
    # leg options
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--scale", type=float, default=1.0, help="batched: sweep counts x scale")
    ap.add_argument("--group-trials", type=int, default=0)
    ap.add_argument("--ctas-per-sm", type=int, default=0)
    ap.add_argument("--rounds", type=int, default=200)
    ap.add_argument("--sweeps-per-round", type=int, default=50)
    ap.add_argument("--graph", default="all", choices=("all",) + GRAPHS)
    ap.add_argument("--leg-trials", dest="leg_trials", type=int, default=1024)
    ap.add_argument("--leg-sweeps", dest="leg_sweeps", type=int, default=2000)
    ap.add_argument("--trace-every", type=int, default=100)
    ap.add_argument("--threads-per-site", type=int, default=0, help="general graphs: 1, 4, 8 or 0 (automatic)")
    ap.add_argument("--strips", type=int, default=0, help="general graphs: CTAs per trial group (1-8; 0: automatic)")
    ap.add_argument("--X", type=int, default=100)
    ap.add_argument("--Y", type=int, default=100)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--budgets", default="1000,3000,10000,30000,100000,300000")
    ap.add_argument("--campaign-trials", type=int, default=512)
    ap.add_argument("--learned-seeds", type=int, default=16)
    ap.add_argument("--learned-train", type=int, default=256)
    ap.add_argument("--learned-budgets", default="3000,10000,30000")
    return ap


def run_leg(name, args):
    a = argparse.Namespace(**vars(args))
    a.trials, a.sweeps = args.leg_trials, args.leg_sweeps
    return LEGS[name](a)


def main(argv=None):
    args = _parser().parse_args(argv)
    if args.impl == "reference":
        return reference_arm(args)

    import torch
    import paper_2505_18508_gb300 as ia
    from paper_2505_18508_gb300 import build as lib_build
    from paper_2505_18508_gb300 import replicas

    ws, rank, local = dist_env()
    lib_build.build()
    torch.cuda.set_device(local)
    if args.leg:
        print(json.dumps({"leg": args.leg, **run_leg(args.leg, args)}), flush=True)
        return 0
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    w = dict(WORKLOAD)
    if args.sweeps:
        w["sweeps"] = args.sweeps
    if args.trials:
        w["trials"] = args.trials
    inst = synth.torus_instance(w["X"], w["Y"], w["inst_seed"])
    betas = synth.linear_betas(w["beta0"], w["beta1"], w["sweeps"])
    T, S, n = w["trials"], w["sweeps"], inst["n"]
    ups = updates_per_step(w)
    prob = ia.Problem.from_instance(inst)
    if args.launch:
        prob.set_launch(*[int(v) for v in args.launch.split(",")])
    dev = torch.device("cuda", local)
    spins = torch.empty((T, n), dtype=torch.int8, device=dev)
    cuts = torch.empty((T,), dtype=torch.int32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)  # > L2 (129 MB)
    stream = torch.cuda.current_stream()

    def seed_of(step):
        return replicas.rank_seed(w["seed"], rank, step)

    for i in range(args.warmup):
        ia.anneal(prob, T, betas, seed_of(-1 - i), out_spins=spins, out_cuts=cuts)
    torch.cuda.synchronize()
    shape = prob.last_launch()
    kernel = {1: "anneal_strip_kernel", 2: "anneal_flow_kernel"}.get(prob.last_kernel(), "?")

    clocks = ClockSampler(local)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    first_cuts = None
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()                       # L2 flush between timed steps (not inside the events)
        starts[i].record(stream)
        ia.anneal(prob, T, betas, seed_of(i), out_spins=spins, out_cuts=cuts)
        ends[i].record(stream)
        if i == 0:
            first_cuts = cuts.clone()
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms = replicas.max_over_ranks(float(np.mean(step_ms)), dist, dev)
    value = replicas.job_value(ws, ups, ms / 1e3)

    # ---- end to end through the C ABI with host buffers: instance upload
    # (ising_create from the host CSR), host betas, device->host copy of all
    # spins and cuts into pinned memory, every step
    h_spins = torch.empty((T, n), dtype=torch.int8, pin_memory=True)
    h_cuts = torch.empty((T,), dtype=torch.int32, pin_memory=True)
    torch.cuda.synchronize()
    e2e_ms = []
    for i in range(args.e2e_steps):
        t0 = time.perf_counter()
        p2 = ia.Problem.from_instance(inst)
        ia.anneal(p2, T, betas, seed_of(100 + i), out_spins=spins, out_cuts=cuts)
        h_spins.copy_(spins, non_blocking=True)
        h_cuts.copy_(cuts, non_blocking=True)
        torch.cuda.synchronize()
        p2.destroy()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_step_ms = float(np.mean(e2e_ms)) if e2e_ms else float("nan")
    h2d = 2 * n + 8 * S                      # packed instance flags + threshold table
    d2h = T * n + 4 * T

    # ---- roofline: integer-multiply pipe (Philox multiplies per update vs IMAD lanes)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_tops = _imad_peak_tops(sms)
    achieved_tops = ups * IMAD_OPS_PER_UPDATE / (ms / 1e3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved_tops, "peak": peak_tops, "unit": "Tops/s (32-bit IMAD)",
                "frac": achieved_tops / peak_tops,
                "traffic": FLOW_TRAFFIC_BYTES if kernel == "anneal_flow_kernel" and (T, S, n) == (1024, 10000, 20000)
                else None,
                "kernel": kernel,
                "peak_source": f"{sms} SMs x {IMAD_LANES_PER_SM} IMAD lanes x sm_max_mhz (measured peaks file)"}

    stats = None
    if args.steps > 0:   # over every rank's trials: the job ran ws * T trials in one step time
        all_cuts = replicas.gather_cuts(first_cuts, dist)
        stats = ttt_stats(all_cuts.cpu().numpy(), ms / 1e3, ws * T, S)

    # ---- the CPU oracle on the host cores (rank 0 of a 1-GPU run only)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        cpu = oracle_throughput(w, inst)
        one = oracle_throughput(w, inst, sweeps=1000, procs=1)
        cpu["single_core"] = {"value": one["value"], "sample": one["sample"]}
        cpu.pop("wall_s")
        cpu.pop("updates")
        ttt = {}
        if stats is not None and (T, S) == (1024, 10000):
            # the headline's step-0 trials 0 .. cores-1 on the oracle: their
            # cuts equal the GPU's bit for bit, and r is the GPU's
            o, oc = oracle_ttt(w, inst, seed_of(0), cores, trials=cores, target=stats["target"], r_gpu=stats["r"])
            o["parity_trials_equal"] = bool(np.array_equal(oc, first_cuts[:cores].cpu().numpy()))
            o["gpu_TTT_s"] = stats["TTT_s_throughput_form"]
            ttt["200x100"] = o
        # the 50x50 workload: all 64 trials on the oracle and on the GPU
        inst1 = synth.torus_instance(SMALL["X"], SMALL["Y"], SMALL["inst_seed"])
        o1, oc1 = oracle_ttt(SMALL, inst1, SMALL["seed"], cores)
        p1 = ia.Problem.from_instance(inst1)
        b1 = synth.linear_betas(SMALL["beta0"], SMALL["beta1"], SMALL["sweeps"])
        ia.anneal(p1, SMALL["trials"], b1, SMALL["seed"])
        res = {}
        g_ms = _cuda_time(lambda: res.setdefault("c", ia.anneal(p1, SMALL["trials"], b1, SMALL["seed"])[1]))
        p1.destroy()
        o1["parity_trials_equal"] = bool(np.array_equal(oc1, res["c"].cpu().numpy()))
        o1["gpu_t_trial_s"] = g_ms / 1e3 / SMALL["trials"]
        o1["gpu_TTT_s"] = o1["gpu_t_trial_s"] * o1["r"] if math.isfinite(o1["r"]) else None
        ttt["50x50"] = o1
        cpu["ttt_99_9"] = ttt

    # ---- secondary legs, each printed on its own line before the headline
    legs = {}
    if rank == 0 and not args.sweeps and not args.trials:
        for name in [x for x in args.legs.split(",") if x]:
            try:
                d = run_leg(name, args) if name != "draw16" else draw16_leg(args, prob, inst)
            except Exception as ex:        # a failed leg is reported, the headline still prints
                d = {"error": f"{type(ex).__name__}: {ex}"}
            legs[name] = d
            print(json.dumps({"leg": name, **_round(d, 6)}), flush=True)

    if rank == 0:
        base = {
            "metric": METRIC, "value": value, "unit": "spin-updates/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, **w, "updates_per_step": ups,
                       "l2": "flushed between steps (256 MB write)", "launch": shape},
            "e2e": {"value": ws * ups / (e2e_step_ms / 1e3), "unit": "spin-updates/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_step_ms},
            "gpu_launches": args.steps,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "clocks": clk,
            "ttt_99_9": stats,
        }
        print(headline_line(base, legs), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    prob.destroy()
    return 0


if __name__ == "__main__":
    sys.exit(main())

"""Benchmark: spin-updates/s and time-to-99.9%-cut of the plain GPU annealer.

Workload (one "step"): the 200x100 toroidal +-1 instance (20,000 spins,
instance seed 2), 1,024 trials x 10,000 Metropolis sweeps, beta linear
0.1 -> 3.0, Philox seed 1002 + step; spins and exact cuts of every trial are
produced on the device.  A step is T*S*n = 2.048e11 spin updates.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun): every rank runs the full workload with its own seeds
(independent trials, weak scaling), no collective on the data path.

Prints one JSON line (rank 0).
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
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
PEAK_HBM_GBS = float(json.load(open(PEAKS_FILE)).get("hbm_gbs", 6800.0)) if os.path.exists(PEAKS_FILE) else 6800.0
# Integer multiply lanes per SM per clock (32-bit IMAD; a 32x32->64 multiply
# counts as two) on this part: 4 sub-partitions x 16 lanes.
IMAD_LANES_PER_SM = 64
# Philox4x32-10 multiplies per spin update: 10 rounds x 2 products x 2 halves / 4 draws
IMAD_OPS_PER_UPDATE = 10
# DRAM bytes (read + write) of one launch of the persistent annealing kernel
# on this workload, from an ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum, --clock-control none) of the same launch
# configuration: 427,008 + 360,704 bytes
FLOW_TRAFFIC_BYTES = 427008 + 360704


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


CNN_FLOP_PER_SITE = 2 * 9 * (3 * 32 + 32 * 32 * 2 + 32 * 1)
CNN_BYTES_PER_SITE = 1 + 3 * 2 * 64 + 4   # spins in, three BF16 maps written and read, FP32 logits out


# ------------------------------------------------------------------ CPU oracle
def _oracle_slice(args):
    import oracle  # test infrastructure: the CPU baseline leg only
    inst, betas, seed, t_begin, t_count = args
    t = time.perf_counter()
    oracle.anneal(inst, betas, seed, t_begin=t_begin, t_count=t_count)
    return time.perf_counter() - t


def oracle_throughput(w, inst, sweeps=3000, trials_per_proc=1, procs=None):
    """The CPU oracle, as it stands, on a bounded sample of the workload:
    `procs` processes (default: every host core), each running
    `trials_per_proc` trials of the first `sweeps` sweeps of the schedule."""
    import multiprocessing as mp
    import oracle
    oracle.lib()  # build before forking workers
    procs = procs or os.cpu_count() or 1
    betas = synth.linear_betas(w["beta0"], w["beta1"], w["sweeps"])[:sweeps]
    jobs = [(inst, betas, w["seed"], p * trials_per_proc, trials_per_proc) for p in range(procs)]
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(procs) as pool:
        times = pool.map(_oracle_slice, jobs)
    wall = time.perf_counter() - t0
    if procs == 1:          # one core: the worker's own time, without the process start-up
        wall = times[0]
    ups = procs * trials_per_proc * sweeps * w["X"] * w["Y"]
    return {"value": ups / wall, "unit": "spin-updates/s", "cores": procs, "kind": "oracle",
            "sample": f"{procs} processes x {trials_per_proc} trial(s) x first {sweeps} sweeps of the "
                      f"{w['X']}x{w['Y']} workload ({ups:.3g} updates, {wall:.1f} s wall)"}


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


def learned_leg(budgets=(1000, 3000, 10000, 30000), every=100, tile=10, n_train=256, train_sweeps=1000,
                steps=800, end_window=500):
    """Config 5 of the workload set: 200x100 tori, 8 seeds x 512 trials, the
    plain annealer against the learned form (network trained on 20,000-spin
    snapshots of the plain annealer on held-out seeds), on the sweep-budget
    ladder.  Per seed: best = the highest cut either form found at any budget,
    target = ceil(0.999 best); per (form, budget): P_s, r and
    TTT = (batch wall time / trials) * r (Eq. 3, 5)."""
    import torch
    import paper_2505_18508_gb300 as ia
    from paper_2505_18508_gb300 import learned, stats
    t0 = time.perf_counter()
    tb = synth.linear_betas(0.1, 3.0, train_sweeps)
    train = [synth.torus_instance(200, 100, 40000 + k) for k in range(n_train)]
    data = learned.make_dataset(train, tb, every, snap_trials=4, target="future")
    net = ia.CNN(synth.cnn_init_params(3, scale=0.7))
    losses = learned.train(net, data, steps, batch=16, lr=2e-3, log_every=steps // 4)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    for d in data:
        d[0].destroy()
    T = 512
    # the network's forward pass on this workload (one proposal round's logits)
    prob = ia.Problem.from_instance(synth.torus_instance(200, 100, 30000))
    s0 = torch.from_numpy(synth.random_spins(T, prob.n, 1)).cuda()
    z = torch.empty((T, prob.n), dtype=torch.float32, device="cuda")
    for _ in range(3):
        net.forward(prob, s0, out=z)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        net.forward(prob, s0, out=z)
    e1.record()
    torch.cuda.synchronize()
    fwd_ms = e0.elapsed_time(e1) / 10
    sites = T * prob.n
    fwd_gbs = CNN_BYTES_PER_SITE * sites / (fwd_ms * 1e-3) / 1e9
    cnn = {"forward_ms": fwd_ms, "sites": sites,
           "useful_tflops": CNN_FLOP_PER_SITE * sites / (fwd_ms * 1e-3) / 1e12,
           "algorithmic_gbs": fwd_gbs, "hbm_frac": fwd_gbs / PEAK_HBM_GBS,
           "note": "forward = 4 tcgen05 convolution launches; 389 algorithmic HBM bytes per site; "
                   "hbm_frac of measured copy bandwidth"}
    prob.destroy()
    # forms, instance by instance: the plain annealer; the learned form with
    # proposals every `every` sweeps over the whole schedule (config 5 as
    # stated); and the same with proposals only in the last `end_window`
    # sweeps, where the annealer has cooled and only coordinated block flips
    # can still lower the energy.  Batched forms, all 8 instances at once: the
    # plain annealer in one persistent launch, and learned_end with the sweeps
    # before its window in one persistent launch.  A batched form's results
    # equal its per-instance form's (checked below); only the wall time, shared
    # by the 8 x T trials, differs.
    forms = ("plain", "learned", "learned_end")
    bforms = {"plain_batched": "plain", "learned_end_batched": "learned_end"}
    probs = [ia.Problem.from_instance(synth.torus_instance(200, 100, 30000 + q)) for q in range(8)]
    seeds = [70000 + q for q in range(8)]
    runs = [{S: {} for S in budgets} for _ in probs]
    batched_same = True
    for S in budgets:
        betas = synth.linear_betas(0.1, 3.0, S)
        end_start = max(0, S - end_window)
        for q, (prob, seed) in enumerate(zip(probs, seeds)):
            for name in forms:
                st = {}
                torch.cuda.synchronize(); a = time.perf_counter()
                if name == "plain":
                    _, c = ia.anneal(prob, T, betas, seed)
                else:
                    start = 0 if name == "learned" else end_start
                    _, c = learned.anneal_learned(prob, net, T, betas, seed, every=every, tile=tile, stats=st,
                                                  start=start)
                torch.cuda.synchronize(); b = time.perf_counter()
                runs[q][S][name] = (c.cpu().numpy(), b - a, st.get("accepted_per_trial"))
        for name, base in bforms.items():
            torch.cuda.synchronize(); a = time.perf_counter()
            if name == "plain_batched":
                _, cs = ia.anneal_batched(probs, [T] * 8, [S] * 8, [betas] * 8, seeds)
            else:
                _, cs = learned.anneal_learned_batched(probs, net, T, betas, seeds, every=every, tile=tile,
                                                       start=end_start)
            torch.cuda.synchronize(); b = time.perf_counter()
            for q in range(8):
                c = cs[q].cpu().numpy()
                batched_same = batched_same and bool(np.array_equal(c, runs[q][S][base][0]))
                runs[q][S][name] = (c, (b - a) / 8, None)   # the batch's wall time per instance
    rows = []
    allforms = forms + tuple(bforms)
    for q in range(8):
        best = int(max(max(v[f][0].max() for f in forms) for v in runs[q].values()))
        tgt = stats.target_cut(best)
        row = {"seed": 30000 + q, "best": best, "target": tgt}
        for S in budgets:
            for name in allforms:
                cuts, wall, acc = runs[q][S][name]
                Ps = stats.success_probability(cuts, tgt)
                r = stats.repetitions(Ps)
                e = {"P_s": Ps, "mean_cut": float(cuts.mean()), "wall_s": wall,
                     "TTT_s": (wall / T) * r if math.isfinite(r) else None}
                if acc is not None:
                    e["accepted_per_trial"] = acc
                row[f"{name}@{S}"] = e
        rows.append(row)
    for prob in probs:
        prob.destroy()
    net.destroy()

    def med(key):
        v = [r[key]["TTT_s"] for r in rows if r[key]["TTT_s"] is not None]
        return float(np.median(v)) if len(v) == len(rows) else None
    ladder = {f"{name}@{S}": {"median_TTT_s": med(f"{name}@{S}"),
                              "reached": sum(r[f"{name}@{S}"]["TTT_s"] is not None for r in rows),
                              "mean_P_s": float(np.mean([r[f"{name}@{S}"]["P_s"] for r in rows]))}
              for S in budgets for name in allforms}

    def best_budget(prefix):
        c = [(v["median_TTT_s"], k) for k, v in ladder.items() if k.startswith(prefix) and v["median_TTT_s"]]
        return min(c) if c else (None, None)
    bp, bl, be = best_budget("plain@"), best_budget("learned@"), best_budget("learned_end@")
    bpb, beb = best_budget("plain_batched@"), best_budget("learned_end_batched@")
    return {"workload": "200x100 tori, seeds 30000-30007, 512 trials each, beta 0.1->3.0 over S sweeps, "
                        f"S in {list(budgets)}; proposals every {every} sweeps, tiles {tile}x{tile} "
                        f"(learned: whole schedule; learned_end: last {end_window} sweeps); *_batched: the 8 "
                        "instances in one persistent launch (learned_end_batched: up to its window), wall time "
                        "shared by all 8 x 512 trials",
            "batched_results_equal_per_instance": batched_same,
            "train": {"instances": n_train, "snapshot_sweeps": train_sweeps, "steps": steps, "loss": losses,
                      "seconds": t_train},
            "cnn_forward": cnn,
            "ladder": ladder,
            "best_median_TTT_s": {"plain": bp[0], "plain_budget": bp[1], "learned": bl[0],
                                  "learned_budget": bl[1], "learned_end": be[0], "learned_end_budget": be[1],
                                  "plain_batched": bpb[0], "plain_batched_budget": bpb[1],
                                  "learned_end_batched": beb[0], "learned_end_batched_budget": beb[1]},
            "per_seed": rows}


def graph_leg(trials=1024, sweeps=2000, reps=3):
    """General sparse graphs through the general-graph kernel (spins in
    shared memory, colour classes in order): a G22-like random graph (2,000
    vertices, 19,990 edges, w = +1), a random graph of the headline's size
    (20,000 vertices, 40,000 edges, w = +-1) and the headline torus given as a
    general graph."""
    import torch
    import paper_2505_18508_gb300 as ia
    out = {}
    inst = synth.torus_instance(200, 100, 2)
    cases = {
        "random_2000v_19990e_w1": synth.random_graph(2000, 19990, 22, weights="one"),
        "random_20000v_40000e_pm1": synth.random_graph(20000, 40000, 81, weights="pm1"),
        "torus_200x100_as_graph": {"n": inst["n"], "row_ptr": inst["row_ptr"], "col": inst["col"],
                                   "J": inst["J"], "h": None},
    }
    betas = synth.linear_betas(0.1, 3.0, sweeps)
    for name, g in cases.items():
        prob = ia.Problem.from_graph(g)
        cuts = torch.empty(trials, dtype=torch.int32, device="cuda")
        ia.anneal(prob, trials, betas, 1, want_spins=False, out_cuts=cuts)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for r in range(reps):
            ia.anneal(prob, trials, betas, 2 + r, want_spins=False, out_cuts=cuts)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        info = prob.graph_info()
        ups = trials * sweeps * g["n"]
        out[name] = {"n": g["n"], "edges": int(len(g["col"]) // 2), "colours": info["colours"], "Dmax": info["Dmax"],
                     "trials": trials, "sweeps": sweeps, "ms": ms, "value": ups / (ms / 1e3),
                     "unit": "spin-updates/s", "best_cut": int(cuts.max().item()),
                     "mean_cut": float(cuts.double().mean().item())}
        prob.destroy()
    return out


def pt_leg(temps=8, chains=128, rounds=200, sweeps_per_round=50):
    """Replica exchange on the headline instance at the headline's update
    budget (temps x chains = 1,024 slots, rounds x sweeps = 10,000 sweeps):
    throughput, and the coldest temperature's cuts against the plain
    annealer's final cuts."""
    import torch
    import paper_2505_18508_gb300 as ia
    inst = synth.torus_instance(200, 100, 2)
    prob = ia.Problem.from_instance(inst)
    betas = np.geomspace(0.5, 3.0, temps)
    ia.anneal_pt(prob, betas, chains, 2, sweeps_per_round, 1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    _, cuts, swaps = ia.anneal_pt(prob, betas, chains, rounds, sweeps_per_round, 1002)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    cold = cuts[(temps - 1) * chains:].cpu().numpy()
    ups = temps * chains * rounds * sweeps_per_round * inst["n"]
    out = {"workload": f"200x100 torus, {temps} temperatures (geometric 0.5..3.0) x {chains} chains, "
                       f"{rounds} rounds x {sweeps_per_round} sweeps", "ms": ms, "value": ups / (ms / 1e3),
           "unit": "spin-updates/s", "swaps": int(swaps.item()),
           "coldest": {"best_cut": int(cold.max()), "mean_cut": float(cold.mean())}}
    prob.destroy()
    return out


def batched_leg(reps=2):
    """Config 3: the 96-instance uneven batch ({50,100,140,200}x100, 32-512
    trials, 2,000-20,000 sweeps) as one graph-replayed persistent launch."""
    import torch
    import paper_2505_18508_gb300 as ia
    cfg = synth.batched_config()
    insts = [synth.torus_instance(c["X"], c["Y"], c["inst_seed"]) for c in cfg]
    probs = [ia.Problem.from_instance(i) for i in insts]
    trials = [c["trials"] for c in cfg]
    sweeps = [c["sweeps"] for c in cfg]
    betas = [synth.linear_betas(0.1, 3.0, S) for S in sweeps]
    seeds = [c["seed"] for c in cfg]
    plan = ia.BatchPlan(probs, trials, sweeps, betas, seeds)
    plan.launch()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        plan.launch()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    ups = sum(t * s * i["n"] for t, s, i in zip(trials, sweeps, insts))
    plan.destroy()
    for p in probs:
        p.destroy()
    return {"workload": "96 tori {50,100,140,200}x100, 32-512 trials, 2,000-20,000 sweeps, one CUDA-graph replay",
            "updates": ups, "ms_per_replay": ms, "value": ups / (ms / 1e3), "unit": "spin-updates/s"}


def dist_env():
    from paper_2505_18508_gb300 import replicas
    return replicas.env()


def reference_arm(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    w = dict(WORKLOAD)
    inst = synth.torus_instance(w["X"], w["Y"], w["inst_seed"])
    sweeps = 1000
    vals = []
    for _ in range(args.warmup):
        oracle_throughput(w, inst, sweeps=sweeps)
    for _ in range(args.steps):
        vals.append(oracle_throughput(w, inst, sweeps=sweeps))
    v = float(np.mean([x["value"] for x in vals]))
    cb = dict(vals[-1])
    cb["value"] = v
    step_ups = vals[-1]["cores"] * sweeps * w["X"] * w["Y"]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "spin-updates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * step_ups / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": {"workload": WORKLOAD_NAME, **w, "updates_per_step": updates_per_step(w)},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": "spin-updates/s", "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ main arm
def main():
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
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-vs-plain comparison")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)

    import torch
    import paper_2505_18508_gb300 as ia
    from paper_2505_18508_gb300 import build as lib_build

    ws, rank, local = dist_env()
    lib_build.build()
    torch.cuda.set_device(local)
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

    from paper_2505_18508_gb300 import replicas

    def seed_of(step):
        return replicas.rank_seed(w["seed"], rank, step)

    for i in range(args.warmup):
        ia.anneal(prob, T, betas, seed_of(-1 - i), out_spins=spins, out_cuts=cuts)
    torch.cuda.synchronize()
    shape = prob.last_launch()

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
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    clk_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tops = sms * IMAD_LANES_PER_SM * clk_mhz * 1e6 / 1e12
    achieved_tops = ups * IMAD_OPS_PER_UPDATE / (ms / 1e3) / 1e12 / 1.0
    roofline = {"bound": "alu", "achieved": achieved_tops, "peak": peak_tops, "unit": "Tops/s (32-bit IMAD)",
                "frac": achieved_tops / peak_tops,
                "traffic": FLOW_TRAFFIC_BYTES if prob.last_kernel() == 2 and (T, S, n) == (1024, 10000, 20000)
                else None,
                "traffic_note": "DRAM bytes per launch (ncu); the spins stay in L2, the path is integer-bound",
                "kernel": {1: "anneal_strip_kernel", 2: "anneal_flow_kernel"}.get(prob.last_kernel(), "?"),
                "peak_source": f"{sms} SMs x {IMAD_LANES_PER_SM} IMAD lanes x "
                f"{clk_mhz:.0f} MHz (sm_max_mhz of measured peaks file)"}

    stats = None
    if args.steps > 0:   # over every rank's trials: the job ran ws * T trials in one step time
        all_cuts = replicas.gather_cuts(first_cuts, dist)
        stats = ttt_stats(all_cuts.cpu().numpy(), ms / 1e3, ws * T, S)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = oracle_throughput(w, inst)
        one = oracle_throughput(w, inst, sweeps=1000, procs=1)   # the oracle on a single host core
        cpu["single_core"] = {"value": one["value"], "sample": one["sample"]}
    # ---- the 16-bit draw mode on the same workload (one Philox block per
    # eight trials): a variant line, not the headline stream
    draw16 = None
    if args.steps > 0:
        prob.set_draw_bits(16)
        for i in range(2):
            ia.anneal(prob, T, betas, seed_of(-10 - i), out_spins=spins, out_cuts=cuts)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(3)]
        for i, (e0, e1) in enumerate(ev):
            flush.zero_()
            e0.record(stream)
            ia.anneal(prob, T, betas, seed_of(200 + i), out_spins=spins, out_cuts=cuts)
            e1.record(stream)
        torch.cuda.synchronize()
        ms16 = float(np.mean([a.elapsed_time(b) for a, b in ev]))
        prob.set_draw_bits(32)
        a16 = ups * (IMAD_OPS_PER_UPDATE / 2) / (ms16 / 1e3) / 1e12
        draw16 = {"value": ws * ups / (ms16 / 1e3), "unit": "spin-updates/s", "ms_per_step": ms16,
                  "workload": "same as the headline, 16-bit draws (decision stream of the 16-bit mode)",
                  "roofline": {"bound": "alu", "achieved": a16, "peak": peak_tops, "frac": a16 / peak_tops,
                               "unit": "Tops/s (32-bit IMAD)", "ops_per_update": IMAD_OPS_PER_UPDATE / 2}}
    batched = None
    if rank == 0 and not args.sweeps and not args.trials:
        batched = batched_leg()
    graphs = None
    pt = None
    if rank == 0 and not args.sweeps and not args.trials:
        graphs = graph_leg()
        pt = pt_leg()
        if stats is not None:
            pt["plain_same_budget"] = {"best_cut": stats["best_cut"], "mean_cut": stats["cut_mean"]}
    campaign = None
    if rank == 0 and not args.sweeps and not args.trials:
        from paper_2505_18508_gb300.campaign import run_campaign
        campaign = run_campaign(prob, (1000, 3000, 10000, 30000, 100000, 300000), 512, 4242)
        campaign["workload"] = ("Fig. 1 style ladder on the headline instance (200x100, seed 2): 512 trials per "
                                "budget, beta 0.1->3.0 over S sweeps, one anneal per budget")
    learned_cmp = None
    if rank == 0 and not args.no_learned and not args.sweeps and not args.trials:
        learned_cmp = learned_leg()

    if rank == 0:
        line = {
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
            "draw16_variant": draw16,
            "campaign": campaign,
            "general_graphs": graphs,
            "replica_exchange": pt,
            "batched": batched,
            "learned_vs_plain": learned_cmp,
            "wall_s_timed": wall,
            "step_ms": step_ms,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    prob.destroy()
    return 0


if __name__ == "__main__":
    sys.exit(main())

"""Time one of the secondary workloads on GPU 0, at full size or scaled down
(for profiling), through the library's public Python API:

    python -m paper_2505_18508_gb300.probe.legs batched [--scale 0.1] [--ctas-per-sm 0]
    python -m paper_2505_18508_gb300.probe.legs pt [--rounds 200] [--sweeps-per-round 50]
    python -m paper_2505_18508_gb300.probe.legs graph [--graph g22] [--sweeps 2000] [--threads-per-site 0] [--strips 0]
    python -m paper_2505_18508_gb300.probe.legs trace [--trace-every 100]

* batched: the 96-instance uneven batch of {50,100,140,200}x100 tori
  (32-512 trials, 2,000-20,000 sweeps, each sweep count times --scale) as one
  graph-replayed persistent launch;
* pt: replica exchange on the 200x100 torus, 8 temperatures (geometric
  0.5..3.0) x 128 chains;
* trace: the 200x100 torus, 1,024 trials x 10,000 sweeps, read out along
  the trajectory (ising_anneal_trace: every trial's cut after every
  --trace-every sweeps, best-so-far cut and configuration) against the same
  anneal read out at the end only;
* graph: 1,024 trials on a general graph: g22 (2,000 vertices, 19,990 edges,
  w = +1), r20k (20,000 vertices, 40,000 edges, w = +-1) or the 200x100 torus
  given as a graph.

Prints one JSON line per timed repetition: milliseconds (CUDA events) and
spin updates per second.  Inputs are seeded and synthetic.
"""
import argparse
import json
import os
import sys


def _setup():
    import torch
    root = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    if root not in sys.path:
        sys.path.insert(0, root)
    torch.cuda.set_device(0)


def _time(fn):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def batched(args):
    import synth
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
    ups = sum(t * s * i["n"] for t, s, i in zip(trials, sweeps, insts))
    plan.launch()
    for _ in range(args.reps):
        ms = _time(plan.launch)
        print(json.dumps({"leg": "batched", "scale": args.scale, "ms": ms, "updates_per_s": ups / (ms * 1e-3)}))
    plan.destroy()
    for p in probs:
        p.destroy()


def pt(args):
    import numpy as np
    import synth
    import paper_2505_18508_gb300 as ia
    inst = synth.torus_instance(200, 100, 2)
    prob = ia.Problem.from_instance(inst)
    betas = np.geomspace(0.5, 3.0, 8)
    ia.anneal_pt(prob, betas, 128, 2, args.sweeps_per_round, 1)
    ups = 8 * 128 * args.rounds * args.sweeps_per_round * inst["n"]
    for r in range(args.reps):
        ms = _time(lambda: ia.anneal_pt(prob, betas, 128, args.rounds, args.sweeps_per_round, 1002 + r))
        print(json.dumps({"leg": "pt", "rounds": args.rounds, "ms": ms, "updates_per_s": ups / (ms * 1e-3),
                          "kernel": prob.last_kernel()}))
    prob.destroy()


def graph(args):
    import torch
    import synth
    import paper_2505_18508_gb300 as ia
    if args.graph == "g22":
        g = synth.random_graph(2000, 19990, 22, weights="one")
    elif args.graph == "r20k":
        g = synth.random_graph(20000, 40000, 81, weights="pm1")
    else:
        inst = synth.torus_instance(200, 100, 2)
        g = {"n": inst["n"], "row_ptr": inst["row_ptr"], "col": inst["col"], "J": inst["J"], "h": None}
    prob = ia.Problem.from_graph(g)
    prob.set_graph_threads_per_site(args.threads_per_site)
    prob.set_launch(strips=args.strips)
    betas = synth.linear_betas(0.1, 3.0, args.sweeps)
    cuts = torch.empty(args.trials, dtype=torch.int32, device="cuda")
    ia.anneal(prob, args.trials, betas, 1, want_spins=False, out_cuts=cuts)
    ups = args.trials * args.sweeps * g["n"]
    for r in range(args.reps):
        ms = _time(lambda: ia.anneal(prob, args.trials, betas, 2 + r, want_spins=False, out_cuts=cuts))
        print(json.dumps({"leg": "graph", "graph": args.graph, "threads_per_site": args.threads_per_site,
                          "strips": prob.last_launch().get("strips"), "ms": ms, "updates_per_s": ups / (ms * 1e-3)}))
    prob.destroy()


def trace(args):
    import synth
    import paper_2505_18508_gb300 as ia
    inst = synth.torus_instance(200, 100, 2)
    prob = ia.Problem.from_instance(inst)
    betas = synth.linear_betas(0.1, 3.0, 10000)
    ups = 1024 * 10000 * inst["n"]
    ia.anneal(prob, 1024, betas, 1)
    ia.anneal_trace(prob, 1024, betas, 1, args.trace_every)
    for r in range(args.reps):
        ms_plain = _time(lambda: ia.anneal(prob, 1024, betas, 1002 + r))
        ms_trace = _time(lambda: ia.anneal_trace(prob, 1024, betas, 1002 + r, args.trace_every))
        print(json.dumps({"leg": "trace", "trace_every": args.trace_every, "ms_plain": ms_plain, "ms_trace": ms_trace,
                          "updates_per_s_trace": ups / (ms_trace * 1e-3), "overhead": ms_trace / ms_plain - 1.0}))
    prob.destroy()


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("leg", choices=["batched", "pt", "graph", "trace"])
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--group-trials", type=int, default=0)
    ap.add_argument("--ctas-per-sm", type=int, default=0)
    ap.add_argument("--rounds", type=int, default=200)
    ap.add_argument("--sweeps-per-round", type=int, default=50)
    ap.add_argument("--graph", default="g22", choices=["g22", "r20k", "torus"])
    ap.add_argument("--trials", type=int, default=1024)
    ap.add_argument("--sweeps", type=int, default=2000)
    ap.add_argument("--trace-every", type=int, default=100)
    ap.add_argument("--threads-per-site", type=int, default=0, help="general graphs: 1, 4, 8 or 0 (automatic)")
    ap.add_argument("--strips", type=int, default=0, help="general graphs: CTAs per trial group (1-8; 0: automatic)")
    args = ap.parse_args(argv)
    _setup()
    {"batched": batched, "pt": pt, "graph": graph, "trace": trace}[args.leg](args)
    return 0


if __name__ == "__main__":
    sys.exit(main())

"""Time the learned stage's network on GPU 0: one forward pass (logits for a
batch of spin configurations) and one gradient (forward, loss, input and
weight gradients), through the library's C ABI.

    python -m paper_2505_18508_gb300.probe.cnn_bench --X 100 --Y 100 --batch 512

Prints one JSON line: milliseconds per call (CUDA events, after warm-up),
useful TFLOP/s (2 * 9 * (3*32 + 32*32*2 + 32*1) flops per site per forward)
and the forward's algorithmic HBM bytes per site: spins in (1 B), the three
BF16 activation maps written and read once each (3 * 2 * 64 B) and FP32
logits out (4 B) = 389 B.  Also the tile proposals on those logits
(ising_propose, 10 x 10 tiles, exact dE <= 0 acceptance; timed last, in
place): 6 algorithmic HBM bytes per site (spins read and written, FP32 logits
read).  Inputs are seeded synthetic tori and spins.
"""
import argparse
import json
import os
import sys

FLOP_PER_SITE = 2 * 9 * (3 * 32 + 32 * 32 * 2 + 32 * 1)
BYTES_PER_SITE = 1 + 3 * 2 * 64 + 4
PROPOSE_BYTES_PER_SITE = 1 + 4 + 1


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--X", type=int, default=100)
    ap.add_argument("--Y", type=int, default=100)
    ap.add_argument("--batch", type=int, default=512)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    args = ap.parse_args(argv)

    import torch
    root = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    if root not in sys.path:
        sys.path.insert(0, root)
    import synth
    import paper_2505_18508_gb300 as ia

    torch.cuda.set_device(0)
    X, Y, B = args.X, args.Y, args.batch
    prob = ia.Problem.from_instance(synth.torus_instance(X, Y, 3))
    net = ia.CNN(synth.cnn_init_params(1, scale=0.7))
    s = torch.from_numpy(synth.random_spins(B, X * Y, 5)).cuda()
    y = torch.from_numpy(synth.random_spins(B, X * Y, 6)).cuda().gt(0).to(torch.uint8)
    z = torch.empty((B, X * Y), dtype=torch.float32, device="cuda")

    def timed(fn, reps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    fwd_ms = timed(lambda: net.forward(prob, s, out=z), args.reps)
    grad_ms = timed(lambda: net.grad(prob, s, y), max(1, args.reps // 4))
    prop_ms = timed(lambda: ia.propose(prob, s, z, 10), args.reps)
    sites = B * X * Y
    out = {
        "workload": f"{B} x {X}x{Y} spin configurations",
        "forward_ms": fwd_ms,
        "forward_tflops": FLOP_PER_SITE * sites / (fwd_ms * 1e-3) / 1e12,
        "forward_gbs": BYTES_PER_SITE * sites / (fwd_ms * 1e-3) / 1e9,
        "grad_ms": grad_ms,
        "grad_status": prob.get_status(),
        "propose_ms": prop_ms,
        "propose_gbs": PROPOSE_BYTES_PER_SITE * sites / (prop_ms * 1e-3) / 1e9,
    }
    print(json.dumps(out), flush=True)
    net.destroy()
    prob.destroy()
    return 0


if __name__ == "__main__":
    sys.exit(main())

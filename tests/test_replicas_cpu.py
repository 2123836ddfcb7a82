"""The host logic of multi-GPU runs on CPU: two gloo ranks (127.0.0.1) check
that the job's step time is the slowest rank's, that the whole-job value
counts every rank's units, that replica seeds differ across ranks, and that
the gather of final cuts concatenates in rank order.  Also: the benchmark's
reference arm exits cleanly on a rank other than 0."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2505_18508_gb300 import replicas
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, lr = replicas.env()
    ms = replicas.max_over_ranks(10.0 + 5.0 * rank, dist)
    cuts = torch.arange(4, dtype=torch.int32) + 100 * rank
    allc = replicas.gather_cuts(cuts, dist)
    seeds = [replicas.rank_seed(1002, rank, s) for s in range(3)]
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(repr({"env": (w, r, lr), "ms": ms, "cuts": allc.tolist(), "seeds": gathered,
                      "value": replicas.job_value(world, 1000.0, ms / 1e3)}))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    res = [eval(open(tmp_path / f"rank{r}.txt").read()) for r in range(2)]
    for r, d in enumerate(res):
        assert d["env"] == (2, r, r)
        assert d["ms"] == 15.0                                  # the slowest rank's time
        assert d["cuts"] == [0, 1, 2, 3, 100, 101, 102, 103]    # rank order
        assert d["value"] == pytest.approx(2 * 1000.0 / 0.015)
    seeds = res[0]["seeds"]
    assert len(set(seeds[0]) | set(seeds[1])) == 6              # distinct across ranks and steps


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import torch
    from paper_2505_18508_gb300 import replicas
    assert replicas.max_over_ranks(3.5) == 3.5
    c = torch.arange(3)
    assert replicas.gather_cuts(c) is c
    assert replicas.job_value(1, 10.0, 2.0) == 5.0


def test_reference_arm_on_rank_one_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_line_keeps_the_contract():
    """Rank 0 of the reference arm (the oracle on the host cores) prints one
    JSON line with the GPU arm's metric, unit and workload config, and the
    keys the benchmark contract asks of it."""
    import json
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "spin-updates/s"
    assert d["higher_is_better"] is True and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 0
    assert d["config"]["workload"] == bench.WORKLOAD_NAME
    assert all(d["config"][k] == v for k, v in bench.WORKLOAD.items())
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"] > 0
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}

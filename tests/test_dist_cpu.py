"""CPU tests of the multi-rank host logic of bench.py, on two `gloo` ranks.

The row ops shard by rows with no exchange between GPUs (weak scaling: each
rank runs the whole step on its own rows), so the only collective work is
host-side bookkeeping: the job's step time is the slowest rank's, the job's
value counts every rank's bytes, each rank draws its own input, and only
rank 0 prints.  These run as two spawned processes on 127.0.0.1.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    from paper_2609_01864_gb300 import synth

    r, w, local = bench.dist_env()
    dist.init_process_group("gloo", init_method="env://", rank=r, world_size=w)
    # step times differ per rank; every rank must see the slowest
    ms = bench.max_over_ranks(10.0 + 7.5 * r, w)
    value = bench.job_value(1 << 30, w, ms)
    # each rank's input is its own draw (seed offset by the rank)
    x = synth.outliers(4, 4096, seed=synth.SEED_DATA + r)
    sums = [torch.zeros(1, dtype=torch.float64) for _ in range(w)]
    dist.all_gather(sums, x.double().sum().reshape(1))
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
        json.dump({"rank": r, "world": w, "local": local, "ms": ms, "value": value,
                   "sums": [float(s.item()) for s in sums]}, f)


def test_two_gloo_ranks_agree_on_the_slowest_step(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r, d in enumerate(res):
        assert (d["rank"], d["world"], d["local"]) == (r, world, r)
        assert d["ms"] == 17.5  # max over ranks, seen by both
        assert d["value"] == pytest.approx((1 << 30) * world / 17.5e-3 / 1e9)
        assert d["sums"] == res[0]["sums"]
    assert res[0]["sums"][0] != res[0]["sums"][1]  # the ranks process different rows


def test_single_rank_needs_no_process_group(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (0, 1, 0)
    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.job_value(2_000_000_000, 1, 1000.0) == pytest.approx(2.0)
    assert bench.job_value(2_000_000_000, 4, 1000.0) == pytest.approx(8.0)


def test_reference_arm_under_torchrun_prints_once():
    """Rank 0 alone times the oracle and prints one JSON line; rank 1 exits 0."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "1", "--ref-seconds", "0.3"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [json.loads(l) for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_ragged_shards_are_contiguous_and_byte_balanced(world):
    """SURVEY-style partitioning of a ragged batch over ranks: contiguous row blocks cut on the prefix sum of
    bytes; the shares tile the row list and differ by less than the widest row."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2609_01864_gb300 import synth
    widths, _ = synth.ragged_widths(20000)
    widths = widths.numpy()
    cuts = [bench.ragged_shard(widths, world, r) for r in range(world)]
    assert cuts[0][0] == 0 and cuts[-1][1] == len(widths)
    assert all(cuts[r][1] == cuts[r + 1][0] for r in range(world - 1))
    share = [int(widths[lo:hi].sum()) for lo, hi in cuts]
    assert max(share) - min(share) <= 2 * int(widths.max())
    assert sum(share) == int(widths.sum())

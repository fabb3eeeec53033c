"""The multi-process path on the CPU (gloo, world size 2).

The single-system step does not shard (replicas only): with N processes every
rank runs its own replica, the timings are max-reduced over the ranks, and
rank 0 reports the whole-job throughput.  Tested here without a GPU: the
max-reduction and the aggregate over two gloo ranks, and the reference arm
under torchrun, where rank 0 alone runs the oracle and prints one line."""
import json
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
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    r, w, local = bench.dist_env()
    d = bench.dist_init(w)
    local_ms = 100.0 + 50.0 * r  # rank 1 is the slow one
    total = bench.reduce_max(d, local_ms)
    steps = 4
    value = w * steps / (total / 1e3)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as fh:
        json.dump({"rank": r, "world": w, "total": total, "value": value}, fh)
    d.barrier()
    d.destroy_process_group()


def test_max_reduce_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp

    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(2)]
    for r in res:
        assert r["world"] == 2 and r["total"] == 150.0  # the slowest rank's time
        assert r["value"] == pytest.approx(2 * 4 / 0.150)  # both replicas' steps over that time


def test_reference_arm_under_torchrun():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus",
           "2", "--steps", "1", "--warmup", "3"]
    env = dict(os.environ, OMP_NUM_THREADS=str(max(1, (os.cpu_count() or 2) // 2)))
    p = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1  # rank 0 only
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0


def _shard_worker(rank, world, port, out_dir):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench
    import mdgen

    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    r, w, _ = bench.dist_env()
    d = bench.dist_init(w)
    systems = mdgen.batch_systems(1, count=200)
    mine, parts = bench.batched_shard(systems, r, w)
    got = [None] * w
    d.all_gather_object(got, {"mine": mine, "parts": parts})
    if r == 0:
        with open(os.path.join(out_dir, "shards.json"), "w") as fh:
            json.dump(got, fh)
    d.barrier()
    d.destroy_process_group()


def test_batched_lpt_shards_over_two_gloo_ranks(tmp_path):
    """The batched form's multi-GPU split: every rank computes the same LPT
    partition of the host cost estimates on its own; the shards are disjoint,
    cover the batch, and their costs differ by at most the largest system's."""
    import torch.multiprocessing as mp

    import mdgen
    import paper_2012_06607_gb300 as md

    port = _free_port()
    mp.start_processes(_shard_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    got = json.load(open(tmp_path / "shards.json"))
    assert got[0]["parts"] == got[1]["parts"]  # same partition on both ranks, no communication needed
    mine = [set(g["mine"]) for g in got]
    assert not (mine[0] & mine[1]) and (mine[0] | mine[1]) == set(range(200))
    costs = md.batched_job_costs(mdgen.batch_systems(1, count=200))
    loads = [sum(costs[i] for i in m) for m in mine]
    assert abs(loads[0] - loads[1]) <= costs.max()


def test_shard_lpt_small_cases():
    import paper_2012_06607_gb300 as md

    assert md.shard_lpt([5.0, 4.0, 3.0, 3.0, 3.0], 2) == [[0, 3], [1, 2, 4]]  # 8 and 10
    assert md.shard_lpt([1.0, 1.0, 1.0], 1) == [[0, 1, 2]]
    assert md.shard_lpt([], 3) == [[], [], []]
    assert md.shard_lpt([2.0, 2.0], 4) == [[0], [1], [], []]
    with pytest.raises(ValueError):
        md.shard_lpt([1.0], 0)

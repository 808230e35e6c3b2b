"""The multi-rank path of bench.py on the CPU: replicas report the slowest rank's time
and the whole-job rate; the reference arm prints only on rank 0."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, lr = bench.rank_env()
    t = bench.reduce_max(10.0 + 5.0 * rank, dist, "cpu")   # rank 1 is the slow one
    q.put((r, w, t, bench.aggregate_rate(w, 20, t)))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29511
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, world, tmax, rate in res:
        assert world == 2 and tmax == 15.0 and rate == pytest.approx(2 * 20 / 15.0)


def test_reference_arm_is_silent_on_other_ranks():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "2", "--warmup", "1"], capture_output=True, text=True, env=env, timeout=120)
    assert p.returncode == 0 and p.stdout.strip() == ""


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference times the FP64 oracle on the host and prints one JSON line
    with the keys the benchmark contract asks for."""
    import json
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    line = json.loads(p.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0
    # the oracle runs on every host core, and the line reports the steps that ran
    cores = len(os.sched_getaffinity(0))
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == cores
    assert line["steps"] == 1 and line["warmup"] == 0 and line["ms_per_step"] > 0
    assert line["cpu_baseline"]["one_thread_value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["unit"] == line["unit"]

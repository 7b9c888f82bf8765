"""CPU checks of bench.py's harness: it parses, the reference arm prints the
contract's JSON line, and the multi-rank timing reduction (max over ranks)
works with world_size 2 over gloo."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_imports_and_parses_args():
    sys.path.insert(0, ROOT)
    import bench
    a = bench.parse_args(["--steps", "7", "--warmup", "3"])
    assert a.steps == 7 and a.warmup == 3 and a.gpus == 1 and a.impl == "ours"
    assert bench.FWD_BYTES > 1024 and bench.BWD_BYTES > 2048


def test_reference_arm_prints_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "Gaussians/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0
    sys.path.insert(0, ROOT)
    import bench
    assert line["config"] == bench.step_config(bench.parse_args([]), 1)  # the same workload as our arm


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    ws, rk = bench.dist_init("gloo")
    v = bench.max_over_ranks(1.0 + rank)
    bench.barrier()
    q.put((rk, ws, v))


def test_max_over_ranks_gloo_world_size_2():
    import multiprocessing as mp
    import random
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = random.randint(20000, 40000)
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert res == [(0, 2, 2.0), (1, 2, 2.0)]


def test_all_cores_oracle_timing():
    """One single-threaded oracle process per host core, started together:
    the line reports every core and a positive rate."""
    sys.path.insert(0, ROOT)
    import bench
    r = bench.cpu_baseline_all_cores(20_000.0, seconds=0.05)
    assert r["kind"] == "oracle" and r["cores"] == (os.cpu_count() or 1) and r["value"] > 0
    assert r["unit"] == "Gaussians/s" and "processes" in r["sample"]

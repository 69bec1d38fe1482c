"""The N > 1 launch path of bench.py on the CPU: two gloo ranks synchronise,
take the slowest rank's time, and report whole-job weak-scaling throughput;
under several ranks the reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    R = bench.Ranks("gloo")
    assert (R.world, R.rank) == (world, rank)
    R.barrier()
    ms = 100.0 + 50.0 * rank          # rank 1 is the slowest
    slowest = R.max(ms)
    out[rank] = (slowest, bench.weak_throughput(R.world, 1000, slowest))
    R.barrier()
    R.close()


def test_two_gloo_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]                   # every rank sees the same max
    slowest, value = res[0]
    assert slowest == 150.0
    assert value == pytest.approx(2 * 1000 * 1e3 / 150.0)


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK")}
    old = dict(os.environ)
    os.environ.clear()
    os.environ.update(env)
    try:
        R = bench.Ranks("gloo")
        assert R.world == 1 and R.dist is None and R.max(3.5) == 3.5
    finally:
        os.environ.clear()
        os.environ.update(old)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip() == ""

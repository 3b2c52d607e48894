"""Multi-GPU runs are independent replicas (no collective on the data path): bench.py's whole-job
aggregation takes the slowest rank's time and the units of every rank.  Checked here with two
gloo ranks on the CPU; the reference arm does its work on rank 0 only."""
import os
import socket
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [120.0, 180.0][rank]
    q.put((rank, bench.replica_throughput(local_ms, 1e9, dist, "cpu")))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_all_units():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        ms, value = out[r]
        assert ms == 180.0
        assert value == pytest.approx(2 * 1e9 / 0.18)


def test_single_process_aggregation_is_the_local_figure():
    import bench
    ms, value = bench.replica_throughput(50.0, 1e9)
    assert ms == 50.0 and value == pytest.approx(2e10)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import bench
    args = types.SimpleNamespace(warmup=0, steps=1, ref_iters=1, gpus=2)
    bench.run_reference(args, rank=1, world=2)
    assert capsys.readouterr().out == ""

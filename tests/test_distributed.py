"""The bench's multi-rank harness on CPU: two gloo ranks agree on the max-over-ranks time, pass the
barrier, and count different replicas (one hash seed per rank).  The reference arm prints on rank 0
only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(dist)
    m = bench.max_over_ranks(dist, float(10 * (rank + 1)))
    seed = bench.SEED + rank  # the replica seed rule of single_stream_setup
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, m, seed))


def test_two_gloo_ranks_agree_on_max_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [20.0, 20.0]          # max over ranks
    assert res[0][2] != res[1][2]                        # each rank counts its own replica


def test_reference_arm_prints_on_rank0_only(monkeypatch, capsys):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench

    class A:
        workload = "rmat_s20"
        c = 100
        steps = 1
        warmup = 0
        gpus = 2
    assert bench.run_reference(A, 2, 1, None) == 0     # rank 1: no work, no output
    assert capsys.readouterr().out == ""

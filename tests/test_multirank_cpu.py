"""The N-GPU bench path on CPU: world-size-2 gloo process groups run the
cross-rank aggregation bench.py uses (largest elapsed time, summed units),
and each rank of the batched workload gets its own ensemble."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_1505_02037_gb300 import workloads as W
        ms, units = bench.over_ranks(10.0 + 5 * rank, 100.0 * (rank + 1), world, "cpu")
        runs = W.ensemble(nruns=8, seed=bench.ENSEMBLE_SEED + rank)
        q.put((rank, ms, units, [r["N"] for r in runs]))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation_and_sharded_ensembles():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, ms, units, _ in out:
        assert ms == 15.0 and units == 300.0, (rank, ms, units)
    assert out[0][3] != out[1][3]  # independent ensembles, one per rank


def test_single_rank_is_identity():
    pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    assert bench.over_ranks(12.5, 7.0, 1, "cpu") == (12.5, 7.0)

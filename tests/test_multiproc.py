"""The N > 1 benchmark path on CPU: world size 2 over gloo.

Each rank is an independent camera stream (its own seeded sequence, no
data-path collective); the only collective is the max of the timed region
over ranks, and the job throughput counts every rank's frames.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from synth import make_sequence
    seed = bench.rank_seed(rank)
    seq = make_sequence("tiny", seed, n_frames=2)
    d, rgb, T, _ = seq.frame(1)
    local_ms = 10.0 * (rank + 1)  # rank 1 is the slower one
    job_ms = bench.max_over_ranks(local_ms, dist, torch.device("cpu"))
    out[rank] = (seed, float(T[0, 3]), int(d.sum()), job_ms, bench.job_throughput(world, 5, job_ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_over_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] != res[1][0]                     # distinct streams
    assert res[0][1:3] != res[1][1:3]                 # different frames and poses: no shared data
    assert res[0][3] == res[1][3] == 20.0             # max over ranks
    assert abs(res[0][4] - 2 * 5 / 0.020) < 1e-9      # all ranks' frames over the slowest time

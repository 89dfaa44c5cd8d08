"""The benchmark's multi-rank path (one independent cavity per rank, no
data-path collective): max-over-ranks timing and the whole-job value, run as
two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    t_local = 1.5 + rank            # rank 1 is the slowest
    t_max = bench.max_over_ranks(t_local)
    v = bench.whole_job_mlups(4096 * 4096, 2000, world, t_max)
    out[rank] = (t_max, v, bench.replica_seed(2, rank))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time_and_whole_job_value():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 2.5
    expect = 2 * 4096 * 4096 * 2000 / 2.5 / 1e6
    assert out[0][1] == pytest.approx(expect) and out[1][1] == pytest.approx(expect)
    assert out[0][2] == 2 and out[1][2] == 3  # rank 0 keeps the single-GPU input


def test_single_process_is_identity():
    import bench

    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.whole_job_mlups(100, 10, 1, 2.0) == pytest.approx(100 * 10 / 2.0 / 1e6)

"""The multi-process slab path's host logic without a GPU, as two and three
gloo ranks on the CPU: the row partition, the halo messages reaching the
right neighbour's halo slots, and the observables' accumulators combined in
rank order into the same bits on every rank."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1608_04118_gb300 import build

    build.build()


def test_row_partition_covers_the_cavity_once():
    from paper_1608_04118_gb300 import ltne as L

    for ny in (4, 5, 17, 64, 1000):
        for n in range(1, ny // 2 + 1):
            y, seen = 0, []
            for i in range(n):
                y0, rows, lo, hi = L.ltne_slab_rows(ny, n, i)
                assert y0 == y and rows >= 2 and rows in (ny // n, ny // n + 1)
                assert lo == (i > 0) and hi == (i < n - 1)
                seen.append(rows)
                y += rows
            assert y == ny
            assert seen == sorted(seen, reverse=True)  # the longer slabs come first
    with pytest.raises(L.LtneError):
        L.ltne_slab_rows(7, 4, 0)  # fewer than 2 rows per slab
    with pytest.raises(L.LtneError):
        L.ltne_slab_rows(64, 4, 4)


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1608_04118_gb300 import ltne as L
    from paper_1608_04118_gb300.slabs import HaloExchange, all_accumulators, combine_accumulators

    nx = 7
    # messages tagged with the sender and the side they leave by
    send_lo = torch.full((5 * nx,), 100.0 * rank + 1) if rank > 0 else None
    send_hi = torch.full((5 * nx,), 100.0 * rank + 2) if rank < world - 1 else None
    recv_lo = torch.zeros(5 * nx) if rank > 0 else None
    recv_hi = torch.zeros(5 * nx) if rank < world - 1 else None
    hx = HaloExchange(rank, world, send_lo, send_hi, recv_lo, recv_hi, host_staged=True)
    for _ in range(3):
        hx.exchange()
    got = (None if recv_lo is None else float(recv_lo[0]),
           None if recv_hi is None else float(recv_hi[0]))
    # accumulators: sums in most slots, maxima in slots 6 and 7
    rng = np.random.default_rng(10 + rank)
    acc = rng.uniform(-1, 1, L.LTNE_NACC)
    parts = all_accumulators(acc)
    comb = combine_accumulators(parts)
    p = L.ltne_default_params(33, 40)
    ob = L.ltne_observables_from_accumulators(p, 12, 1, np.abs(comb), allow_nonfinite=True)
    out[rank] = (got, acc, comb, ob)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_exchange_halos_and_combine_accumulators(world):
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        lo, hi = out[r][0]
        # the halo below holds what the rank below sent upwards, and so on
        assert lo == (None if r == 0 else 100.0 * (r - 1) + 2)
        assert hi == (None if r == world - 1 else 100.0 * (r + 1) + 1)
    accs = [np.asarray(out[r][1]) for r in range(world)]
    expect = accs[0].copy()
    for a in accs[1:]:
        for k in range(len(expect)):
            expect[k] = max(expect[k], a[k]) if k in (6, 7) else expect[k] + a[k]
    for r in range(world):
        assert np.array_equal(out[r][2], expect)  # the same bits on every rank
        assert out[r][3] == out[0][3]

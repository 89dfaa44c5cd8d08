"""The benchmark's host-side logic without a GPU: the multi-rank path (one
independent cavity per rank, no data-path collective: max-over-ranks timing
and the whole-job value, run as two gloo ranks on the CPU), the reference
arm's JSON line and the CPU-baseline object."""
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


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference: the FP64 oracle on the host cores, one JSON
    line with the reference keys (a small lattice, two steps)."""
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n", "64",
                        "--steps", "2", "--warmup", "1"], cwd=root, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "MLUPS" and line["value"] > 0
    assert line["steps"] == 2 and line["warmup"] == 1 and line["higher_is_better"] is True
    cpu = line["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_cpu_baseline_reports_one_core_and_the_small_configuration():
    import bench

    cpu = bench.cpu_baseline_oracle(64, target_s=0.2)
    assert cpu["kind"] == "oracle" and cpu["value"] > 0 and cpu["cores"] >= 1
    assert cpu["one_core"]["value"] > 0
    assert cpu["c1_64x64_1e4_steps_s"] > 0

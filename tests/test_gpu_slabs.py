"""Row-slab decomposition on one GPU: the lattice advanced as 2-4 slabs of
rows with their own buffers and halo rows exchanged by device copies after
every step gives the same bits as the undivided step (the decomposition a
multi-GPU run would use, exercised without a second GPU)."""
import numpy as np
import pytest

from paper_1608_04118_gb300 import workloads as W
from tests.helpers import cavity_for

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_04118_gb300 import build

    build.build()


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("nslabs", [1, 2, 3, 4])
def test_slabs_equal_the_undivided_step(storage, nslabs):
    nx, ny = 67, 45
    cfg = W.random_params(81, nx, ny)
    phi = W.porosity_field(nx, ny, 0.4, 0.9, seed=82).reshape(-1)
    fields = W.random_fields(nx, ny, 83)
    a = cavity_for(cfg, storage=storage, phi=phi).set_schedule(128, 2, 1)
    a.set_fields(porosity=phi, **fields).step(150)
    b = cavity_for(cfg, storage=storage, phi=phi)
    b.set_fields(porosity=phi, **fields).step_slabs(nslabs, 100).step_slabs(nslabs, 50)
    fa, fb = a.fields(), b.fields()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), (nslabs, k)
    assert a.get_state() == b.get_state()
    assert b.observables()["step"] == 150


def test_slabs_continue_with_plain_steps():
    """Slab steps and plain steps interleave on the same state."""
    nx, ny = 96, 40
    cfg = W.random_params(84, nx, ny)
    a = cavity_for(cfg, storage="f32").set_schedule(128, 2, 1).set_fields().step(91)
    b = cavity_for(cfg, storage="f32").set_schedule(128, 2, 1).set_fields()
    b.step(30).step_slabs(3, 31).step(30)
    fa, fb = a.fields(), b.fields()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k


def test_slabs_reject_unsupported_forms():
    from paper_1608_04118_gb300.ltne import LtneError

    cfg = W.random_params(85, 40, 20)
    with pytest.raises(LtneError):
        cavity_for(cfg, storage="f16").set_fields().step_slabs(2, 5)
    with pytest.raises(LtneError):
        cavity_for(cfg, storage="f32").set_fields().step_slabs(11, 5)  # < 2 rows per slab


# ---- one slab per process ---------------------------------------------------

def _free_port():
    import socket

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _slab_rank(rank, world, port, nx, ny, params, phi, fields, steps, path):
    """One process: its slab of the cavity on cuda:0, halos through gloo
    (staged through host memory), the whole fields gathered at the end."""
    import os

    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    from paper_1608_04118_gb300.slabs import DistributedCavity

    dc = DistributedCavity(nx, ny, **params)
    dc.set_fields(porosity=phi, **fields)
    obs = []
    for k in steps:
        dc.step(k)
        obs.append(dc.observables())
    f = dc.gather_fields()
    launches = dc.slab.launches
    dc.close()
    if rank == 0:
        np.savez(path, obs=np.array([[o[k] for k in sorted(o)] for o in obs]),
                 keys=np.array(sorted(obs[0])), launches=launches, **f)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("storage,world", [("f32", 2), ("f32", 3), ("f64", 2)])
def test_processes_with_one_slab_each_equal_the_undivided_step(storage, world, tmp_path):
    """2 or 3 processes on the one GPU, each advancing one row slab of a
    cavity with per-node porosity (Ergun medium) from random fields; the
    halos move between the processes through gloo between steps (no kernel
    waits on another process).  The gathered fields are the bits of the
    undivided lattice (one node per thread), which derives the Ergun
    diameter itself while the slabs are given ltne_ergun_diameter of the
    whole field; the combined observables match it to rounding."""
    import torch.multiprocessing as mp

    from paper_1608_04118_gb300.ltne import LTNE_K_ERGUN, ltne_ergun_diameter
    from tests.helpers import phys

    nx, ny = 70, 47
    cfg = dict(W.random_params(86, nx, ny), ergun=True)
    phi = W.porosity_field(nx, ny, 0.4, 0.9, seed=87).reshape(-1)
    fields = W.random_fields(nx, ny, 88)
    steps = (60, 1, 39)
    a = cavity_for(cfg, storage=storage, phi=phi).set_schedule(64, 2, 1)
    a.set_fields(porosity=phi, **fields)
    ref_obs = []
    for k in steps:
        a.step(k)
        ref_obs.append(a.observables())
    ref = a.fields()
    d = ltne_ergun_diameter(phi, ny - 1, cfg["Da"])
    params = dict(phys(cfg), storage=storage, permeability=LTNE_K_ERGUN, porosity_field=1, d_p=d)
    path = str(tmp_path / "slabs.npz")
    mp.spawn(_slab_rank, args=(world, _free_port(), nx, ny, params, phi, fields, steps, path),
             nprocs=world, join=True)
    got = np.load(path)
    for k in ref:
        assert np.array_equal(got[k], ref[k]), k
    keys = [str(k) for k in got["keys"]]
    assert int(got["launches"]) == sum(steps)
    for row, ob in zip(got["obs"], ref_obs):
        o = dict(zip(keys, row))
        for k in ("Nu_f_hot", "Nu_s_hot", "Nu_f_cold", "Nu_s_cold", "mass", "energy",
                  "mean_Tf", "mean_Ts", "Fo"):
            assert o[k] == pytest.approx(ob[k], rel=1e-6, abs=1e-12), k
        for k in ("max_u", "max_dT", "step", "nonfinite"):
            assert o[k] == ob[k], k
        if np.isnan(ob["residual"]):
            assert np.isnan(o["residual"])
        else:
            assert o["residual"] == pytest.approx(ob["residual"], rel=1e-5)


def test_slab_handle_rejects_whole_lattice_calls():
    from paper_1608_04118_gb300 import ltne as L

    p = dict(Ra=1e4, storage="f32")
    s = L.SlabCavity(40, 20, 2, 0, **p).set_fields()
    for call in (lambda: L.ltne_step(s.h, 3), lambda: L.ltne_observables(s.h),
                 lambda: L.ltne_set_schedule(s.h, 128, 1, 2), lambda: L.ltne_set_staging(s.h, 1)):
        with pytest.raises(L.LtneError):
            call()
    with pytest.raises(L.LtneError):  # the diameter of a whole field cannot come from a slab
        L.SlabCavity(40, 20, 2, 1, storage="f32", permeability=L.LTNE_K_ERGUN, porosity_field=1)
    with pytest.raises(L.LtneError):  # 16-bit storage: node-keyed rounding
        L.SlabCavity(40, 20, 2, 1, storage="f16")

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

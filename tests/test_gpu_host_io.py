"""Host-side staging of the fields through the C ABI on lattices large enough
that a field crosses the pinned staging buffers more than once (32 MB each):
the porosity pass (range check, conversion and Ergun mean in one read of
the field), the failure of set_fields part-way through, and get_fields into
caller-owned arrays."""
import numpy as np
import pytest

from paper_1608_04118_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# 4096 x 2100 FP64: 1024 rows per pinned block, so the porosity field goes
# up in three blocks, and the Ergun mean's chunk 31 (rows 1017-1050) spans
# the first two
NX, NY = 4096, 2100


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_04118_gb300 import build

    build.build()


def _cavity(**kw):
    from paper_1608_04118_gb300.ltne import Cavity, LTNE_K_ERGUN

    c = W.C2_THROUGHPUT
    return Cavity(NX, NY, storage="f64", Ra=c["Ra"], Pr=c["Pr"], Da=c["Da"], H=c["H"],
                  gamma_sf=c["gamma_sf"], permeability=LTNE_K_ERGUN, porosity_field=1, **kw)


def _phi():
    c = W.C2_THROUGHPUT
    return W.porosity_field(NX, NY, c["phi_lo"], c["phi_hi"], 5).reshape(-1)


def test_staged_porosity_derives_the_ergun_diameter_bits():
    """A handle that derives the Ergun diameter while staging the field
    steps the same bits (FP64: the diameter enters every node's drag) as
    one given ltne_ergun_diameter of the field."""
    from paper_1608_04118_gb300.ltne import ltne_ergun_diameter

    phi = _phi()
    d = ltne_ergun_diameter(phi, NY - 1, W.C2_THROUGHPUT["Da"])
    a = _cavity().set_fields(porosity=phi).step(3)
    fa = a.fields()
    a.close()
    b = _cavity(d_p=d).set_fields(porosity=phi).step(3)
    fb = b.fields()
    b.close()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k
    assert np.abs(fa["ux"]).max() > 0  # the drag has acted


def test_set_fields_failing_in_a_later_block_leaves_no_fields():
    """A porosity value out of (0, 1) in the last staged block is found after
    earlier blocks were copied: set_fields fails with INVALID_ARG, the
    handle then has no fields (STATE), and a valid call restores it."""
    from paper_1608_04118_gb300.ltne import LTNE_ERR_INVALID_ARG, LTNE_ERR_STATE, LtneError

    phi = _phi()
    c = _cavity().set_fields(porosity=phi).step(2)
    bad = phi.copy()
    bad[-7] = 1.0
    with pytest.raises(LtneError) as e:
        c.set_fields(porosity=bad)
    assert e.value.code == LTNE_ERR_INVALID_ARG
    with pytest.raises(LtneError) as e:
        c.step(1)
    assert e.value.code == LTNE_ERR_STATE
    f1 = c.set_fields(porosity=phi).step(2).fields()
    f2 = _cavity().set_fields(porosity=phi).step(2).fields()
    for k in f1:
        assert np.array_equal(f1[k], f2[k]), k
    c.close()


def test_fields_into_caller_arrays():
    from paper_1608_04118_gb300.ltne import FIELD_KEYS

    phi = _phi()
    c = _cavity().set_fields(porosity=phi).step(4)
    ref = c.fields()
    out = {k: np.full((NY, NX), np.nan) for k in FIELD_KEYS}
    got = c.fields(out=out)
    for k in FIELD_KEYS:
        assert got[k] is out[k]
        assert np.array_equal(out[k], ref[k]), k
    with pytest.raises(ValueError):
        c.fields(out=dict(out, Tf=np.empty((NX, NY))))
    with pytest.raises(ValueError):
        c.fields(out=dict(out, Ts=np.empty((NY, NX), dtype=np.float32)))
    c.close()

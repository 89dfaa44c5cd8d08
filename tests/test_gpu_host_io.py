"""Whole fields between the caller's host arrays and the device through the
C ABI, in both host I/O forms: staged (host threads convert through two
pinned 32 MB buffers) and direct (kernels read and write the host arrays
themselves, where the GPU reaches pageable host memory).  The lattice is
large enough that a field crosses the pinned buffers more than once.
Checked: the porosity pass (range check, conversion and Ergun mean in one
read of the field) derives the Ergun diameter of ltne_ergun_diameter, the
two forms give the same bits and the same errors, a failure part-way
leaves the handle without fields, and get_fields fills caller-owned
arrays (pageable or page-locked; the direct form writes only page-locked
ones with a kernel)."""
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


def _direct_supported():
    from paper_1608_04118_gb300.ltne import LTNE_HOST_IO_DIRECT, LtneError

    c = _cavity(nx=64, ny=64)
    try:
        c.set_host_io(LTNE_HOST_IO_DIRECT)
        return True
    except LtneError:
        return False
    finally:
        c.close()


def _modes():
    from paper_1608_04118_gb300.ltne import LTNE_HOST_IO_DIRECT, LTNE_HOST_IO_STAGED

    return [LTNE_HOST_IO_STAGED] + ([LTNE_HOST_IO_DIRECT] if _direct_supported() else [])


def _cavity(mode=None, nx=NX, ny=NY, storage="f64", **kw):
    from paper_1608_04118_gb300.ltne import Cavity, LTNE_K_ERGUN

    c = W.C2_THROUGHPUT
    cav = Cavity(nx, ny, storage=storage, Ra=c["Ra"], Pr=c["Pr"], Da=c["Da"], H=c["H"],
                 gamma_sf=c["gamma_sf"], permeability=LTNE_K_ERGUN, porosity_field=1, **kw)
    if mode is not None:
        cav.set_host_io(mode)
    return cav


def _pinned_fields(nx, ny):
    """Caller arrays in page-locked host memory (where the direct form writes
    with a kernel; pageable ones are staged)."""
    from paper_1608_04118_gb300.ltne import FIELD_KEYS

    return {k: torch.empty((ny, nx), dtype=torch.float64, pin_memory=True).numpy()
            for k in FIELD_KEYS}


def _phi(nx=NX, ny=NY):
    c = W.C2_THROUGHPUT
    return W.porosity_field(nx, ny, c["phi_lo"], c["phi_hi"], 5).reshape(-1)


def test_the_default_form_is_direct_where_the_device_allows_it():
    from paper_1608_04118_gb300.ltne import LTNE_HOST_IO_DIRECT, LTNE_HOST_IO_STAGED

    c = _cavity(nx=64, ny=64)
    assert c.host_io == (LTNE_HOST_IO_DIRECT if _direct_supported() else LTNE_HOST_IO_STAGED)
    assert c.set_host_io(LTNE_HOST_IO_STAGED).host_io == LTNE_HOST_IO_STAGED
    c.close()


def test_porosity_pass_derives_the_ergun_diameter_bits():
    """A handle that derives the Ergun diameter while reading the field
    steps the same bits (FP64: the diameter enters every node's drag) as
    one given ltne_ergun_diameter of the field, in every host I/O form."""
    from paper_1608_04118_gb300.ltne import ltne_ergun_diameter

    phi = _phi()
    d = ltne_ergun_diameter(phi, NY - 1, W.C2_THROUGHPUT["Da"])
    b = _cavity(d_p=d).set_fields(porosity=phi).step(3)
    fb = b.fields()
    b.close()
    assert np.abs(fb["ux"]).max() > 0  # the drag has acted
    for mode in _modes():
        a = _cavity(mode).set_fields(porosity=phi).step(3)
        fa = a.fields()
        a.close()
        for k in fa:
            assert np.array_equal(fa[k], fb[k]), (mode, k)


@pytest.mark.parametrize("storage", ["f32", "f64"])
def test_direct_and_staged_forms_give_the_same_bits(storage):
    from paper_1608_04118_gb300.ltne import FIELD_KEYS

    modes = _modes()
    if len(modes) < 2:
        pytest.skip("the device does not reach pageable host memory")
    nx, ny = 2500, 1700  # padded rows; FP64 fields span two pinned blocks
    phi = _phi(nx, ny)
    fields = W.random_fields(nx, ny, 91)
    got = []
    for mode in modes:
        c = _cavity(mode, nx=nx, ny=ny, storage=storage)
        c.set_fields(porosity=phi, **fields)
        f0 = {k: v.copy() for k, v in c.fields(out=_pinned_fields(nx, ny)).items()}
        c.step(5)
        f1 = {k: v.copy() for k, v in c.fields(out=_pinned_fields(nx, ny)).items()}
        got.append((f0, f1, c.get_state()))
        # pageable arrays (staged in either form), and the other form, read
        # the same state back to the same bits
        fp = c.fields()
        c.set_host_io(modes[1 - modes.index(mode)])
        f2 = c.fields(out=_pinned_fields(nx, ny))
        for k in FIELD_KEYS:
            assert np.array_equal(f1[k], fp[k]), (mode, k)
            assert np.array_equal(f1[k], f2[k]), (mode, k)
        c.close()
    (a0, a1, sa), (b0, b1, sb) = got
    for k in FIELD_KEYS:
        assert np.array_equal(a0[k], b0[k]), k
        assert np.array_equal(a1[k], b1[k]), k
    assert sa == sb


@pytest.mark.parametrize("bad", ["porosity_one", "porosity_nan", "rho_inf"])
def test_set_fields_failing_part_way_leaves_no_fields(bad):
    """A value out of range in the last staged block is found after earlier
    blocks were copied (staged) or while the kernels read the arrays
    (direct): set_fields fails with INVALID_ARG, the handle then has no
    fields (STATE), and a valid call restores it."""
    from paper_1608_04118_gb300.ltne import LTNE_ERR_INVALID_ARG, LTNE_ERR_STATE, LtneError

    phi = _phi()
    ref = _cavity().set_fields(porosity=phi).step(2).fields()
    for mode in _modes():
        c = _cavity(mode).set_fields(porosity=phi).step(2)
        p, rho = phi.copy(), None
        if bad == "porosity_one":
            p[-7] = 1.0
        elif bad == "porosity_nan":
            p[-7] = np.nan
        else:
            rho = np.ones(NX * NY)
            rho[-7] = np.inf
        with pytest.raises(LtneError) as e:
            c.set_fields(porosity=p, rho=rho)
        assert e.value.code == LTNE_ERR_INVALID_ARG, mode
        with pytest.raises(LtneError) as e:
            c.step(1)
        assert e.value.code == LTNE_ERR_STATE, mode
        f = c.set_fields(porosity=phi).step(2).fields()
        for k in f:
            assert np.array_equal(f[k], ref[k]), (mode, k)
        c.close()


def test_fields_into_caller_arrays():
    from paper_1608_04118_gb300.ltne import FIELD_KEYS

    phi = _phi()
    for mode in _modes():
        c = _cavity(mode).set_fields(porosity=phi).step(4)
        ref = c.fields()
        for out in ({k: np.full((NY, NX), np.nan) for k in FIELD_KEYS}, _pinned_fields(NX, NY)):
            got = c.fields(out=out)
            for k in FIELD_KEYS:
                assert got[k] is out[k]
                assert np.array_equal(out[k], ref[k]), (mode, k)
        with pytest.raises(ValueError):
            c.fields(out=dict(out, Tf=np.empty((NX, NY))))
        with pytest.raises(ValueError):
            c.fields(out=dict(out, Ts=np.empty((NY, NX), dtype=np.float32)))
        c.close()

"""C ABI checks that need no GPU: the library loads, exports every symbol
include/ltne.h declares, the Python records match the C layout, and the
host-side validation returns the documented status codes."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


@pytest.fixture(scope="module")
def lt():
    from paper_1608_04118_gb300 import build

    build.build()
    from paper_1608_04118_gb300 import ltne

    ltne.load()
    return ltne


def declared_functions():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(ltne_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(lt):
    names = declared_functions()
    assert "ltne_step" in names and "ltne_create" in names
    lib = C.CDLL(lt.LIB_PATH)
    for n in sorted(names):
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", lt.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\b(ltne_\w+)\b", out))
    assert names <= exported
    # the binding wraps exactly the declared functions
    assert set(lt.SIGNATURES) == names


def _c_layout(struct, fields):
    src = ['#include <stdio.h>', '#include <stddef.h>', '#include "ltne.h"', "int main(void){",
           'printf("%%zu\\n", sizeof(%s));' % struct]
    for f in fields:
        src.append('printf("%%zu\\n", offsetof(%s, %s));' % (struct, f))
    src.append("return 0;}")
    d = os.path.join(ROOT, "_build")
    os.makedirs(d, exist_ok=True)
    c = os.path.join(d, "layout_%s.c" % struct)
    exe = os.path.join(d, "layout_%s" % struct)
    open(c, "w").write("\n".join(src))
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
    vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    return vals[0], vals[1:]


@pytest.mark.parametrize("name", ["ltne_params", "ltne_obs"])
def test_struct_layout_matches_header(lt, name):
    py = getattr(lt, name)
    fields = [f for f, _ in py._fields_]
    size, offs = _c_layout(name, fields)
    assert C.sizeof(py) == size
    assert [getattr(py, f).offset for f in fields] == offs


def test_defaults_follow_section4(lt):
    """The relaxation rates, the thermal weight parameter and the viscosity
    ratio default to the paper's Sec. 4 values (tests/golden); T_ref
    defaults to the mean wall temperature."""
    from tests.helpers import golden

    g = golden("sec4_parameters")
    p = lt.ltne_default_params(64, 64)
    for k in ("s_e", "s_eps", "s_q", "zeta_e", "zeta_nu", "eta_e", "eta_nu", "varpi", "J_e"):
        assert getattr(p, k) == g[k], k
    assert p.T_ref == 0.5


def _create(lt, **kw):
    p = lt.ltne_default_params(kw.pop("nx", 32), kw.pop("ny", 32), **kw)
    h = C.c_void_p()
    rc = lt.load().ltne_create(C.byref(p), None, C.byref(h))
    if h:
        lt.ltne_destroy(h)
    return rc


def test_create_validation_codes(lt):
    assert _create(lt) == lt.LTNE_OK
    assert _create(lt, nx=3) == lt.LTNE_ERR_INVALID_ARG
    assert _create(lt, porosity=1.0) == lt.LTNE_ERR_INVALID_ARG
    assert _create(lt, porosity=0.0) == lt.LTNE_ERR_INVALID_ARG
    assert _create(lt, varpi=1.2) == lt.LTNE_ERR_INVALID_ARG
    assert _create(lt, storage=9) == lt.LTNE_ERR_INVALID_ARG
    assert _create(lt, Pr=float("nan")) == lt.LTNE_ERR_INVALID_ARG
    assert _create(lt, Ra=0.0) == lt.LTNE_ERR_INVALID_ARG  # no viscosity without nu_override
    assert _create(lt, Ra=0.0, nu_override=0.1) == lt.LTNE_OK
    assert _create(lt, s_q=2.0) == lt.LTNE_ERR_UNSTABLE_TAU
    assert _create(lt, nu_override=1e-7, Ra=0.0) == lt.LTNE_OK  # s_nu -> 2 from below
    assert _create(lt, Ra=1e12, nx=8, ny=8) == lt.LTNE_OK
    # thermal diffusivity so large that eta_alpha leaves (0, 2) cannot happen
    # (it only tends to 0); a negative rate input is rejected
    assert _create(lt, zeta_e=-0.5) == lt.LTNE_ERR_UNSTABLE_TAU


def test_workspace_size_and_state_calls_without_gpu(lt):
    p = lt.ltne_default_params(100, 70)
    h = lt.ltne_create(p)
    try:
        nb = lt.ltne_workspace_bytes(h)
        # two 19-plane population buffers of padded 128 x 70 fp32 planes at least
        assert nb >= 2 * 19 * 128 * 70 * 4
        lib = lt.load()
        # calls that need a workspace report the order error, not a crash
        assert lib.ltne_step(h, 1) == lt.LTNE_ERR_STATE
        assert lib.ltne_set_fields(h, None, None, None, None, None, None) == lt.LTNE_ERR_STATE
        assert lib.ltne_bind_workspace(h, C.c_void_p(256), 10) == lt.LTNE_ERR_WORKSPACE
        assert lib.ltne_bind_workspace(h, C.c_void_p(257), nb) == lt.LTNE_ERR_WORKSPACE
        assert lib.ltne_step(h, -1) == lt.LTNE_ERR_INVALID_ARG
    finally:
        lt.ltne_destroy(h)
    assert lt.ltne_error_string(lt.LTNE_ERR_UNSTABLE_TAU).startswith("LTNE_ERR_UNSTABLE_TAU")


def test_option_validation_without_gpu(lt):
    import ctypes as C

    lib = lt.load()
    # local h_v needs a positive D_p / L; switches are 0 or 1
    assert _create(lt, hv_local=1) == lt.LTNE_OK
    assert _create(lt, hv_local=1, Dp_over_L=0.0) == lt.LTNE_ERR_INVALID_ARG
    assert _create(lt, hv_local=2) == lt.LTNE_ERR_INVALID_ARG
    assert _create(lt, thermal_correction=1) == lt.LTNE_OK
    assert _create(lt, thermal_correction=-1) == lt.LTNE_ERR_INVALID_ARG
    # the batched form is FP32 cavities with uniform porosity and neither option
    for kw in (dict(hv_local=1), dict(thermal_correction=1), dict(storage=lt.LTNE_F64),
               dict(porosity_field=1), dict(bc=lt.LTNE_BC_PERIODIC)):
        arr = (lt.ltne_params * 2)(lt.ltne_default_params(32, 32),
                                   lt.ltne_default_params(48, 32, **kw))
        b = C.c_void_p()
        assert lib.ltne_batch_create(arr, 2, None, C.byref(b)) == lt.LTNE_ERR_INVALID_ARG, kw
    arr = (lt.ltne_params * 2)(lt.ltne_default_params(32, 32), lt.ltne_default_params(64, 32))
    b = C.c_void_p()
    assert lib.ltne_batch_create(arr, 2, None, C.byref(b)) == lt.LTNE_OK
    assert lt.ltne_batch_nodes(b) == 32 * 32 + 64 * 32
    assert lt.ltne_batch_workspace_bytes(b) > 2 * 19 * 4 * (32 * 32 + 64 * 32)
    # a schedule needs a bound workspace
    assert lib.ltne_batch_set_schedule(b, 64, 2, 0, 1) == lt.LTNE_ERR_STATE
    lt.ltne_batch_destroy(b)
    # the adjoint needs a bound workspace and rejects the local h_v model
    p = lt.ltne_default_params(32, 32, porosity_field=1, hv_local=1)
    h = lt.ltne_create(p)
    J, dH = C.c_double(), C.c_double()
    phi = (C.c_double * (32 * 32))(*([0.5] * (32 * 32)))
    assert lib.ltne_adjoint(h, phi, None, None, None, 10, 4, C.c_void_p(256), 1 << 20, None,
                            C.byref(J), C.byref(dH)) == lt.LTNE_ERR_STATE
    assert lt.ltne_adjoint_workspace_bytes(h, 100, 10) > 0
    assert lt.ltne_adjoint_workspace_bytes(h, 0, 10) == 0
    # adjoint register budget: by size by default, either build on request
    assert lt.ltne_get_adjoint_schedule(h) == lt.LTNE_ADJ_AUTO
    for bad in (-1, 3):
        assert lib.ltne_set_adjoint_schedule(h, bad) == lt.LTNE_ERR_INVALID_ARG
    for mode in (lt.LTNE_ADJ_CAPPED, lt.LTNE_ADJ_ONE_WAVE, lt.LTNE_ADJ_AUTO):
        assert lib.ltne_set_adjoint_schedule(h, mode) == lt.LTNE_OK
        assert lt.ltne_get_adjoint_schedule(h) == mode
    lt.ltne_destroy(h)
    # step schedules: default per storage type; two nodes per thread need
    # float arithmetic and at most 128 threads per block
    for storage, default, side in ((lt.LTNE_F32, (128, 1, 2), 2048),
                                   (lt.LTNE_F16DEV, (32, 4, 2), 1024),
                                   (lt.LTNE_BF16DEV, (32, 4, 2), 1024),
                                   (lt.LTNE_F64, (64, 2, 1), 1024)):
        # the large-lattice default from side^2 nodes (2^22 FP32, 2^20 16-bit)
        h = lt.ltne_create(lt.ltne_default_params(side, side, storage=storage))
        assert lt.ltne_get_schedule(h) == default
        lt.ltne_destroy(h)
        h = lt.ltne_create(lt.ltne_default_params(side, side - 1, storage=storage))
        assert lt.ltne_get_schedule(h) == (64, 2, 1)
        lt.ltne_destroy(h)
        h = lt.ltne_create(lt.ltne_default_params(32, 32, storage=storage))
        assert lt.ltne_get_schedule(h) == (64, 2, 1)
        for bad in ((48, 2, 1), (16, 1, 1), (512, 1, 1), (128, 4, 1), (128, 2, 3), (128, 0, 1),
                    (64, 4, 2), (256, 1, 2)):
            assert lib.ltne_set_schedule(h, *bad) == lt.LTNE_ERR_INVALID_ARG, bad
        assert lib.ltne_set_schedule(h, 64, 2, 2) == (
            lt.LTNE_ERR_INVALID_ARG if storage == lt.LTNE_F64 else lt.LTNE_OK)
        assert lib.ltne_set_schedule(h, 256, 1, 1) == lt.LTNE_OK
        assert lt.ltne_get_schedule(h) == (256, 1, 1)
        # staged tiles: float arithmetic and cavity walls only
        assert lib.ltne_set_staging(h, 2) == lt.LTNE_ERR_INVALID_ARG
        assert lib.ltne_set_staging(h, 1) == (
            lt.LTNE_ERR_INVALID_ARG if storage == lt.LTNE_F64 else lt.LTNE_OK)
        assert lt.ltne_get_staging(h) == (0 if storage == lt.LTNE_F64 else 1)
        lt.ltne_destroy(h)
        h = lt.ltne_create(lt.ltne_default_params(32, 32, storage=storage,
                                                  bc=lt.LTNE_BC_PERIODIC))
        assert lib.ltne_set_staging(h, 1) == lt.LTNE_ERR_INVALID_ARG
        assert lt.ltne_slab_scratch_bytes(h, 2) == 0  # slabs: cavity walls only
        lt.ltne_destroy(h)
        # slabs: FP32 / FP64 cavities, at least two rows per slab
        h = lt.ltne_create(lt.ltne_default_params(32, 20, storage=storage))
        supported = storage in (lt.LTNE_F32, lt.LTNE_F64)
        assert (lt.ltne_slab_scratch_bytes(h, 4) > 0) == supported
        assert lt.ltne_slab_scratch_bytes(h, 11) == 0
        assert lib.ltne_step_slabs(h, 2, 1, None, 0) in (
            lt.LTNE_ERR_STATE if supported else lt.LTNE_ERR_INVALID_ARG,)
        lt.ltne_destroy(h)


def _ergun_diameter_in_the_documented_order(phi, L, Da):
    """The Ergun mean's summation order as include/ltne.h and the library
    state it, restated with Python floats (IEEE doubles): chunks of 2048
    values, 32 lane sums per chunk (lane l takes values l, l + 32, ... in
    order), the lane sums combined by strides 16, 8, 4, 2, 1, the chunk
    sums added in order."""
    import math

    n = phi.size
    chunks = []
    for c in range((n + 2047) // 2048):
        v = []
        for lane in range(32):
            s = 0.0
            for j in range(64):
                i = c * 2048 + 32 * j + lane
                if i < n:
                    ph = float(phi[i])
                    s += ph * ph * ph / ((1.0 - ph) * (1.0 - ph))
            v.append(s)
        st = 16
        while st >= 1:
            for lane in range(st):
                v[lane] = v[lane] + v[lane + st]
            st //= 2
        chunks.append(v[0])
    acc = 0.0
    for x in chunks:
        acc += x
    return L * math.sqrt(150.0 * Da / (acc / n))


def test_ergun_diameter_follows_its_documented_order():
    """ltne_ergun_diameter (host code, no device) gives the bits of the
    documented summation order -- the order the device's porosity kernel
    also takes -- and the oracle's diameter to rounding."""
    from oracle import ergun_diameter
    from paper_1608_04118_gb300 import ltne as lt
    from paper_1608_04118_gb300 import workloads as W

    for nx, ny, seed in ((100, 50, 3), (64, 32, 4), (7, 5, 5)):
        phi = W.porosity_field(nx, ny, 0.3, 0.9, seed).reshape(-1)
        d = lt.ltne_ergun_diameter(phi, ny - 1, 1e-3)
        assert d == _ergun_diameter_in_the_documented_order(phi, ny - 1, 1e-3), (nx, ny)
        assert d == pytest.approx(ergun_diameter(phi, ny - 1, 1e-3), rel=1e-14)
    bad = W.porosity_field(10, 10, 0.3, 0.9, 6).reshape(-1)
    bad[57] = 1.0
    with pytest.raises(lt.LtneError):
        lt.ltne_ergun_diameter(bad, 9, 1e-3)

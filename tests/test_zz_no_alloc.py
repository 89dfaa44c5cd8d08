"""The allocation-free observables entry point.

ltne_observables_static() reduces fields that the caller already holds on
the device, with its scratch in a fixed device array inside the library, so
callers that cannot allocate device memory at that point (a plug-in whose
host application owns every allocation, a thread without access to the
allocator, a loop that must not allocate) can still get the observables.  It must agree with ltne_observables(), which
uses the handle's workspace, and keep agreeing on later calls that reuse the
same scratch.  This file is collected last so that a failure here comes after
every other test has run.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

KEYS = ("Nu_f_hot", "Nu_s_hot", "Nu_f_cold", "Nu_s_cold", "mass", "energy", "max_u", "max_dT",
        "mean_Tf", "mean_Ts", "Fo")


def _entry(L):
    fn = L.load().ltne_observables_static
    fn.restype = C.c_int
    fn.argtypes = [C.POINTER(L.ltne_params), C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                   C.c_void_p, C.POINTER(L.ltne_obs)]
    return fn


def test_static_observables_match_workspace_observables():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_04118_gb300 import build

    build.build()
    from paper_1608_04118_gb300 import ltne as L
    from paper_1608_04118_gb300 import workloads as W

    fn = _entry(L)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    nx, ny = 300, 130
    phi = W.porosity_field(nx, ny, 0.3, 0.9, seed=41)
    cfg = dict(Ra=1e5, Da=1e-3, H=50.0, gamma_sf=5.0, sigma=1.3, T_hot=1.0, T_cold=0.0,
               T_ref=0.5)
    cav = L.Cavity(nx, ny, storage="f32", permeability=L.LTNE_K_ERGUN, porosity_field=1, **cfg)
    cav.set_fields(porosity=phi.reshape(-1))
    por = torch.from_numpy(phi.astype(np.float32)).to(dev)
    for call, steps in enumerate((400, 250)):
        cav.step(steps)
        ref = cav.observables()
        f = cav.fields()
        # the caller's own copy of the fields: five planes of deviations
        # (rho - 1, ux, uy, T_f - T0, T_s - T0) with row pitch nx
        planes = np.stack([f["rho"] - 1.0, f["ux"], f["uy"], f["Tf"] - 0.5, f["Ts"] - 0.5])
        fields = torch.from_numpy(planes.astype(np.float32)).to(dev).contiguous()
        torch.cuda.synchronize()
        out = L.ltne_obs()
        rc = fn(C.byref(cav.params), C.c_void_p(fields.data_ptr()), nx,
                C.c_void_p(por.data_ptr()), ref["step"], C.c_void_p(stream.cuda_stream),
                C.byref(out))
        assert rc == L.LTNE_OK, L.ltne_error_string(rc)
        got = out.as_dict()
        for k in KEYS:
            assert got[k] == pytest.approx(ref[k], rel=1e-12, abs=1e-14), (call, k)
        assert got["step"] == ref["step"] and got["nonfinite"] == 0
        assert np.isnan(got["residual"])  # no snapshot is kept by this variant


def test_static_observables_rejects_lattices_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_04118_gb300 import ltne as L

    fn = _entry(L)
    out = L.ltne_obs()
    # 8448 x 8192 passes every parameter check (its 19 population planes
    # stay below 2^32 elements) but needs 33 x 128 = 4224 pass-1 blocks, more
    # than the 4096 partial vectors of the fixed array; 8192 x 8192 (4096
    # blocks) is the largest square served.  Rejected before any device
    # work: the pointer is never dereferenced.
    for nx, ny in ((8448, 8192), (8192, 8256), (16384, 16384)):
        p = L.ltne_default_params(nx, ny)
        rc = fn(C.byref(p), C.c_void_p(256), nx, None, 0, None, C.byref(out))
        assert rc == L.LTNE_ERR_INVALID_ARG, (nx, ny)

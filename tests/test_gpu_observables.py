"""The FP64 observables against an FP64 accumulation of the same FP32 fields.

ltne_observables() reduces the fields of the current state: each thread of
the reduction sums at most 64 nodes' terms in FP32 and everything above is
FP64; the wall-flux integrals of Nu are FP64 from the first add.  Here the
fields the device holds are read back (exact in FP64) and the wall Nusselt
numbers, mass, energy and residual are summed again on the host with
correctly rounded sums.  The bounds follow from the FP32 chains: at most 64
additions of terms of one sign class each rounded to half an FP32 ulp, the
chains' errors independent, so the relative error of a sum of N terms is
about 2^-24 sqrt(64 / N) -- 1e-11 to 1e-10 at these sizes (mass and energy
are asserted at 1e-11 and 1e-9), against about 2^-24 sqrt(2048) ~ 3e-6 per
partial when a whole warp's 32 x 64 nodes were summed in FP32."""
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


def host_observables(f, phi32, cfg):
    """Nu (trapezoid of the second-order wall stencil), mass and energy of
    one field set, summed in FP64 (math.fsum: correctly rounded)."""
    import math

    Th, Tc, T0, sigma = cfg["T_hot"], cfg["T_cold"], cfg["T_ref"], cfg["sigma"]
    ny = f["Tf"].shape[0]
    w = np.ones(ny)
    w[0] = w[-1] = 0.5
    dT = Th - Tc
    out = {}
    for ph, key in (("f", "Tf"), ("s", "Ts")):
        T = f[key]
        qh = 1.5 * Th - 2.0 * T[:, 1] + 0.5 * T[:, 2]
        qc = -1.5 * Tc + 2.0 * T[:, -2] - 0.5 * T[:, -3]
        out["Nu_%s_hot" % ph] = math.fsum(w * qh) / dT
        out["Nu_%s_cold" % ph] = math.fsum(w * qc) / dT
    out["mass"] = math.fsum(f["rho"].ravel())
    e = phi32 * f["Tf"] + (1.0 - phi32) * sigma * f["Ts"]
    out["energy"] = math.fsum(e.ravel())
    return out


def host_residual(a, b):
    """max over u, T_f, T_s of ||X_b - X_a|| / ||X_b|| in FP64."""
    import math

    def rel(d2, x2):
        return math.sqrt(math.fsum(d2.ravel()) / math.fsum(x2.ravel()))

    du2 = (b["ux"] - a["ux"]) ** 2 + (b["uy"] - a["uy"]) ** 2
    r = rel(du2, b["ux"] ** 2 + b["uy"] ** 2)
    for k in ("Tf", "Ts"):
        r = max(r, rel((b[k] - a[k]) ** 2, b[k] ** 2))
    return r


@pytest.mark.parametrize("n,per_node", [(8192, False), (2048, True)])
def test_observables_agree_with_fp64_sums_of_the_same_fields(n, per_node):
    """8192 x 8192 (the reduced-storage configuration's physics, uniform
    porosity) and 2048 x 2048 (the throughput configuration's, porosity per
    node), FP32 storage with the default schedules, from random fields; and
    the same state restored from a checkpoint into a second handle."""
    if per_node:
        cfg = dict(W.C2_THROUGHPUT, nx=n, ny=n)
        phi = W.porosity_field(n, n, cfg["phi_lo"], cfg["phi_hi"], cfg["seed"])
        phi32 = phi.astype(np.float32).astype(np.float64)
        kw = dict(phi=phi.reshape(-1))
    else:
        cfg = dict(W.C5_REDUCED, nx=n, ny=n)
        phi = None
        phi32 = float(np.float32(cfg["porosity"]))
        kw = {}
    fields = W.random_fields(n, n, 61)
    c = cavity_for(cfg, storage="f32", **kw)
    c.set_fields(porosity=None if phi is None else phi.reshape(-1), **fields).step(30)
    ob1 = c.observables()
    f1 = c.fields()
    c.step(7)
    ob2 = c.observables()
    f2 = c.fields()
    blob = c.get_state()
    c.close()
    torch.cuda.empty_cache()
    ref1 = host_observables(f1, phi32, cfg)
    ref2 = host_observables(f2, phi32, cfg)
    for ob, ref in ((ob1, ref1), (ob2, ref2)):
        for k in ("Nu_f_hot", "Nu_s_hot", "Nu_f_cold", "Nu_s_cold"):
            assert ob[k] == pytest.approx(ref[k], rel=1e-11), (k, ob[k], ref[k])
        assert ob["mass"] == pytest.approx(ref["mass"], rel=1e-11)
        assert ob["energy"] == pytest.approx(ref["energy"], rel=1e-9)
    assert np.isnan(ob1["residual"])
    assert ob2["residual"] == pytest.approx(host_residual(f1, f2), rel=1e-6)
    # the same state through the stand-alone reduction pass
    d = cavity_for(cfg, storage="f32", **kw).set_state(blob)
    ob3 = d.observables()
    d.close()
    for k in ("Nu_f_hot", "Nu_s_hot", "Nu_f_cold", "Nu_s_cold", "mass", "energy", "mean_Tf",
              "mean_Ts"):
        assert ob3[k] == pytest.approx(ob2[k], rel=1e-12), k
    assert ob3["max_u"] == ob2["max_u"] and ob3["max_dT"] == ob2["max_dT"]


def test_repeated_observables_and_residual_reference():
    """A second call with no step between gives residual 0 and the same
    sums; after steps the residual is taken against the previous call."""
    cfg = W.random_params(62, 130, 70)
    c = cavity_for(cfg, storage="f32").set_fields(**W.random_fields(130, 70, 63)).step(20)
    a = c.observables()
    b = c.observables()
    assert np.isnan(a["residual"]) and b["residual"] == 0.0
    for k in ("Nu_f_hot", "mass", "energy", "max_u"):
        assert b[k] == pytest.approx(a[k], rel=1e-13)
    f1 = c.fields()
    c.step(5).step(6)  # two calls: the snapshot stays the one of the last observables
    f2 = c.fields()
    r = c.observables()["residual"]
    assert r == pytest.approx(host_residual(f1, f2), rel=1e-6)

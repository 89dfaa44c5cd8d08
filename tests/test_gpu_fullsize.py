"""Parity at the benchmark sizes, on sampled outputs.

The CUDA path runs the whole lattice (4096 x 4096 FP32 with per-node
porosity, 8192 x 8192 with 16-bit storage) in the launch configuration the
benchmark times.  The oracle recomputes windows of it: after k steps a
node's value depends only on nodes within 2k + 2 of it, so a window of the
cavity run by the oracle (the real walls where the window touches them,
fake walls or periodic wrap elsewhere, and the full cavity's length scale)
reproduces every node farther than that from its fake edges.
"""
import numpy as np
import pytest

from paper_1608_04118_gb300 import workloads as W
from tests.helpers import cavity_for, field_errors, phys, rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _windows(n, wn, margin):
    """(x0, y0, bc, (ys, xs) check slices in window coordinates)."""
    lo, hi = slice(0, wn - margin), slice(margin, wn)
    mid = slice(margin, wn - margin)
    return [
        (0, 0, 0, (lo, lo)),                          # hot wall, bottom wall, corner
        (n - wn, n - wn, 0, (hi, hi)),                # cold wall, top wall, corner
        (0, n // 2 - wn // 2, 0, (mid, lo)),          # hot wall, middle height
        (n // 2 - wn // 2, 0, 0, (lo, mid)),          # bottom wall, middle
        (n // 3, (2 * n) // 3, 1, (mid, mid)),        # interior (periodic window)
    ]


def _check(cfg, storage, n, k, seed, tol, deviations=True):
    """Run the n x n cavity on the GPU for k steps from random fields and
    compare five windows with the oracle.  deviations=True measures T - T_0
    and rho - 1 (stricter than the full values); False measures u, T_f and
    T_s as they are, the quantities the accuracy targets name."""
    from oracle import Oracle, OracleParams, ergun_diameter

    phi = None
    cfg = dict(cfg, nx=n, ny=n)
    cfg_orc = cfg
    if cfg.get("ergun"):
        phi = W.porosity_field(n, n, cfg["phi_lo"], cfg["phi_hi"], cfg["seed"])
        # the CUDA path derives the Ergun diameter from the whole field
        # itself; the oracle's windows see only part of it and are given it
        cfg_orc = dict(cfg, d_p=ergun_diameter(phi, n - 1, cfg["Da"]))
    fields = W.random_fields(n, n, seed)
    cav = cavity_for(cfg, storage=storage, phi=None if phi is None else phi.reshape(-1))
    cav.set_fields(porosity=None if phi is None else phi.reshape(-1), **fields)
    cav.step(k)
    got = cav.fields()
    assert cav.observables()["nonfinite"] == 0
    cav.close()
    del cav
    torch.cuda.empty_cache()

    wn, margin = 2 * k + 112, 2 * k + 4
    errs = []
    for x0, y0, bc, (ys, xs) in _windows(n, wn, margin):
        sl = (slice(y0, y0 + wn), slice(x0, x0 + wn))
        sub = {k2: v.reshape(n, n)[sl].reshape(-1) for k2, v in fields.items()}
        p = OracleParams.make(wn, wn, bc=bc, ergun_K=int(bool(cfg.get("ergun"))), L_ref=n - 1.0,
                              **phys(cfg_orc))
        o = Oracle(p, phi=None if phi is None else phi[sl].reshape(-1))
        o.init(rho=sub["rho"], ux=sub["ux"], uy=sub["uy"], Tf=sub["T_f"], Ts=sub["T_s"]).step(k)
        ref = o.macros()
        g = {k2: v[sl] for k2, v in got.items()}
        T0, r0 = (0.5, 1.0) if deviations else (0.0, None)
        e = dict(
            u=rel_l2(np.stack([g["ux"][ys, xs], g["uy"][ys, xs]]),
                     np.stack([ref["ux"][ys, xs], ref["uy"][ys, xs]])),
            Tf=rel_l2(g["Tf"][ys, xs] - T0, ref["Tf"][ys, xs] - T0),
            Ts=rel_l2(g["Ts"][ys, xs] - T0, ref["Ts"][ys, xs] - T0))
        if r0 is not None:
            e["rho"] = rel_l2(g["rho"][ys, xs] - r0, ref["rho"][ys, xs] - r0)
        errs.append(e)
        for key, v in e.items():
            assert v <= tol, (storage, (x0, y0), key, e)
    return errs


def test_c2_fp32_4096_sampled_windows():
    """4096 x 4096, FP32, per-node porosity U[0.3, 0.9] with the Ergun
    medium, the particle diameter derived by the CUDA path from the whole
    field: five windows (both isothermal walls, both adiabatic walls, all
    four corners' neighbourhoods and the interior) after 40 steps.  Errors
    are measured on the deviations (T - T_0, rho - 1), which is stricter than
    on the full values."""
    _check(W.C2_THROUGHPUT, "f32", 4096, 40, seed=31, tol=1e-5)


BF16_FLOOR = ("BF16 deviations from the rest equilibrium cannot reach 1e-3 in u: one "
              "stochastic rounding of the exact state already puts 1.2e-3 into j/rho")


@pytest.mark.parametrize("storage", [
    "f16", pytest.param("bf16", marks=pytest.mark.xfail(strict=True, reason=BF16_FLOOR))])
def test_c5_reduced_8192_sampled_windows(storage):
    """8192 x 8192 with FP16 / BF16 deviation storage and FP32 arithmetic,
    cavity physics of the reduced-storage configuration (Ra 1e6, H 1000):
    rel-L2 of u, T_f and T_s within the reduced-storage target 1e-3."""
    _check(W.C5_REDUCED, storage, 8192, 24, seed=32, tol=1e-3, deviations=False)


_C2_LONG = {}


def _c2_long_reference(n, steps):
    """The oracle's run of the throughput cavity's physics (porosity
    U[0.3, 0.9] seed 2, Ergun medium with the diameter from the mean Da,
    Ra 1e6, H 100, gamma_sf 10) from rest; both sides derive the diameter
    from the field on their own."""
    key = (n, steps)
    if key not in _C2_LONG:
        from oracle import Oracle, OracleParams

        c = W.C2_THROUGHPUT
        phi = W.porosity_field(n, n, c["phi_lo"], c["phi_hi"], c["seed"]).reshape(-1)
        p = OracleParams.make(n, n, ergun_K=1, **phys(c))
        o = Oracle(p, phi=phi).init().step(steps)
        _C2_LONG[key] = (phi, o.macros(), o.observables())
    return _C2_LONG[key]


@pytest.mark.parametrize("n,steps,schedule", [(1024, 2500, (64, 2, 1)), (1024, 2500, (128, 1, 2)),
                                               (512, 10_000, (64, 2, 1))])
def test_c2_physics_full_field_long_run(n, steps, schedule):
    """The throughput configuration's own physics from rest, full fields
    against the oracle: rel-L2 of u, T_f and T_s within 1e-5 and the four
    wall Nusselt numbers within 1e-4.  At 1024 x 1024 for 2500 steps with one
    node per thread (the default at this size) and with two nodes per thread
    in 128 x 1 blocks (the 4096 x 4096 default); at 512 x 512 for the 10^4
    steps the FP32 target is stated for."""
    phi, ref, ob_ref = _c2_long_reference(n, steps)
    cfg = dict(W.C2_THROUGHPUT, nx=n, ny=n)
    cav = cavity_for(cfg, storage="f32", phi=phi).set_schedule(*schedule)
    cav.set_fields(porosity=phi).step(steps)
    got, ob = cav.fields(), cav.observables()
    cav.close()
    err = field_errors(got, ref)
    for k in ("u", "Tf", "Ts"):
        assert err[k] <= 1e-5, (k, err)
    for k in ("Nu_f_hot", "Nu_s_hot", "Nu_f_cold", "Nu_s_cold"):
        assert ob[k] == pytest.approx(ob_ref[k], rel=1e-4), (k, ob[k], ob_ref[k])
    assert ob["mass"] == pytest.approx(ob_ref["mass"], rel=1e-6)
    assert ob["max_u"] > 1e-4  # the flow has started (1024^2: max |u| 3.8e-4 after 2500 steps)

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
from tests.helpers import cavity_for, phys, rel_l2

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


def _check(cfg, storage, n, k, seed, tol):
    from oracle import Oracle, OracleParams, ergun_diameter

    phi = None
    if cfg.get("ergun"):
        phi = W.porosity_field(n, n, cfg["phi_lo"], cfg["phi_hi"], cfg["seed"])
        cfg = dict(cfg, d_p=ergun_diameter(phi, n - 1, cfg["Da"]))
    fields = W.random_fields(n, n, seed)
    cfg = dict(cfg, nx=n, ny=n)
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
                              **phys(cfg))
        o = Oracle(p, phi=None if phi is None else phi[sl].reshape(-1))
        o.init(rho=sub["rho"], ux=sub["ux"], uy=sub["uy"], Tf=sub["T_f"], Ts=sub["T_s"]).step(k)
        ref = o.macros()
        g = {k2: v[sl] for k2, v in got.items()}
        e = dict(
            u=rel_l2(np.stack([g["ux"][ys, xs], g["uy"][ys, xs]]),
                     np.stack([ref["ux"][ys, xs], ref["uy"][ys, xs]])),
            Tf=rel_l2(g["Tf"][ys, xs] - 0.5, ref["Tf"][ys, xs] - 0.5),
            Ts=rel_l2(g["Ts"][ys, xs] - 0.5, ref["Ts"][ys, xs] - 0.5),
            rho=rel_l2(g["rho"][ys, xs] - 1.0, ref["rho"][ys, xs] - 1.0))
        errs.append(e)
        for key, v in e.items():
            assert v <= tol, (storage, (x0, y0), key, e)
    return errs


def test_c2_fp32_4096_sampled_windows():
    """4096 x 4096, FP32, per-node porosity U[0.3, 0.9] with the Ergun
    medium: five windows (both isothermal walls, both adiabatic walls, all
    four corners' neighbourhoods and the interior) after 40 steps.  Errors
    are measured on the deviations (T - T_0, rho - 1), which is stricter than
    on the full values."""
    _check(W.C2_THROUGHPUT, "f32", 4096, 40, seed=31, tol=1e-5)


@pytest.mark.parametrize("storage,tol", [("f16", 2e-3), ("bf16", 2e-2)])
def test_c5_reduced_8192_sampled_windows(storage, tol):
    """8192 x 8192 with FP16 / BF16 deviation storage and FP32 arithmetic,
    cavity physics of the reduced-storage configuration (Ra 1e6, H 1000)."""
    _check(W.C5_REDUCED, storage, 8192, 24, seed=32, tol=tol)

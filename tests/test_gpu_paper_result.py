"""The paper's only printed result (Sec. 4): in the metallic-foam cavity
with the local heat transfer coefficient of Eq. 52 (phi = 0.8, F_phi =
0.068, Da = 1e-4, gamma_sf = 1000, sigma = 1, Pr = 1, J_e = 1, T_h = 11,
T_c = T_0 = 1), the steady solid-to-fluid temperature difference at
mid-height grows with Ra, and at Ra = 1e9 (192 x 192) its maximum is about
10 %.  Reproduced here with u_m = |u| of the previous state in Eq. 52."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PAPER = dict(Pr=1.0, Da=1e-4, porosity=0.8, gamma_sf=1000.0, sigma=1.0, J_e=1.0, T_hot=11.0,
             T_cold=1.0, T_ref=1.0, F_phi=0.068, hv_local=1, Dp_over_L=0.0135)


def _steady_dtheta(Ra, n, steps):
    from paper_1608_04118_gb300.ltne import Cavity

    c = Cavity(n, n, storage="f32", Ra=Ra, **PAPER).set_fields().step(steps)
    ob = c.observables()
    c.step(2000)
    ob = c.observables()
    assert ob["nonfinite"] == 0
    assert ob["residual"] < 1e-4  # steady (FP32 round-off floor)
    f = c.fields()
    y0, y1 = (n - 1) // 2, n // 2  # mid-height, between the two middle rows for even n
    dtheta = 0.5 * ((f["Ts"][y0] - f["Tf"][y0]) + (f["Ts"][y1] - f["Tf"][y1])) / 10.0
    return float(np.abs(dtheta).max())


def test_max_solid_fluid_difference_about_ten_percent_at_ra_1e9():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d6 = _steady_dtheta(1e6, 128, 150_000)
    d8 = _steady_dtheta(1e8, 192, 400_000)
    d9 = _steady_dtheta(1e9, 192, 700_000)
    assert d6 < d8 < d9
    assert 0.08 <= d9 <= 0.12, d9

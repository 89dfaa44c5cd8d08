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

from tests.helpers import golden

G = golden("sec4_parameters")
PAPER = dict({k: G[k] for k in ("Pr", "Da", "porosity", "gamma_sf", "sigma", "J_e", "T_hot",
                                "T_cold", "T_ref", "F_phi", "Dp_over_L")}, hv_local=1)
RESULT = golden("sec4_max_dtheta")


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
    dT = PAPER["T_hot"] - PAPER["T_cold"]
    dtheta = 0.5 * ((f["Ts"][y0] - f["Tf"][y0]) + (f["Ts"][y1] - f["Tf"][y1])) / dT
    return float(np.abs(dtheta).max())


def test_max_solid_fluid_difference_about_ten_percent_at_ra_1e9():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d6 = _steady_dtheta(1e6, 128, 150_000)
    d8 = _steady_dtheta(1e8, 192, 400_000)
    d9 = _steady_dtheta(RESULT["Ra"], int(RESULT["n"]), 700_000)
    assert d6 < d8 < d9
    assert RESULT["band_lo"] <= d9 <= RESULT["band_hi"], d9

"""Errors of the FP32 / FP16 / BF16 storage forms against the FP64 oracle as
a run from rest goes on: the reduced-storage physics (phi 0.6, Da 1e-2,
Ra 1e6, H 1000) on the down-sized 512^2 cavity after 250 to 10^4 steps, and
the 64^2 plain-method cavity (Ra 1e4, H 10) after 1000 to 10^4 steps.
Asserted: FP32 within 1e-5 (u, T_f, T_s) at every mark; FP16 within 1e-3 in
u, T_f and T_s at every mark and in the wall Nusselt numbers over the
configured 2000-step run; BF16 above 1e-3 in u at the end of each run (one
stochastic rounding of deviations from the rest equilibrium into 8
significand bits already puts about 1.2e-3 into u).  Run with
``LTNE_CURVE_JSON=<path>`` to write the whole table."""
import json
import os

import numpy as np
import pytest

from paper_1608_04118_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-3
PHYS = ("Ra", "Pr", "Da", "porosity", "H", "gamma_sf", "sigma", "T_hot", "T_cold", "T_ref")
RUNS = {
    "c5_512": (dict(W.C5_REDUCED, nx=512, ny=512), (250, 500, 1000, 2000, 4000, 10000)),
    "c1_64": (W.C1_PLAIN_64, (1000, 2500, 5000, 10000)),
}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_04118_gb300 import build

    build.build()


def _errors(got, gobs, ref, robs):
    un = np.linalg.norm(np.stack([ref["ux"], ref["uy"]]))
    e = {"u": float(np.linalg.norm(np.stack([got["ux"] - ref["ux"], got["uy"] - ref["uy"]])) / un)}
    for f in ("Tf", "Ts"):
        e[f] = float(np.linalg.norm(got[f] - ref[f]) / np.linalg.norm(ref[f]))
    e["Nu"] = max(float(abs(gobs[q] - robs[q]) / abs(robs[q]))
                  for q in ("Nu_f_hot", "Nu_s_hot", "Nu_f_cold", "Nu_s_cold"))
    return e


@pytest.fixture(scope="module")
def curve():
    from oracle import Oracle, OracleParams
    from paper_1608_04118_gb300.ltne import Cavity

    out = {}
    for name, (cfg, marks) in RUNS.items():
        phys = {k: cfg[k] for k in PHYS}
        m = cfg["nx"]
        o = Oracle(OracleParams.make(m, m, **phys)).init()
        cavs = {st: Cavity(m, m, storage=st, **phys).set_fields() for st in ("f32", "f16", "bf16")}
        done, rows = 0, []
        for k in marks:
            o.step(k - done)
            for cav in cavs.values():
                cav.step(k - done)
            done = k
            ref, robs = o.macros(), o.observables()
            row = {"steps": k}
            for st, cav in cavs.items():
                row[st] = _errors(cav.fields(), cav.observables(), ref, robs)
            rows.append(row)
        for cav in cavs.values():
            cav.close()
        out[name] = rows
    path = os.environ.get("LTNE_CURVE_JSON")
    if path:
        with open(path, "w") as fh:
            json.dump(out, fh, indent=1)
    return out


@pytest.mark.parametrize("name", sorted(RUNS))
def test_fp32_and_fp16_fields_within_the_targets(curve, name):
    for row in curve[name]:
        assert max(row["f32"][k] for k in ("u", "Tf", "Ts")) <= 1e-5, row
        assert max(row["f16"][k] for k in ("u", "Tf", "Ts")) <= TOL, row


def test_fp16_nusselt_within_the_target_over_the_configured_run(curve):
    for row in curve["c5_512"]:
        if row["steps"] <= W.C5_REDUCED["steps"]:
            assert row["f16"]["Nu"] <= TOL, row


@pytest.mark.parametrize("name", sorted(RUNS))
def test_bf16_velocity_above_the_target(curve, name):
    assert curve[name][-1]["bf16"]["u"] > TOL, curve[name]

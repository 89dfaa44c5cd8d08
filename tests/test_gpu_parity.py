"""Parity of the CUDA step (through the C ABI) with the FP64 oracle.

Tolerances: FP64 storage agrees with the oracle to rounding (rel-L2 of u,
T_f, T_s <= 1e-10 after 10^4 steps); FP32 storage within rel-L2 <= 1e-5
and Nusselt numbers within 1e-4 relative.
"""
import numpy as np
import pytest

from paper_1608_04118_gb300 import workloads as W
from tests.helpers import cavity_for, field_errors, oracle_for, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_04118_gb300 import build

    build.build()
    import oracle

    oracle.build()


TOL = {"f64": 1e-10, "f32": 1e-5}


def _init_kw_oracle(fields):
    if fields is None:
        return {}
    return dict(rho=fields["rho"], ux=fields["ux"], uy=fields["uy"], Tf=fields["T_f"],
                Ts=fields["T_s"])


def run_pair(cfg, steps, storage, phi=None, bc=0, fields=None):
    o = oracle_for(cfg, phi=phi, bc=bc).init(**_init_kw_oracle(fields)).step(steps)
    c = cavity_for(cfg, storage=storage, phi=phi, bc=bc)
    c.set_fields(porosity=phi, **(fields or {})).step(steps)
    return c, o


# The periodic box has no walls to hold the buoyant flow back: with seed 4's
# draw its flow accelerates past |u| = 0.2 and the method itself diverges
# (the oracle as much as the CUDA path), which compares nothing; seed 24
# keeps |u| below 0.01.
@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("shape,bc,seed", [((8, 8), 0, 1), ((16, 16), 0, 2), ((13, 11), 0, 3),
                                           ((9, 17), 1, 24), ((12, 10), 2, 5), ((5, 4), 0, 6)])
def test_brute_force_small(storage, shape, bc, seed):
    nx, ny = shape
    cfg = W.random_params(seed, nx, ny)
    fields = W.random_fields(nx, ny, seed + 100)
    c, o = run_pair(cfg, 200, storage, bc=bc, fields=fields)
    err = field_errors(c.fields(), o.macros())
    for k in ("u", "Tf", "Ts"):
        assert err[k] <= TOL[storage] * (1 if storage == "f64" else 2), (k, err)
    assert err["rho_abs"] <= (1e-12 if storage == "f64" else 1e-6), err


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_internal_generation_and_constant_forchheimer(storage):
    """Internal generation (Q_f, Q_s of Eqs. 30-31, 43-45), a constant
    Forchheimer coefficient and the Ergun permeability with a given particle
    diameter, from random initial fields."""
    cfg = dict(W.random_params(12, 23, 19), qf=2e-4, qs=-1e-4, F_phi=0.068, ergun=True, d_p=0.9)
    phi = W.porosity_field(23, 19, 0.35, 0.85, seed=13).reshape(-1)
    fields = W.random_fields(23, 19, 112)
    c, o = run_pair(cfg, 300, storage, phi=phi, fields=fields)
    err = field_errors(c.fields(), o.macros())
    for k in ("u", "Tf", "Ts"):
        assert err[k] <= TOL[storage] * (1 if storage == "f64" else 2), (k, err)
    if storage == "f64":
        ob, ref = c.observables(), o.observables()
        assert ob["energy"] == pytest.approx(ref["energy"], rel=1e-11)


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_multitile_ragged_per_node_porosity(storage):
    """300 x 70 spans several 128-wide tiles with a ragged tail; per-node
    porosity with the Ergun medium (Eq. 7) and d from the mean Da."""
    nx, ny = 300, 70
    cfg = dict(W.C2_THROUGHPUT, nx=nx, ny=ny, Ra=1e5)
    phi = W.porosity_field(nx, ny, 0.3, 0.9, seed=21)
    c, o = run_pair(cfg, 200, storage, phi=phi.reshape(-1))
    err = field_errors(c.fields(), o.macros())
    for k in ("u", "Tf", "Ts"):
        assert err[k] <= TOL[storage], (k, err)


def test_c1_cavity_full_run():
    """The 64 x 64 cavity (Ra 1e4, Da 1e-2, phi 0.6, H 10) for 10^4 steps."""
    cfg = W.C1_PLAIN_64
    o = oracle_for(cfg).init().step(cfg["steps"])
    ref, ob_ref = o.macros(), o.observables()
    for storage in ("f64", "f32"):
        c = cavity_for(cfg, storage=storage).set_fields().step(cfg["steps"])
        err = field_errors(c.fields(), ref)
        for k in ("u", "Tf", "Ts"):
            assert err[k] <= TOL[storage], (storage, k, err)
        ob = c.observables()
        for k in ("Nu_f_hot", "Nu_s_hot", "Nu_f_cold", "Nu_s_cold"):
            tol = 1e-10 if storage == "f64" else 1e-4
            assert ob[k] == pytest.approx(ob_ref[k], rel=tol), (storage, k)
        assert ob["mass"] == pytest.approx(ob_ref["mass"], rel=1e-12 if storage == "f64" else 1e-6)
        assert ob["energy"] == pytest.approx(ob_ref["energy"],
                                             rel=1e-12 if storage == "f64" else 1e-6)
        assert ob["step"] == cfg["steps"]
        assert ob["nonfinite"] == 0


def test_observables_match_oracle_fp64():
    cfg = dict(W.random_params(7, 33, 29))
    phi = W.porosity_field(33, 29, 0.4, 0.8, seed=8).reshape(-1)
    cfg["ergun"] = True
    c, o = run_pair(cfg, 500, "f64", phi=phi)
    ob, ref = c.observables(), o.observables()
    for k in ("Nu_f_hot", "Nu_s_hot", "Nu_f_cold", "Nu_s_cold", "mass", "energy", "max_u",
              "max_dT", "mean_Tf", "mean_Ts", "Fo"):
        assert ob[k] == pytest.approx(ref[k], rel=1e-10, abs=1e-14), k
    assert np.isnan(ob["residual"])
    c.step(10)
    ob2 = c.observables()
    assert 0 < ob2["residual"] < 1


def test_graph_replay_is_bitwise_equal_to_single_steps():
    cfg = W.random_params(9, 70, 40)
    a = cavity_for(cfg).set_fields()
    b = cavity_for(cfg).set_fields()
    a.step(100)  # graph replays + single launches
    for _ in range(100):
        b.step(1)
    fa, fb = a.fields(), b.fields()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k
    assert a.get_state()[64:] == b.get_state()[64:]
    assert a.launches == b.launches == 100


def test_handles_on_concurrent_host_threads():
    """Two lattices large enough for the host worker pool (set_fields with
    all fields given, steps, get_fields), driven from two host threads at
    once, give the bits of the same runs done one after the other: a pass
    that finds the pool busy runs on its own thread."""
    import threading

    nx, ny = 640, 600
    cfgs = [W.random_params(90 + k, nx, ny) for k in range(2)]
    fields = [W.random_fields(nx, ny, 190 + k) for k in range(2)]
    phis = [W.porosity_field(nx, ny, 0.4, 0.9, seed=290 + k).reshape(-1) for k in range(2)]

    def run(k, out):
        torch.cuda.set_device(0)
        c = cavity_for(cfgs[k], storage="f32", phi=phis[k])
        for _ in range(3):
            c.set_fields(porosity=phis[k], **fields[k]).step(40)
            out[k] = c.fields()
        c.close()

    seq, par = {}, {}
    for k in range(2):
        run(k, seq)
    ts = [threading.Thread(target=run, args=(k, par)) for k in range(2)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    for k in range(2):
        for f in seq[k]:
            assert np.array_equal(seq[k][f], par[k][f]), (k, f)


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16"])
def test_checkpoint_resume_bitwise(storage):
    cfg = W.random_params(10, 48, 40)
    a = cavity_for(cfg, storage=storage).set_fields().step(150)
    blob = a.get_state()
    a.step(150)
    b = cavity_for(cfg, storage=storage).set_state(blob).step(150)
    fa, fb = a.fields(), b.fields()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), (storage, k)
    assert b.observables()["step"] == 300


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_unpadded_lattice_state_is_deterministic(storage):
    """A lattice without row or plane padding (128 x 64) is zeroed only in
    the macro set its fields are staged into: two runs from scratch give the
    same state blobs, and a run resumed from a checkpoint the same fields."""
    cfg = W.random_params(17, 128, 64)
    fields = W.random_fields(128, 64, 117)
    a = cavity_for(cfg, storage=storage).set_fields(T_f=fields["T_f"]).step(60)
    b = cavity_for(cfg, storage=storage).set_fields(T_f=fields["T_f"]).step(60)
    blob = a.get_state()
    assert blob[64:] == b.get_state()[64:]
    a.step(40)
    c = cavity_for(cfg, storage=storage).set_state(blob).step(40)
    fa, fc = a.fields(), c.fields()
    for k in fa:
        assert np.array_equal(fa[k], fc[k]), (storage, k)
    o = oracle_for(cfg).init(Tf=fields["T_f"]).step(100)
    err = field_errors(fa, o.macros())
    assert err["Tf"] <= (2e-5 if storage == "f32" else 1e-3), err


def test_nonfinite_is_reported():
    """A NaN planted in a checkpoint on the host surfaces as the non-finite
    status of the observables (no device fault involved)."""
    cfg = W.random_params(11, 32, 32)
    a = cavity_for(cfg).set_fields().step(5)
    blob = bytearray(a.get_state())
    # first f_0 value of node (5, 5): header 64 bytes, plane 0, pitch 64 floats
    off = 64 + 4 * (5 * 64 + 5)
    blob[off:off + 4] = np.array([np.nan], dtype=np.float32).tobytes()
    a.set_state(bytes(blob)).step(3)
    from paper_1608_04118_gb300.ltne import LtneError, LTNE_ERR_NONFINITE

    with pytest.raises(LtneError) as ei:
        a.observables()
    assert ei.value.code == LTNE_ERR_NONFINITE
    assert a.observables(allow_nonfinite=True)["nonfinite"] > 0


# The reduced-storage target is rel-L2 <= 1e-3 for u, T_f and T_s; it is
# applied to the wall Nusselt numbers too.  BF16 cannot meet it with
# deviations from the rest equilibrium: a single stochastic rounding of the
# exact state already carries 1.2e-3 into j/rho (tests/test_storage_floor.py),
# so its cases assert the target and are expected to fail.
BF16_FLOOR = ("BF16 deviations from the rest equilibrium cannot reach 1e-3 in u: one "
              "stochastic rounding of the exact state already puts 1.2e-3 into j/rho")
RED = pytest.mark.xfail(strict=True, reason=BF16_FLOOR)


@pytest.mark.parametrize("storage", ["f16", pytest.param("bf16", marks=RED)])
def test_reduced_storage_64_cavity_10k_steps(storage):
    """FP16 / BF16 deviation storage (stochastic rounding) with FP32
    arithmetic on the 64 x 64 cavity after 10^4 steps, against the oracle."""
    cfg = W.C1_PLAIN_64
    o = oracle_for(cfg).init().step(cfg["steps"])
    c = cavity_for(cfg, storage=storage).set_fields().step(cfg["steps"])
    err = field_errors(c.fields(), o.macros())
    for k in ("u", "Tf", "Ts"):
        assert err[k] <= 1e-3, (storage, k, err)


@pytest.mark.parametrize("schedule", [(128, 2, 1), (32, 4, 2)])
@pytest.mark.parametrize("storage,tol_u,tol_T,tol_nu", [
    ("f32", 1e-5, 1e-5, 1e-4), ("f16", 1e-3, 1e-3, 1e-3),
    pytest.param("bf16", 1e-3, 1e-3, 1e-3, marks=RED)])
def test_reduced_storage_512_parity_run(storage, tol_u, tol_T, tol_nu, schedule):
    """Physics of the reduced-storage configuration (Ra 1e6, H 1000, phi 0.6,
    Da 1e-2) on the down-sized 512 x 512 cavity for 2000 steps: per-field
    relative L2 errors against the FP64 oracle."""
    cfg = dict(W.C5_REDUCED, nx=W.C5_REDUCED["parity_n"], ny=W.C5_REDUCED["parity_n"])
    ref = _c5_oracle(cfg)
    c = cavity_for(cfg, storage=storage).set_schedule(*schedule).set_fields().step(cfg["steps"])
    err = field_errors(c.fields(), ref["fields"])
    assert err["u"] <= tol_u, err
    assert err["Tf"] <= tol_T and err["Ts"] <= tol_T, err
    ob = c.observables()
    for k in ("Nu_f_hot", "Nu_s_hot", "Nu_f_cold", "Nu_s_cold"):
        assert ob[k] == pytest.approx(ref["obs"][k], rel=tol_nu), (k, ob[k], ref["obs"][k])


_C5_CACHE = {}


def _c5_oracle(cfg):
    if "ref" not in _C5_CACHE:
        o = oracle_for(cfg).init().step(cfg["steps"])
        _C5_CACHE["ref"] = {"fields": o.macros(), "obs": o.observables()}
    return _C5_CACHE["ref"]


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_local_heat_transfer_coefficient_eq52(storage):
    """Per-node h_v from the correlation of Eq. 52 (H_p = 0.376 Re^0.644
    Pr^0.37, Re = u_m D_p / nu_f, D_p = 0.0135 L) with u_m the node's |u| in
    the previous state, from random initial fields (so the initial |u|
    matters), per-node porosity and the paper's validation parameters
    (phi around 0.8, F_phi 0.068, gamma_sf 1000, T_h 11, T_c = T_0 = 1)."""
    nx, ny = 41, 37
    cfg = dict(nx=nx, ny=ny, Ra=1e6, Pr=1.0, Da=1e-4, porosity=0.8, gamma_sf=1000.0, sigma=1.0,
               T_hot=11.0, T_cold=1.0, T_ref=1.0, F_phi=0.068, hv_local=1, Dp_over_L=0.0135,
               ergun=True)
    phi = W.porosity_field(nx, ny, 0.7, 0.9, seed=14).reshape(-1)
    fields = W.random_fields(nx, ny, 114, du=0.02, dT=0.3)
    fields["T_f"] = fields["T_f"] + 0.5
    fields["T_s"] = fields["T_s"] + 0.5
    c, o = run_pair(cfg, 400, storage, phi=phi, fields=fields)
    err = field_errors(c.fields(), o.macros())
    for k in ("u", "Tf", "Ts"):
        assert err[k] <= TOL[storage] * (1 if storage == "f64" else 3), (k, err)
    blob = c.get_state()
    c.step(50)
    d = cavity_for(cfg, storage=storage, phi=phi).set_state(blob).step(50)
    fa, fb = c.fields(), d.fields()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_thermal_correction_term(storage):
    """The correction term of Sec. 3.2 (off by default, as in the paper)
    switched on, in a convecting cavity with per-node porosity."""
    cfg = dict(W.random_params(15, 29, 27), thermal_correction=1, ergun=True)
    phi = W.porosity_field(29, 27, 0.4, 0.85, seed=16).reshape(-1)
    fields = W.random_fields(29, 27, 116)
    c, o = run_pair(cfg, 300, storage, phi=phi, fields=fields)
    err = field_errors(c.fields(), o.macros())
    for k in ("u", "Tf", "Ts"):
        assert err[k] <= TOL[storage] * (1 if storage == "f64" else 2), (k, err)

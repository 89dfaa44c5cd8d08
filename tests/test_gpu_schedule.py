"""Launch schedules of the step kernel: one node per thread, or two
neighbouring nodes per thread in paired FP32 arithmetic.

Both forms run the same per-node arithmetic, so each must match the FP64
oracle within the FP32 tolerance on its own, the two must agree with each
other to a few FP32 rounding steps, and the block shape must not change a
single bit (every node's result, and its stochastic-rounding stream in the
16-bit forms, depend only on the node and the step).  Odd widths leave a
one-node pair at the end of each row; cavity pairs that hold a left/right
wall node take the one-node path inside the pair kernel.
"""
import numpy as np
import pytest

from paper_1608_04118_gb300 import workloads as W
from tests.helpers import cavity_for, field_errors, oracle_for

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


def _run(cfg, steps, storage, schedule, phi=None, bc=0, fields=None):
    c = cavity_for(cfg, storage=storage, phi=phi, bc=bc).set_schedule(*schedule)
    c.set_fields(porosity=phi, **(fields or {})).step(steps)
    return c


def _oracle(cfg, steps, phi=None, bc=0, fields=None):
    kw = {}
    if fields is not None:
        kw = dict(rho=fields["rho"], ux=fields["ux"], uy=fields["uy"], Tf=fields["T_f"],
                  Ts=fields["T_s"])
    return oracle_for(cfg, phi=phi, bc=bc).init(**kw).step(steps)


@pytest.mark.parametrize("npt", [1, 2])
@pytest.mark.parametrize("shape,bc,seed", [((8, 8), 0, 11), ((13, 11), 0, 12), ((4, 6), 0, 13),
                                           ((9, 17), 1, 14), ((12, 10), 2, 15),
                                           ((15, 9), 2, 16), ((67, 45), 0, 17)])
def test_f32_schedules_match_oracle(npt, shape, bc, seed):
    nx, ny = shape
    cfg = W.random_params(seed, nx, ny)
    fields = W.random_fields(nx, ny, seed + 100)
    phi = W.porosity_field(nx, ny, 0.4, 0.9, seed=seed + 200).reshape(-1) if bc == 0 else None
    c = _run(cfg, 200, "f32", (64, 2, npt), phi=phi, bc=bc, fields=fields)
    o = _oracle(cfg, 200, phi=phi, bc=bc, fields=fields)
    err = field_errors(c.fields(), o.macros())
    for k in ("u", "Tf", "Ts"):
        assert err[k] <= 2e-5, (k, err)
    assert err["rho_abs"] <= 1e-6, err


def test_pair_and_one_node_forms_agree():
    """A 130 x 67 porous cavity with the local h_v model and the correction
    term, 600 steps: the two forms differ only by FP32 contraction order."""
    nx, ny = 130, 67
    cfg = dict(nx=nx, ny=ny, Ra=1e6, Pr=1.0, Da=1e-4, porosity=0.8, gamma_sf=1000.0, sigma=1.0,
               T_hot=11.0, T_cold=1.0, T_ref=1.0, F_phi=0.068, hv_local=1, Dp_over_L=0.0135,
               thermal_correction=1, ergun=True)
    phi = W.porosity_field(nx, ny, 0.7, 0.9, seed=21).reshape(-1)
    a = _run(cfg, 600, "f32", (128, 2, 1), phi=phi).fields()
    b = _run(cfg, 600, "f32", (64, 2, 2), phi=phi).fields()
    err = field_errors(a, b)
    for k in ("u", "Tf", "Ts"):
        assert err[k] <= 1e-6, (k, err)


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("npt", [1, 2])
def test_block_shape_changes_no_bit(storage, npt):
    nx, ny = 203, 77
    cfg = W.random_params(31, nx, ny)
    phi = W.porosity_field(nx, ny, 0.3, 0.9, seed=32).reshape(-1)
    ref = None
    shapes = (((128, 2), (32, 1), (64, 4), (256, 1), (32, 8)) if npt == 1 else
              ((32, 4), (32, 1), (64, 2), (128, 1), (32, 2)))
    for shape in shapes:
        f = _run(cfg, 150, storage, shape + (npt,), phi=phi).fields()
        if ref is None:
            ref = f
            continue
        for k in f:
            assert np.array_equal(f[k], ref[k]), (shape, k)


RED = pytest.mark.xfail(strict=True, reason="BF16 deviations from the rest equilibrium cannot "
                        "reach 1e-3 in u: one stochastic rounding of the exact state already "
                        "puts 1.2e-3 into j/rho")


@pytest.mark.parametrize("schedule", [(128, 2, 1), (32, 4, 2)])
@pytest.mark.parametrize("storage", ["f16", pytest.param("bf16", marks=RED)])
def test_reduced_storage_both_forms_64_cavity(storage, schedule):
    """The forms of the 16-bit kernels on the 64 x 64 cavity after 10^4
    steps against the oracle, at the reduced-storage target 1e-3."""
    cfg = W.C1_PLAIN_64
    o = oracle_for(cfg).init().step(cfg["steps"])
    c = cavity_for(cfg, storage=storage).set_schedule(*schedule).set_fields().step(cfg["steps"])
    err = field_errors(c.fields(), o.macros())
    for k in ("u", "Tf", "Ts"):
        assert err[k] <= 1e-3, (storage, k, err)


def test_schedule_change_between_steps_continues_the_run():
    """Changing the schedule mid-run drops the captured graphs and continues
    from the same state."""
    nx, ny = 96, 64
    cfg = W.random_params(41, nx, ny)
    a = cavity_for(cfg, storage="f32").set_schedule(128, 1, 2).set_fields().step(70)
    a.set_schedule(64, 2, 2).step(70)
    b = cavity_for(cfg, storage="f32").set_schedule(128, 1, 2).set_fields().step(140)
    fa, fb = a.fields(), b.fields()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k


@pytest.mark.parametrize("storage", ["f64", "f16"])
def test_autotuner_picks_a_valid_schedule(storage):
    from paper_1608_04118_gb300.autotune import cavity_candidates, tune_cavity

    nx, ny = 200, 96
    cfg = W.random_params(51, nx, ny)
    cav = cavity_for(cfg, storage=storage).set_fields()
    best, sec, table = tune_cavity(cav, steps=4, warmup=1)
    cands = list(cavity_candidates(storage))
    assert [t[0] for t in table] == cands and best in cands and sec > 0
    assert cav.schedule == best
    # the tuned schedule gives the same bits as a fresh run with it
    a = cav.set_fields().step(60).fields()
    b = cavity_for(cfg, storage=storage).set_schedule(*best).set_fields().step(60).fields()
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def _staged_pair(cfg, steps, storage, phi, staged):
    c = cavity_for(cfg, storage=storage, phi=phi).set_schedule(64, 2, 2)
    if staged:
        c.set_staging(1)
    return c.set_fields(porosity=phi).step(steps)


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_staged_tiles_give_the_same_bits(storage):
    """The two-node kernel fed from TMA-staged shared-memory tiles against
    the direct two-node kernel: the same bits, on a ragged cavity (odd width,
    partial tiles, walls), on one with more tiles than resident blocks (the
    persistent loop reuses both stages many times) and with the local h_v
    model and the correction term."""
    cases = [(203, 77, {}, 61), (1100, 300, {}, 62),
             (130, 67, dict(hv_local=1, Dp_over_L=0.0135, thermal_correction=1), 63)]
    for nx, ny, extra, seed in cases:
        cfg = dict(W.random_params(seed, nx, ny), **extra)
        phi = W.porosity_field(nx, ny, 0.4, 0.9, seed=seed + 1).reshape(-1)
        a = _staged_pair(cfg, 150, storage, phi, staged=False)
        b = _staged_pair(cfg, 150, storage, phi, staged=True)
        assert b.staging == 1
        fa, fb = a.fields(), b.fields()
        for k in fa:
            assert np.array_equal(fa[k], fb[k]), (nx, ny, k)
        assert b.observables()["nonfinite"] == 0


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    from paper_1608_04118_gb300.ltne import ltne_check_bounded_wait

    s = torch.cuda.current_stream()
    assert ltne_check_bounded_wait(s.cuda_stream, 5000) == 1
    cfg = W.random_params(71, 300, 40)
    c = cavity_for(cfg, storage="f16").set_staging(1).set_fields().step(40)
    assert c.observables()["step"] == 40

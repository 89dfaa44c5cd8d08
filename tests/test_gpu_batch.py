"""Batched form: many cavities of uneven size and parameters in one launch
per step.  Parity with the oracle cavity by cavity, independence of the
launch schedule, and agreement with the single-lattice path."""
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


def small_batch(count=12, seed=70):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        ny = int(rng.integers(6, 41))
        nx = ny * int(rng.choice([1, 2]))
        p = W.random_params(seed + i, nx, ny)
        out.append(p)
    return out


def _batch(cavs):
    from paper_1608_04118_gb300.ltne import Batch

    keys = ("nx", "ny", "Ra", "Pr", "Da", "porosity", "H", "gamma_sf", "sigma", "J_e", "T_hot",
            "T_cold", "T_ref", "Ma", "varpi") + W.RATE_KEYS
    return Batch([{k: c[k] for k in keys if k in c} for c in cavs])


def test_small_batch_matches_oracle_per_cavity():
    cavs = small_batch()
    b = _batch(cavs).set_fields().step(300)
    for i, c in enumerate(cavs):
        ref = oracle_for(c).init().step(300).macros()
        err = field_errors(b.fields(i), ref)
        for k in ("u", "Tf", "Ts"):
            assert err[k] <= 1e-5, (i, c["nx"], c["ny"], k, err)


@pytest.mark.parametrize("schedules", [
    ((128, 2, 0, 1), (32, 4, 3, 1), (64, 2, 152, 1), (256, 1, 1, 1)),
    ((64, 2, 0, 2), (128, 1, 5, 2), (256, 1, 152, 2), (64, 4, 1, 2))])
def test_schedule_does_not_change_results(schedules):
    """Tile shape and grid size change no bit for a fixed number of nodes per
    thread (one, or two in paired FP32 arithmetic)."""
    cavs = small_batch(8, seed=71)
    runs = []
    for sch in schedules:
        b = _batch(cavs).set_schedule(*sch).set_fields().step(77)
        runs.append([b.fields(i) for i in range(len(cavs))])
    for r in runs[1:]:
        for a, c in zip(runs[0], r):
            for k in a:
                assert np.array_equal(a[k], c[k]), k


@pytest.mark.parametrize("npt", [1, 2])
def test_batch_equals_single_lattice_path(npt):
    cavs = small_batch(6, seed=72)
    b = _batch(cavs).set_schedule(128 if npt == 1 else 64, 2, 0, npt).set_fields().step(120)
    obs = b.observables()
    for i, c in enumerate(cavs):
        s = cavity_for(c, storage="f32").set_schedule(128 if npt == 1 else 64, 2, npt)
        s = s.set_fields().step(120)
        fs, fb = s.fields(), b.fields(i)
        for k in fs:
            assert np.allclose(fb[k], fs[k], rtol=0, atol=1e-6 * max(1.0, np.abs(fs[k]).max())), k
        so = s.observables()
        for k in ("Nu_f_hot", "Nu_s_hot", "mass", "energy"):
            assert obs[i][k] == pytest.approx(so[k], rel=1e-6), (i, k)
        assert obs[i]["step"] == 120


def test_c3_workload_all_cavities_100_steps():
    """The 256-cavity workload (sides 64..512, aspect 1-2, log-uniform Ra, Da,
    H and conductivity ratio; seed 3) with the autotuned schedule: every
    cavity against the oracle after 100 steps."""
    cavs = W.batch_cavities(256, seed=3)
    b = _batch(cavs)
    from paper_1608_04118_gb300.autotune import tune_batch

    tune_batch(b, steps=2, warmup=1)
    b.set_fields().step(100)
    for i, c in enumerate(cavs):
        ref = oracle_for(c).init().step(100).macros()
        err = field_errors(b.fields(i), ref)
        for k in ("u", "Tf", "Ts"):
            assert err[k] <= 1e-5, (i, c["nx"], c["ny"], k, err)
    obs = b.observables()
    assert all(o["nonfinite"] == 0 for o in obs)


def test_c3_workload_eight_cavities_5000_steps():
    """Eight cavities of the workload (seeded choice among those of at most
    128 x 1024 nodes, which bounds the oracle's time) after the workload's
    full 5000 steps, run inside the whole 256-cavity batch."""
    cavs = W.batch_cavities(256, seed=3)
    b = _batch(cavs)
    b.set_fields().step(5000)
    small = [i for i, c in enumerate(cavs) if c["nx"] * c["ny"] <= 128 * 1024]
    pick = np.random.default_rng(33).choice(small, size=8, replace=False)
    for i in pick:
        c = cavs[int(i)]
        ref = oracle_for(c).init().step(5000).macros()
        err = field_errors(b.fields(int(i)), ref)
        for k in ("u", "Tf", "Ts"):
            assert err[k] <= 1e-5, (int(i), c["nx"], c["ny"], k, err)

"""Reverse-mode adjoint of the time step: gradients of
J = (Nu_f,hot + Nu_s,hot)/2 with respect to the per-node porosity and H.

Reference gradients: the oracle compiled for complex arithmetic gives
complex-step derivatives Im J(theta + i h e_k)/h, exact to round-off
(h = 1e-30); FP64 central differences of the forward step serve as a second
witness at the full 256 x 256 x 4000-step size.  The Ergun particle
diameter is held fixed in every variant (it is computed once from the
unperturbed field).
"""
import numpy as np
import pytest

from paper_1608_04118_gb300 import workloads as W
from tests.helpers import cavity_for, phys

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_04118_gb300 import build

    build.build()


# Every non-hydrodynamic rate distinct and varpi away from 2/5, so that a
# transposed rate on the wrong moment changes the gradient.
SMALL = dict(nx=20, ny=16, Ra=1e5, Pr=1.0, Da=1e-3, H=50.0, gamma_sf=3.0, sigma=1.2, T_hot=1.0,
             T_cold=0.0, T_ref=0.5, ergun=True, s_e=1.3, s_eps=0.9, s_q=1.7, zeta_e=1.5,
             zeta_nu=0.85, eta_e=1.25, eta_nu=1.6, varpi=0.55)


def _complex_step(cfg, phi, steps, nodes, h=1e-30):
    from oracle import ComplexOracle, OracleParams

    p = OracleParams.make(cfg["nx"], cfg["ny"], ergun_K=1, **phys(cfg))
    out = {}
    for k in list(nodes) + [-1]:
        o = ComplexOracle(p, phi=phi).perturb(int(k), h).init().step(steps)
        re, im = o.objective()
        out[int(k)] = im / h
        out["J"] = re
    return out


@pytest.fixture(scope="module")
def small_reference():
    phi = W.porosity_field(SMALL["nx"], SMALL["ny"], 0.4, 0.8, seed=44).reshape(-1)
    nodes = W.fd_nodes(SMALL["nx"], SMALL["ny"], 12, seed=45)
    ref = _complex_step(SMALL, phi, 120, nodes)
    return phi, nodes, ref


@pytest.mark.parametrize("storage,tol", [("f64", 1e-9), ("f32", 1e-3)])
def test_adjoint_matches_complex_step_oracle(small_reference, storage, tol):
    """120 steps in segments of 16 (the last one ragged)."""
    phi, nodes, ref = small_reference
    cav = cavity_for(SMALL, storage=storage, phi=phi)
    J, g, dH = cav.adjoint(phi, 120, segment=16)
    g = g.double().cpu().numpy().reshape(-1)
    assert J == pytest.approx(ref["J"], rel=1e-12 if storage == "f64" else 1e-5)
    gref = np.array([ref[int(k)] for k in nodes])
    scale = np.abs(gref).max()
    err = np.abs(g[nodes] - gref)
    assert err.max() <= tol * scale, (storage, err / scale)
    assert dH == pytest.approx(ref[-1], rel=tol, abs=tol * abs(ref[-1]))
    # the step counter and the fields are those of a plain run of 120 steps
    ob = cav.observables()
    assert ob["step"] == 120
    assert 0.5 * (ob["Nu_f_hot"] + ob["Nu_s_hot"]) == pytest.approx(J, rel=1e-12)


@pytest.mark.parametrize("sched", [1, 2])
@pytest.mark.parametrize("nx,ny,seg", [(4, 4, 3), (6, 5, 7), (9, 7, 40)])
def test_every_node_on_tiny_cavities(nx, ny, seg, sched):
    """The gradient at every node -- walls, corners and the interior nodes the
    walls are rebuilt from included -- against the complex-step oracle, FP64,
    40 steps: in segments of 3 (graph replays between a first and a last
    segment run on the stream), of 7 (ragged) and in one segment; both
    register budgets of the transposed collision."""
    cfg = dict(SMALL, nx=nx, ny=ny, Ra=1e3, Da=1e-2)
    phi = W.porosity_field(nx, ny, 0.4, 0.8, seed=50 + nx).reshape(-1)
    ref = _complex_step(cfg, phi, 40, range(nx * ny))
    cav = cavity_for(cfg, storage="f64", phi=phi).set_adjoint_schedule(sched)
    J, g, dH = cav.adjoint(phi, 40, segment=seg)
    g = g.cpu().numpy().reshape(-1)
    gref = np.array([ref[k] for k in range(nx * ny)])
    assert J == pytest.approx(ref["J"], rel=1e-12)
    assert np.abs(g - gref).max() <= 1e-9 * np.abs(gref).max(), np.abs(g - gref).reshape(ny, nx)
    assert dH == pytest.approx(ref[-1], rel=1e-9)


@pytest.mark.parametrize("steps,seg", [(1, 1), (1, 4), (2, 1), (3, 2), (5, 2)])
def test_fewest_steps(steps, seg):
    """One to five steps in segments of one or two (a last segment of one
    step, a single ragged segment, a segment longer than the run): every
    node against the complex-step oracle, FP64.  After one or two steps the
    wall Nusselt numbers do not yet depend on the porosity (the fluid starts
    at rest and both phases at one temperature): the gradient is zero up to
    round-off on both sides."""
    nx, ny = 6, 5
    cfg = dict(SMALL, nx=nx, ny=ny, Ra=1e3, Da=1e-2)
    phi = W.porosity_field(nx, ny, 0.4, 0.8, seed=80 + steps).reshape(-1)
    ref = _complex_step(cfg, phi, steps, range(nx * ny))
    cav = cavity_for(cfg, storage="f64", phi=phi)
    J, g, dH = cav.adjoint(phi, steps, segment=seg)
    g = g.cpu().numpy().reshape(-1)
    gref = np.array([ref[k] for k in range(nx * ny)])
    assert J == pytest.approx(ref["J"], rel=1e-12)
    assert np.abs(g - gref).max() <= 1e-9 * max(np.abs(gref).max(), 1e-6)
    assert dH == pytest.approx(ref[-1], rel=1e-9, abs=1e-12)
    assert cav.observables()["step"] == steps


@pytest.mark.parametrize("storage,tol", [("f32", 1e-5), ("f64", 1e-12)])
def test_register_budgets_agree(storage, tol):
    """Both builds of the transposed collision, and the size-based choice, on
    a lattice that fits one wave (all registers by default) and on one that
    does not (capped by default): the default gives the bits of the build it
    picks, a repeated run the same bits, and the other build agrees to
    rounding (under a register cap the compiler may contract a different
    set of multiply-adds)."""
    for nx, ny, auto in ((40, 30, 1), (400, 300, 2)):
        cfg = dict(SMALL, nx=nx, ny=ny)
        phi = W.porosity_field(nx, ny, 0.4, 0.8, seed=60).reshape(-1)
        outs = {}
        for sched in (0, 1, 2, 1):
            cav = cavity_for(cfg, storage=storage, phi=phi).set_adjoint_schedule(sched)
            J, g, dH = cav.adjoint(phi, 30, segment=6)
            outs.setdefault(sched, []).append((J, g.double().cpu().numpy(), dH))
            cav.close()
        a, b = outs[0][0], outs[auto][0]
        assert a[0] == b[0] and a[2] == b[2] and np.array_equal(a[1], b[1])
        r1, r2 = outs[1]
        assert r1[0] == r2[0] and r1[2] == r2[2] and np.array_equal(r1[1], r2[1])
        c = outs[2][0]
        assert c[0] == r1[0]  # J: the forward pass is the same
        assert c[2] == pytest.approx(r1[2], rel=tol)
        assert np.abs(c[1] - r1[1]).max() <= tol * np.abs(r1[1]).max()


def test_segment_length_does_not_change_the_gradient(small_reference):
    phi, nodes, _ = small_reference
    outs = []
    for seg in (1, 7, 120, 500):
        cav = cavity_for(SMALL, storage="f64", phi=phi)
        J, g, dH = cav.adjoint(phi, 120, segment=seg)
        outs.append((J, g.cpu().numpy(), dH))
    for J, g, dH in outs[1:]:
        assert J == outs[0][0]
        assert np.array_equal(g, outs[0][1])
        assert dH == outs[0][2]


def _J_fp64(cfg, phi, steps, d_p, H=None):
    c = dict(cfg, d_p=d_p)
    if H is not None:
        c["H"] = H
    cav = cavity_for(c, storage="f64", phi=phi).set_fields(porosity=phi).step(steps)
    ob = cav.observables()
    cav.close()
    return 0.5 * (ob["Nu_f_hot"] + ob["Nu_s_hot"])


def test_directional_derivative_dot_product(small_reference):
    """<dJ/dphi, v> equals the FP64 central difference along a random v."""
    from oracle import ergun_diameter

    phi, _, _ = small_reference
    d = ergun_diameter(phi, SMALL["ny"] - 1, SMALL["Da"])
    cav = cavity_for(dict(SMALL, d_p=d), storage="f64", phi=phi)
    _, g, _ = cav.adjoint(phi, 120, segment=16)
    v = np.random.default_rng(46).standard_normal(phi.size)
    eps = 1e-6
    fd = (_J_fp64(SMALL, phi + eps * v, 120, d) - _J_fp64(SMALL, phi - eps * v, 120, d)) / (2 * eps)
    assert float(g.cpu().numpy().reshape(-1) @ v) == pytest.approx(fd, rel=1e-6)


def test_c4_fp32_adjoint_vs_fp64_central_differences():
    """256 x 256, porosity U[0.4, 0.8] (seed 4), Ra 1e5, Da 1e-3 (Ergun, mean),
    H 50, 4000 steps, ceil(sqrt(4000)) = 64-step segments: the FP32 adjoint
    against FP64 central differences of the forward step on 32 interior nodes
    (seed 40) and H."""
    from oracle import ergun_diameter

    c = W.C4_ADJOINT
    nx, ny, steps = c["nx"], c["ny"], c["steps"]
    cfg = {k: v for k, v in c.items() if k not in ("phi_lo", "phi_hi", "seed", "steps",
                                                   "fd_nodes", "fd_seed")}
    phi = W.porosity_field(nx, ny, c["phi_lo"], c["phi_hi"], c["seed"]).reshape(-1)
    d = ergun_diameter(phi, ny - 1, c["Da"])
    cfg["d_p"] = d
    cav = cavity_for(cfg, storage="f32", phi=phi)
    J, g, dH = cav.adjoint(phi, steps, segment=64)
    g = g.double().cpu().numpy().reshape(-1)
    nodes = W.fd_nodes(nx, ny, c["fd_nodes"], c["fd_seed"])
    h = 1e-5
    fd = []
    for k in nodes:
        pp, pm = phi.copy(), phi.copy()
        pp[k] += h
        pm[k] -= h
        fd.append((_J_fp64(cfg, pp, steps, d) - _J_fp64(cfg, pm, steps, d)) / (2 * h))
    fd = np.array(fd)
    hH = 1e-4 * cfg["H"]
    fdH = (_J_fp64(cfg, phi, steps, d, H=cfg["H"] + hH)
           - _J_fp64(cfg, phi, steps, d, H=cfg["H"] - hH)) / (2 * hH)
    scale = np.abs(fd).max()
    assert np.abs(g[nodes] - fd).max() <= 1e-3 * scale, np.abs(g[nodes] - fd) / scale
    assert np.linalg.norm(g[nodes] - fd) <= 1e-3 * np.linalg.norm(fd)
    assert dH == pytest.approx(fdH, rel=1e-3)
    J64 = _J_fp64(cfg, phi, steps, d)
    assert J == pytest.approx(J64, rel=1e-5)


def test_autograd_function_returns_the_adjoint_gradient(small_reference):
    from paper_1608_04118_gb300.autograd import wall_nusselt

    phi, nodes, ref = small_reference
    t = torch.tensor(phi.reshape(SMALL["ny"], SMALL["nx"]), dtype=torch.float64,
                     requires_grad=True)
    H = torch.tensor(SMALL["H"], dtype=torch.float64, requires_grad=True)
    kw = {k: v for k, v in phys(SMALL).items() if k != "H"}
    J = wall_nusselt(t, H, 120, 16, "f64", **kw)
    (2.0 * J).backward()
    gref = np.array([ref[int(k)] for k in nodes])
    got = t.grad.numpy().reshape(-1)[nodes] / 2.0
    assert np.abs(got - gref).max() <= 1e-9 * np.abs(gref).max()
    assert float(H.grad) / 2.0 == pytest.approx(ref[-1], rel=1e-9)


def test_adjoint_with_thermal_correction_term():
    """The transposed correction term of Sec. 3.2: FP64 adjoint against the
    complex-step oracle with the term switched on."""
    cfg = dict(SMALL, thermal_correction=1)
    phi = W.porosity_field(cfg["nx"], cfg["ny"], 0.4, 0.8, seed=48).reshape(-1)
    nodes = W.fd_nodes(cfg["nx"], cfg["ny"], 8, seed=49)
    ref = _complex_step(cfg, phi, 90, nodes)
    cav = cavity_for(cfg, storage="f64", phi=phi)
    J, g, dH = cav.adjoint(phi, 90, segment=10)
    g = g.cpu().numpy().reshape(-1)
    gref = np.array([ref[int(k)] for k in nodes])
    assert J == pytest.approx(ref["J"], rel=1e-12)
    assert np.abs(g[nodes] - gref).max() <= 1e-9 * np.abs(gref).max()
    assert dH == pytest.approx(ref[-1], rel=1e-9)

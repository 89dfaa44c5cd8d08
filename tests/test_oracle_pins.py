"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the passage it checks.  None of them retypes the oracle's
formulas: they check identities between the paper's equations, invariants,
closed-form solutions and textbook lattice properties, chosen so that a
dropped term, a wrong sign or index or a transposed operand in the oracle
fails at least one of them.
"""
import numpy as np
import pytest

from oracle import Oracle, OracleParams, lattice_tables
from oracle.ltne_oracle import BC_CAVITY, BC_CHANNEL, BC_PERIODIC


def _e():
    e, w, M, Mi, N, Ni = lattice_tables()
    return e[0], e[1], w, M, Mi, N, Ni


# ---------------------------------------------------------------- p1 -----
def test_velocity_set_and_weights_are_isotropic():
    """Eq. 8 and the weights below Eq. 24: the D2Q9 set must reproduce the
    isotropic lattice tensors up to fourth order with cs^2 = 1/3."""
    ex, ey, w, *_ = _e()
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    E = np.stack([ex, ey])
    assert np.allclose(E @ w, 0, atol=1e-15)
    T2 = np.einsum("i,ai,bi->ab", w, E, E)
    assert np.allclose(T2, np.eye(2) / 3, atol=1e-15)
    T3 = np.einsum("i,ai,bi,ci->abc", w, E, E, E)
    assert np.allclose(T3, 0, atol=1e-15)
    T4 = np.einsum("i,ai,bi,ci,di->abcd", w, E, E, E, E)
    d = np.eye(2)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.allclose(T4, iso, atol=1e-15)
    # opposite pairs exist for every moving direction
    for i in range(1, 9):
        assert sum((ex[j] == -ex[i]) and (ey[j] == -ey[i]) for j in range(9)) == 1


def test_moment_matrices_match_their_definitions():
    """Eq. 13 rows are the moments named in Eq. 14 (rho, e, epsilon, j, q,
    p_xx, p_xy, as polynomials of e_i); Eq. 36 rows are [1, e_x, e_y,
    5e^2-4, e_x^2-e_y^2] as the paper defines them above the table."""
    ex, ey, w, M, Mi, N, Ni = _e()
    e2 = ex ** 2 + ey ** 2
    rows = np.array([
        np.ones(9), 3 * e2 - 4, (9 * e2 ** 2 - 21 * e2 + 8) / 2,
        ex, (3 * e2 - 5) * ex, ey, (3 * e2 - 5) * ey, ex ** 2 - ey ** 2, ex * ey])
    assert np.array_equal(M, rows)
    ex5, ey5 = ex[:5], ey[:5]
    e25 = ex5 ** 2 + ey5 ** 2
    rowsN = np.array([np.ones(5), ex5, ey5, 5 * e25 - 4, ex5 ** 2 - ey5 ** 2])
    assert np.array_equal(N, rowsN)


def test_moment_matrices_orthogonal_and_inverses():
    """M M^T = diag(9,36,36,6,12,6,12,4,4); N N^T = diag(5,2,2,20,4) (both
    exact in integers); the numerically formed inverses invert them."""
    ex, ey, w, M, Mi, N, Ni = _e()
    assert np.array_equal(M @ M.T, np.diag([9, 36, 36, 6, 12, 6, 12, 4, 4]).astype(float))
    assert np.array_equal(N @ N.T, np.diag([5, 2, 2, 20, 4]).astype(float))
    assert np.allclose(Mi @ M, np.eye(9), atol=1e-14)
    assert np.allclose(Ni @ N, np.eye(5), atol=1e-14)


# ---------------------------------------------------------------- p2 -----
def _box(nx=8, ny=8, **kw):
    return Oracle(OracleParams.make(nx, ny, **kw))


def test_equilibrium_moments_consistent():
    """Eq. 15 equals M times Eq. 24; Eq. 37 equals N times Eq. 50; Eq. 38
    equals N times Eq. 51, including the (-4 + 5 varpi) T entry."""
    rng = np.random.default_rng(11)
    ex, ey, w, M, Mi, N, Ni = _e()
    for varpi in (0.4, 0.7):
        o = _box(varpi=varpi)
        for _ in range(20):
            rho, ux, uy = rng.uniform(0.8, 1.2), rng.uniform(-0.1, 0.1), rng.uniform(-0.1, 0.1)
            Tf, Ts, phi = rng.uniform(-1, 2), rng.uniform(-1, 2), rng.uniform(0.3, 0.95)
            fe, gfe, gse, me, _ = o.equilibria(rho, ux, uy, Tf, Ts, phi)
            assert np.allclose(M @ fe, me, atol=1e-15, rtol=0)
            nfeq = np.array([Tf, ux * Tf / phi, uy * Tf / phi, (-4 + 5 * varpi) * Tf, 0])
            nseq = np.array([Ts, 0, 0, (-4 + 5 * varpi) * Ts, 0])
            assert np.allclose(N @ gfe, nfeq, atol=1e-14, rtol=0)
            assert np.allclose(N @ gse, nseq, atol=1e-14, rtol=0)
            # f^eq carries exactly the mass, momentum and the porous
            # momentum flux rho cs^2 I + rho u u / phi of Sec. 3.1.
            E = np.stack([ex, ey])
            assert fe.sum() == pytest.approx(rho, abs=1e-15)
            assert np.allclose(E @ fe, rho * np.array([ux, uy]), atol=1e-15)
            Pi = np.einsum("i,ai,bi->ab", fe, E, E)
            u = np.array([ux, uy])
            assert np.allclose(Pi, rho / 3 * np.eye(2) + rho * np.outer(u, u) / phi, atol=1e-15)


# ---------------------------------------------------------------- p3 -----
def test_forcing_moments():
    """The velocity-space forcing used for Eq. 16 (reading of a garbled
    equation) must carry zero mass, momentum rho F and second moment
    rho (uF + Fu)/phi, and M S must equal the closed form
    (0, 6 rho u.F/phi, -6 rho u.F/phi, rho Fx, -rho Fx, rho Fy, -rho Fy,
    2 rho (ux Fx - uy Fy)/phi, rho (ux Fy + uy Fx)/phi)."""
    rng = np.random.default_rng(12)
    ex, ey, w, M, Mi, N, Ni = _e()
    E = np.stack([ex, ey])
    o = _box()
    for _ in range(20):
        rho, ux, uy = rng.uniform(0.8, 1.2), rng.uniform(-0.1, 0.1), rng.uniform(-0.1, 0.1)
        Fx, Fy, phi = rng.uniform(-1e-3, 1e-3), rng.uniform(-1e-3, 1e-3), rng.uniform(0.3, 0.95)
        *_, S = o.equilibria(rho, ux, uy, 0.5, 0.5, phi, Fx, Fy)
        u, F = np.array([ux, uy]), np.array([Fx, Fy])
        assert abs(S.sum()) < 1e-18
        assert np.allclose(E @ S, rho * F, atol=1e-18, rtol=1e-13)
        P = np.einsum("i,ai,bi->ab", S, E, E)
        assert np.allclose(P, rho * (np.outer(u, F) + np.outer(F, u)) / phi, atol=1e-18, rtol=1e-12)
        uF = u @ F
        closed = np.array([0, 6 * rho * uF / phi, -6 * rho * uF / phi, rho * Fx, -rho * Fx,
                           rho * Fy, -rho * Fy, 2 * rho * (ux * Fx - uy * Fy) / phi,
                           rho * (ux * Fy + uy * Fx) / phi])
        assert np.allclose(M @ S, closed, atol=1e-18, rtol=1e-12)


# ---------------------------------------------------------------- p4 -----
def test_velocity_solve_satisfies_implicit_definition():
    """Eq. 20 with Eqs. 21-22 must solve Eq. 19 with the force of Eq. 5,
    and the temperatures of Eqs. 43-44 must solve Eqs. 41-42."""
    rng = np.random.default_rng(13)
    ex, ey, w, *_ = _e()
    E = np.stack([ex, ey])
    for trial in range(30):
        phi = rng.uniform(0.3, 0.9)
        kw = dict(porosity=phi, Da=10 ** rng.uniform(-4, -1), H=10 ** rng.uniform(-1, 3),
                  Ra=10 ** rng.uniform(3, 6), gamma_sf=10 ** rng.uniform(-1, 2),
                  sigma=rng.uniform(0.5, 2), qf=rng.uniform(-1e-4, 1e-4),
                  qs=rng.uniform(-1e-4, 1e-4), ext_ax=rng.uniform(-1e-4, 1e-4))
        o = _box(16, 16, **kw)
        d = o.derived()
        K, Fphi = o.medium()
        K, Fphi = K[0, 0], Fphi[0, 0]
        f = w * rng.uniform(0.9, 1.1, 9)
        gf = rng.uniform(0.0, 0.3, 5)
        gs = rng.uniform(0.0, 0.3, 5)
        _, _, _, m, _, _ = o.node(0, f, gf, gs)
        u = np.array([m["ux"], m["uy"]])
        G = np.array([m["Gx"], m["Gy"]])
        umag = np.hypot(*u)
        Fvec = -phi * d["nu_f"] / K * u - phi * Fphi / np.sqrt(K) * umag * u + phi * G
        assert np.allclose([m["Fx"], m["Fy"]], Fvec, rtol=1e-13, atol=1e-20)
        lhs = m["rho"] * u
        rhs = E @ f + 0.5 * m["rho"] * Fvec
        assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-17)
        # Eq. 41 with Eq. 42 (a, b are the per-node exchange coefficients)
        Srf = m["a"] * (m["Ts"] - m["Tf"]) + kw["qf"]
        Srs = m["b"] * (m["Tf"] - m["Ts"]) + kw["qs"]
        assert m["Tf"] == pytest.approx(gf.sum() + 0.5 * Srf, rel=1e-13, abs=1e-15)
        assert m["Ts"] == pytest.approx(gs.sum() + 0.5 * Srs, rel=1e-13, abs=1e-15)
        # buoyancy is along +y for T_f above T_0 (reading: gravity along -y)
        assert m["Gy"] == pytest.approx(d["gbeta"] * (m["Tf"] - 0.5), rel=1e-13, abs=1e-20)


def test_parameter_mapping_reproduces_dimensionless_groups():
    """The lattice values recover the groups of Sec. 2 (Ra, Pr, Da, J_e,
    gamma_sf / sigma) and the transport relations of Eqs. 23 and 49."""
    o = _box(33, 65, Ra=3e5, Pr=0.7, J_e=1.3, gamma_sf=7.0, sigma=2.0, H=40.0)
    d = o.derived()
    L = 64.0
    assert d["L"] == L
    Ra = d["gbeta"] * 1.0 * L ** 3 / (d["nu_f"] * d["alpha_f"])
    assert Ra == pytest.approx(3e5, rel=1e-12)
    assert d["nu_f"] / d["alpha_f"] == pytest.approx(0.7, rel=1e-14)
    assert d["nu_e"] / d["nu_f"] == pytest.approx(1.3, rel=1e-14)
    assert d["alpha_s"] / d["alpha_f"] == pytest.approx(7.0 / 2.0, rel=1e-14)
    assert d["cs2"] * (1 / d["s_nu"] - 0.5) == pytest.approx(d["nu_e"], rel=1e-13)
    assert d["csT2"] * (1 / d["zeta_alpha"] - 0.5) == pytest.approx(d["alpha_f"], rel=1e-13)
    assert d["csT2"] * (1 / d["eta_alpha"] - 0.5) == pytest.approx(d["alpha_s"], rel=1e-13)
    # H_v = h_v L^2 / k_f  =>  h_v / (rho c)_f = H alpha_f / L^2
    assert d["hv_over_rhoc_f"] * L ** 2 / d["alpha_f"] == pytest.approx(40.0, rel=1e-13)


def test_ergun_medium():
    """Eq. 7 per node; with the particle diameter fixed from the mean
    Darcy number, the mean of K / L^2 over the nodes equals Da."""
    rng = np.random.default_rng(14)
    phi = rng.uniform(0.3, 0.9, size=(20, 24))
    o = Oracle(OracleParams.make(24, 20, ergun_K=1, Da=1e-3), phi=phi)
    K, F = o.medium()
    L = 19.0
    assert (K / L ** 2).mean() == pytest.approx(1e-3, rel=1e-12)
    # ratios between nodes follow phi^3 / (1 - phi)^2, independent of d
    r = (phi ** 3 / (1 - phi) ** 2)
    assert np.allclose(K / K[0, 0], r / r[0, 0], rtol=1e-12)
    assert np.allclose(F ** 2 * 150 * phi ** 3, 1.75 ** 2, rtol=1e-12)


# ---------------------------------------------------------------- p5 -----
def test_conservation_periodic():
    """Periodic box, uniform porosity, no internal generation: total mass
    and total energy sum[phi sum g_f + (1-phi) sigma sum g_s] are conserved
    because the interphase sources cancel (the remark after Eq. 42)."""
    rng = np.random.default_rng(15)
    nx = ny = 16
    o = Oracle(OracleParams.make(nx, ny, bc=BC_PERIODIC, Ra=1e5, H=50.0, gamma_sf=5.0,
                                 sigma=1.7, porosity=0.45))
    o.init(rho=1 + 0.01 * rng.standard_normal(nx * ny), ux=0.02 * rng.standard_normal(nx * ny),
           uy=0.02 * rng.standard_normal(nx * ny), Tf=rng.uniform(0, 1, nx * ny),
           Ts=rng.uniform(0, 1, nx * ny))
    ob0 = o.observables()
    o.step(2000)
    ob1 = o.observables()
    # round-off only: at most a few ulp of drift per step
    tol = 2000 * 4 * np.finfo(float).eps
    assert ob1["mass"] == pytest.approx(ob0["mass"], rel=tol)
    assert ob1["energy"] == pytest.approx(ob0["energy"], rel=tol)
    # and the run did something
    assert ob1["max_dT"] < 0.5 * ob0["max_dT"]


# ---------------------------------------------------------------- p6 -----
@pytest.mark.parametrize("H,phi,sigma,gsf", [(200.0, 0.6, 1.0, 1.0), (5e3, 0.35, 2.5, 30.0)])
def test_interphase_relaxation_trapezoid_law(H, phi, sigma, gsf):
    """Uniform fields with T_f != T_s: Eqs. 41-46 with the (I - Q/2) source
    treatment of Eqs. 32-33 advance the difference by the trapezoid rule,
    D^{n+1} = D^n (1 - k/2)/(1 + k/2) with k = a + b, to round-off, while
    phi T_f + (1 - phi) sigma T_s stays fixed."""
    nx = ny = 4
    o = Oracle(OracleParams.make(nx, ny, bc=BC_PERIODIC, Ra=1e4, H=H, porosity=phi,
                                 sigma=sigma, gamma_sf=gsf))
    o.init(Tf=np.full(nx * ny, 0.9), Ts=np.full(nx * ny, 0.1))
    mac = o.macros()
    _, _, _, m, _, _ = o.node(0, *[x[0, 0] for x in o.get_pops()])
    k = m["a"] + m["b"]
    r = (1 - k / 2) / (1 + k / 2)
    D0 = mac["Tf"][0, 0] - mac["Ts"][0, 0]
    W0 = phi * mac["Tf"][0, 0] + (1 - phi) * sigma * mac["Ts"][0, 0]
    for n in range(1, 40):
        o.step(1)
        mac = o.macros()
        D = mac["Tf"] - mac["Ts"]
        assert np.allclose(D, D0 * r ** n, rtol=1e-12, atol=1e-15)
        W = phi * mac["Tf"] + (1 - phi) * sigma * mac["Ts"]
        assert np.allclose(W, W0, rtol=1e-14)
    # the continuous law exp(-k t) is matched to the trapezoid rule's O(k^3)
    assert abs(np.log(abs(r)) + k) <= k ** 3 / 12 * 1.01 + 1e-15


# ---------------------------------------------------------------- p7/p8 --
def test_uniform_forchheimer_flow():
    """Uniform periodic flow under a constant body acceleration A: the
    momentum grows by rho F per step, i.e. rho u^{n+1} - rho F(u^{n+1})/2 =
    rho u^n + rho F(u^n)/2 with F from Eq. 5, and u tends to the root of
    nu/K u + F_phi/sqrt(K) u^2 = A."""
    nx = ny = 4
    A = 2e-4
    o = Oracle(OracleParams.make(nx, ny, bc=BC_PERIODIC, Ra=0.0, nu_override=0.05, Da=1e-3,
                                 porosity=0.5, ext_ax=A, T_hot=0.5, T_cold=0.5))
    o.init()
    K, Fp = o.medium()
    K, Fp = K[0, 0], Fp[0, 0]
    nu, phi = 0.05, 0.5

    def F(u):
        return -phi * nu / K * u - phi * Fp / np.sqrt(K) * abs(u) * u + phi * A

    u_prev = o.macros()["ux"][0, 0]
    rho = o.macros()["rho"][0, 0]
    for _ in range(200):
        o.step(1)
        mac = o.macros()
        u = mac["ux"][0, 0]
        assert np.allclose(mac["ux"], u, rtol=0, atol=1e-17)
        assert np.allclose(mac["uy"], 0, atol=1e-17)
        assert rho * u - 0.5 * rho * F(u) == pytest.approx(rho * u_prev + 0.5 * rho * F(u_prev),
                                                           rel=1e-12, abs=1e-18)
        u_prev = u
    o.step(20000)
    u = o.macros()["ux"][0, 0]
    a, b = nu / K, Fp / np.sqrt(K)
    u_inf = (-a + np.sqrt(a * a + 4 * b * A)) / (2 * b)
    assert u == pytest.approx(u_inf, rel=1e-10)


# ---------------------------------------------------------------- p9 -----
def test_cavity_centro_symmetry():
    """Uniform porosity, walls at +1 / -1 and T_0 = 0: the cavity of Sec. 4
    is symmetric under the half-turn x -> L - x, y -> L - y, which maps T to
    -T and u to -u, at every step.  (With T_0 != 0 the advective part
    (e_i.u) T_0 / (2 phi) of Eq. 50 is even under the half-turn, so the
    weakly compressible flow breaks the symmetry at O(Ma^2); every term is
    odd in T only when T_0 = 0.)"""
    nx, ny = 24, 24
    o = Oracle(OracleParams.make(nx, ny, Ra=1e5, H=20.0, gamma_sf=3.0, T_hot=1.0, T_cold=-1.0,
                                 T_ref=0.0))
    o.init()
    for _ in range(4):
        o.step(150)
        m = o.macros()
        for k in ("Tf", "Ts", "ux", "uy"):
            assert np.allclose(m[k], -m[k][::-1, ::-1], rtol=0, atol=1e-13)
        assert np.abs(m["ux"]).max() > 1e-4
        assert np.allclose(m["rho"], m["rho"][::-1, ::-1], rtol=0, atol=1e-13)


# ---------------------------------------------------------------- p10 ----
def _brinkman(ny):
    nu, nu_e_ratio, phi, Da, A = 0.1, 1.5, 0.6, 5e-3, 1e-6
    o = Oracle(OracleParams.make(4, ny, bc=BC_CHANNEL, Ra=0.0, nu_override=nu, J_e=nu_e_ratio,
                                 porosity=phi, Da=Da, F_phi=0.0, ext_ax=A, T_hot=0.5,
                                 T_cold=0.5))
    o.init()
    K = o.medium()[0][0, 0]
    L = ny - 1.0
    o.step(int(40 * K / (phi * nu)) + 4 * int(L * L / (nu * nu_e_ratio)))
    ux = o.macros()["ux"][:, 1]
    y = np.arange(ny)
    r = np.sqrt(phi * nu / (K * nu * nu_e_ratio))
    ua = A * K / nu * (1 - np.cosh(r * (y - L / 2)) / np.cosh(r * L / 2))
    return np.linalg.norm(ux - ua) / np.linalg.norm(ua)


@pytest.mark.slow
def test_brinkman_channel_profile():
    """Steady channel flow with the Forchheimer term off obeys the Brinkman
    equation nu_e u'' - phi nu_f u / K + phi A = 0 (Eqs. 2, 5), whose
    solution is a cosh profile; the error falls at about second order."""
    errs = [_brinkman(ny) for ny in (17, 33, 65)]
    assert errs[2] <= 1e-3
    order = np.log2(errs[1] / errs[2])
    assert order > 1.6, errs


# ---------------------------------------------------------------- p11 ----
def test_pure_conduction_walls_and_nusselt():
    """Ra = 0: steady conduction between the isothermal walls is linear in
    x for both phases and Nu = 1 on both walls, which checks the wall
    rebuild and the wall-flux stencil."""
    nx = ny = 16
    o = Oracle(OracleParams.make(nx, ny, Ra=0.0, nu_override=0.2, H=30.0, gamma_sf=4.0,
                                 sigma=1.5, T_hot=1.0, T_cold=0.0))
    o.init()
    o.step(12000)
    ob = o.observables()
    for k in ("Nu_f_hot", "Nu_s_hot", "Nu_f_cold", "Nu_s_cold"):
        assert ob[k] == pytest.approx(1.0, abs=1e-10)
    m = o.macros()
    x = np.arange(nx)
    lin = 1.0 - x / (nx - 1.0)
    for k in ("Tf", "Ts"):
        assert np.allclose(m[k][1:-1, :], lin[None, :], atol=1e-10)
    assert np.abs(m["ux"]).max() == 0 and np.abs(m["uy"]).max() == 0


# ---------------------------------------------------------------- p12 ----
@pytest.mark.slow
def test_lte_limit():
    """Large interphase coefficient drives T_f -> T_s (local thermal
    equilibrium); the gap shrinks roughly as 1/H."""
    gaps, fields = [], []
    for H in (1e2, 1e4, 1e6):
        o = Oracle(OracleParams.make(32, 32, Ra=1e4, H=H, gamma_sf=10.0))
        o.init().step(3000)
        gaps.append(o.observables()["max_dT"])
        fields.append(o.macros()["Tf"])
    assert gaps[0] > gaps[1] > gaps[2]
    for a, b in zip(gaps, gaps[1:]):
        assert 30 < a / b < 300
    assert np.abs(fields[1] - fields[2]).max() < np.abs(fields[0] - fields[2]).max()


# ---------------------------------------------------------------- p13 ----
def test_solid_diffusivity_chapman_enskog():
    """A sine mode of T_s with u = 0 and H = 0 decays at alpha_s k^2 with
    alpha_s = c_sT^2 (1/eta_alpha - 1/2) (Eq. 49, c_sT^2 = varpi/2)."""
    nx, ny = 128, 3
    o = Oracle(OracleParams.make(nx, ny, bc=BC_PERIODIC, Ra=0.0, nu_override=0.1, H=0.0,
                                 gamma_sf=3.0, sigma=1.0))
    d = o.derived()
    x = np.arange(nx)
    k = 2 * np.pi / nx
    Ts = 0.5 + 0.1 * np.sin(k * x)
    o.init(Ts=np.tile(Ts, ny))

    def amp():
        t = o.macros()["Ts"][1]
        return 2 * np.mean((t - 0.5) * np.sin(k * x))

    o.step(200)
    a1 = amp()
    o.step(1800)
    a2 = amp()
    rate = -np.log(a2 / a1) / 1800
    assert rate == pytest.approx(d["alpha_s"] * k * k, rel=1e-3)


# ---------------------------------------------------------------- p15 ----
def test_complex_step_gradient_matches_central_differences():
    """The complex-step variant (gradient reference of the adjoint) agrees
    with FP64 central differences of the real oracle, for the porosity of an
    interior node and for H, with the Ergun diameter held fixed."""
    from oracle import ComplexOracle

    nx, ny, steps = 12, 10, 60
    phi = np.random.default_rng(47).uniform(0.4, 0.8, nx * ny)
    kw = dict(ergun_K=1, Ra=1e5, Da=1e-3, H=50.0, gamma_sf=3.0, sigma=1.2)
    d = Oracle(OracleParams.make(nx, ny, **kw), phi=phi).derived()["d_ergun"]
    kw["d_p"] = d

    def J(ph, H=50.0):
        o = Oracle(OracleParams.make(nx, ny, **dict(kw, H=H)), phi=ph).init().step(steps)
        return o.objective()[0]

    pairs = []
    for k in (3 * nx + 4, 5 * nx + 7, 2 * nx + 1):
        co = ComplexOracle(OracleParams.make(nx, ny, **kw), phi=phi).perturb(k, 1e-30)
        cs = co.init().step(steps).objective()[1] / 1e-30
        h = 1e-4  # round-off of J (~1e-15) / h stays far below the tolerance
        pp, pm = phi.copy(), phi.copy()
        pp[k] += h
        pm[k] -= h
        pairs.append((cs, (J(pp) - J(pm)) / (2 * h)))
    co = ComplexOracle(OracleParams.make(nx, ny, **kw), phi=phi).perturb(-1, 1e-30)
    cs = co.init().step(steps).objective()[1] / 1e-30
    pairs.append((cs, (J(phi, 50.0 + 1e-2) - J(phi, 50.0 - 1e-2)) / 2e-2))
    cs, fd = np.array(pairs).T
    assert np.abs(cs - fd).max() <= 1e-6 * np.abs(fd).max(), (cs, fd)


# ---------------------------------------------------------------- f3 -----
def test_internal_generation_uniform_box():
    """Internal generation Q''' (Eqs. 30-31, 43-45) in a uniform periodic box:
    the weighted temperature phi T_f + (1-phi) sigma T_s grows by exactly
    phi Q_f + (1-phi) sigma Q_s per step (the exchange terms cancel), and
    the phase difference follows the trapezoid recurrence
    D^{n+1} (1 + k/2) = D^n (1 - k/2) + (Q_f - Q_s), k = a + b."""
    nx = ny = 4
    phi, sigma, qf, qs = 0.55, 1.7, 3e-4, -1e-4
    o = Oracle(OracleParams.make(nx, ny, bc=BC_PERIODIC, Ra=1e4, H=300.0, porosity=phi,
                                 sigma=sigma, gamma_sf=2.0, qf=qf, qs=qs))
    o.init(Tf=np.full(nx * ny, 0.7), Ts=np.full(nx * ny, 0.2))
    _, _, _, m, _, _ = o.node(0, *[x[0, 0] for x in o.get_pops()])
    k = m["a"] + m["b"]
    mac = o.macros()
    W0 = phi * mac["Tf"][0, 0] + (1 - phi) * sigma * mac["Ts"][0, 0]
    D = mac["Tf"][0, 0] - mac["Ts"][0, 0]
    for n in range(1, 30):
        o.step(1)
        mac = o.macros()
        W = phi * mac["Tf"] + (1 - phi) * sigma * mac["Ts"]
        assert np.allclose(W, W0 + n * (phi * qf + (1 - phi) * sigma * qs), rtol=1e-13, atol=1e-15)
        D = (D * (1 - k / 2) + (qf - qs)) / (1 + k / 2)
        assert np.allclose(mac["Tf"] - mac["Ts"], D, rtol=1e-12, atol=1e-15)
    o.step(5000)
    mac = o.macros()
    assert np.allclose(mac["Tf"] - mac["Ts"], (qf - qs) / k, rtol=1e-9)


# ---------------------------------------------------------------- f2 -----
@pytest.mark.parametrize("Pr", [5.0, 1.0])
def test_correction_term_removes_the_unwanted_flux(Pr):
    """Sec. 3.2 (Eq. 47): the thermal equation carries an unwanted flux
    (1/zeta_alpha - 1/2) d_t1(u T_f / phi); under a uniform force with no
    pressure gradient d_t1 u = F, so a temperature profile advected by the
    accelerating flow drifts by -(1/zeta_alpha - 1/2) sum_n F/phi against the
    exact displacement integral of u/phi dt.  The correction term
    dt N^-1 (I - Q/2) C with C~_i = w~_i T_f (e_i.F)/(phi c_sT^2) removes it."""
    nx, ny, N, A, phi = 64, 3, 300, 2e-5, 0.7
    x = np.arange(nx)
    k = 2 * np.pi / nx
    drift = {}
    for tc in (0, 1):
        o = Oracle(OracleParams.make(nx, ny, bc=BC_PERIODIC, Ra=0.0, nu_override=0.1, Pr=Pr,
                                     Da=1e6, porosity=phi, F_phi=0.0, ext_ax=A, H=0.0,
                                     T_hot=0.5, T_cold=0.5, thermal_correction=tc))
        o.init(Tf=np.tile(0.5 + 0.1 * np.sin(k * x), ny), Ts=np.full(nx * ny, 0.5))
        c = 1 / o.derived()["zeta_alpha"] - 0.5

        def phase():
            t = o.macros()["Tf"][1] - 0.5
            return np.angle(np.sum(t * np.exp(-1j * k * x)))

        p0 = phase()
        u = [o.macros()["ux"][1].mean()]
        for _ in range(N):
            o.step(1)
            u.append(o.macros()["ux"][1].mean())
        u = np.array(u)
        X_exact = np.sum(0.5 * (u[1:] + u[:-1])) / phi  # u is linear in time here
        drift[tc] = -(phase() - p0) / k - X_exact
    F_over_phi_sum = A * N
    assert drift[0] == pytest.approx(-c * F_over_phi_sum, rel=0.15)
    assert abs(drift[1]) <= 0.15 * c * F_over_phi_sum


# ---------------------------------------------------------------- f1 -----
def _hv_by_hand(u, nu, Pr, L, Dp_over_L):
    """h_v / (rho c)_f of Eq. 52 written out from the paper's definitions:
    H_p = h_v D_p^2 / k_f = 0.376 Re^0.644 Pr^0.37, Re = u_m D_p / nu_f,
    D_p = (D_p / L) L, and h_v / (rho c)_f = H_p alpha_f / D_p^2 with
    alpha_f = nu_f / Pr."""
    Dp = Dp_over_L * L
    Re = u * Dp / nu
    Hp = 0.376 * Re ** 0.644 * Pr ** 0.37
    return Hp * (nu / Pr) / Dp ** 2


@pytest.mark.parametrize("u,Pr,Dp_over_L,phi,sigma", [
    (0.05, 0.7, 0.0135, 0.6, 1.0),
    (0.02, 0.7, 0.0135, 0.6, 1.0),
    (0.05, 3.0, 0.0135, 0.45, 2.0),
    (0.03, 1.0, 0.05, 0.8, 0.5)])
def test_local_exchange_coefficient_eq52_uniform_flow(u, Pr, Dp_over_L, phi, sigma):
    """Eq. 52 in a uniform periodic box moving at a constant |u| (no force:
    permeability so large that the Darcy drag is below FP64 resolution, no
    Forchheimer term, no buoyancy): the local h_v is the same at every node
    and every step, so T_f - T_s follows the trapezoid law of Eqs. 41-46,
    D^{n+1} (1 + k/2) = D^n (1 - k/2), with k = a + b = h_v/(rho c)_f
    (1/phi + 1/((1 - phi) sigma)) and h_v from Eq. 52 computed here by hand.
    Four cases vary |u|, Pr, D_p and the phase weights, so a wrong
    exponent, D_p, Pr factor or length scale changes k."""
    nx = ny = 4
    nu, L = 0.05, 100.0
    o = Oracle(OracleParams.make(nx, ny, bc=BC_PERIODIC, Ra=0.0, nu_override=nu, Pr=Pr,
                                 Da=1e300, F_phi=0.0, porosity=phi, sigma=sigma, gamma_sf=2.0,
                                 hv_local=1, Dp_over_L=Dp_over_L, L_ref=L, T_hot=0.5,
                                 T_cold=0.5))
    ang = 0.3
    n = nx * ny
    o.init(ux=np.full(n, u * np.cos(ang)), uy=np.full(n, u * np.sin(ang)), Tf=np.full(n, 0.8),
           Ts=np.full(n, 0.3))
    hv = _hv_by_hand(u, nu, Pr, L, Dp_over_L)
    k = hv / phi + hv / ((1 - phi) * sigma)
    assert 1e-3 < k < 1.0  # the exchange is resolved and the law is non-trivial
    r = (1 - k / 2) / (1 + k / 2)
    mac = o.macros()
    D0 = mac["Tf"][0, 0] - mac["Ts"][0, 0]
    # the temperature solve of S_0 already used this k: A_f - A_s = D (1 + k/2)
    gf, gs = o.get_pops()[1:]
    assert gf[0, 0].sum() - gs[0, 0].sum() == pytest.approx(D0 * (1 + k / 2), rel=1e-13)
    for step in range(1, 30):
        o.step(1)
        mac = o.macros()
        assert np.allclose(np.hypot(mac["ux"], mac["uy"]), u, rtol=1e-13)
        assert np.allclose(mac["Tf"] - mac["Ts"], D0 * r ** step, rtol=1e-12, atol=1e-15)


# ---------------------------------------------------------------- p13' ---
@pytest.mark.parametrize("varpi", [0.4, 0.6])
def test_fluid_diffusivity_chapman_enskog(varpi):
    """A sine mode of T_f with u = 0 and H = 0 decays at alpha_f k^2, with
    alpha_f = c_sT^2 (1/zeta_alpha - 1/2) (Eq. 49, c_sT^2 = varpi/2) and
    alpha_f = nu_f / Pr computed here from the inputs.  The solid phase is
    given a diffusivity 12.5 times smaller (gamma_sf / sigma = 0.08), so a
    fluid phase relaxed with the solid-phase rates (Eq. 40 in place of
    Eq. 39) decays far too slowly, and the solid mode, started equal, must
    decay at alpha_s k^2 alongside."""
    nx, ny = 128, 3
    nu, Pr, gsf, sig = 0.1, 2.0, 0.2, 2.5
    o = Oracle(OracleParams.make(nx, ny, bc=BC_PERIODIC, Ra=0.0, nu_override=nu, Pr=Pr, H=0.0,
                                 gamma_sf=gsf, sigma=sig, varpi=varpi))
    alpha_f = nu / Pr
    alpha_s = gsf / sig * alpha_f
    x = np.arange(nx)
    k = 2 * np.pi / nx
    T = 0.5 + 0.1 * np.sin(k * x)
    o.init(Tf=np.tile(T, ny), Ts=np.tile(T, ny))

    def amps():
        m = o.macros()
        return [2 * np.mean((m[key][1] - 0.5) * np.sin(k * x)) for key in ("Tf", "Ts")]

    o.step(200)
    a1 = amps()
    o.step(1800)
    a2 = amps()
    rate_f = -np.log(a2[0] / a1[0]) / 1800
    rate_s = -np.log(a2[1] / a1[1]) / 1800
    assert rate_f == pytest.approx(alpha_f * k * k, rel=1e-3)
    assert rate_s == pytest.approx(alpha_s * k * k, rel=1e-3)


# ---------------------------------------------------------------- rates --
def test_relaxation_rates_act_on_their_moments():
    """Eq. 17 and Eqs. 39-40 place each relaxation rate on one moment.  In a
    spatially uniform periodic state streaming moves equal values between
    equal nodes, so only the collision acts: with u = 0, no force and no
    exchange (H = 0), the non-equilibrium part of every non-conserved moment
    is multiplied by (1 - rate) per step (Eq. 10; Eqs. 32-33), the conserved
    moments stay put.  Every rate is distinct here, and the hydrodynamic ones
    are computed from the inputs by Eqs. 23 and 49, so a rate on the wrong
    moment, a wrong varpi in c_sT^2 or in the (-4 + 5 varpi) entry of
    Eqs. 37-38, or a mix-up of the two phases' rates fails."""
    ex, ey, w, M, Mi, N, Ni = _e()
    nu, Je, Pr, gsf, sig, varpi = 0.07, 1.3, 0.8, 3.0, 1.4, 0.55
    rates = dict(s_e=0.7, s_eps=1.3, s_q=1.6, zeta_e=0.9, zeta_nu=1.5, eta_e=1.25, eta_nu=0.6)
    nx = ny = 3
    o = Oracle(OracleParams.make(nx, ny, bc=BC_PERIODIC, Ra=0.0, nu_override=nu, J_e=Je, Pr=Pr,
                                 H=0.0, gamma_sf=gsf, sigma=sig, varpi=varpi, porosity=0.55,
                                 **rates))
    s_nu = 1 / (3 * Je * nu + 0.5)                       # Eq. 23, c_s^2 = 1/3
    csT2 = varpi / 2                                      # Eq. 49
    zeta_a = 1 / ((nu / Pr) / csT2 + 0.5)
    eta_a = 1 / ((gsf / sig * nu / Pr) / csT2 + 0.5)
    s = np.array([0, rates["s_e"], rates["s_eps"], 0, rates["s_q"], 0, rates["s_q"], s_nu, s_nu])
    qf = np.array([0, zeta_a, zeta_a, rates["zeta_e"], rates["zeta_nu"]])
    qs = np.array([0, eta_a, eta_a, rates["eta_e"], rates["eta_nu"]])
    rho, Tf, Ts = 1.02, 0.7, 0.35
    c3 = -4 + 5 * varpi
    meq = np.array([rho, -2 * rho, rho, 0, 0, 0, 0, 0, 0])        # Eq. 15 at u = 0
    nfeq = np.array([Tf, 0, 0, c3 * Tf, 0])                      # Eq. 37 at u = 0
    nseq = np.array([Ts, 0, 0, c3 * Ts, 0])                      # Eq. 38
    dm = np.array([0, 0.011, -0.007, 0, 0.004, 0, -0.003, 0.006, -0.005])
    dnf = np.array([0, 0.012, -0.009, 0.02, -0.015])
    dns = np.array([0, -0.008, 0.011, -0.013, 0.017])
    f0 = np.linalg.solve(M, meq + dm)
    gf0 = np.linalg.solve(N, nfeq + dnf)
    gs0 = np.linalg.solve(N, nseq + dns)
    nn = nx * ny
    o.set_pops(np.tile(f0, nn), np.tile(gf0, nn), np.tile(gs0, nn))
    for step in range(1, 6):
        o.step(1)
        f, gf, gs = o.get_pops()
        for node in range(nn):
            y, x = divmod(node, nx)
            assert np.allclose(M @ f[y, x] - meq, dm * (1 - s) ** step, rtol=1e-12, atol=1e-15)
            assert np.allclose(N @ gf[y, x] - nfeq, dnf * (1 - qf) ** step, rtol=1e-12,
                               atol=1e-15)
            assert np.allclose(N @ gs[y, x] - nseq, dns * (1 - qs) ** step, rtol=1e-12,
                               atol=1e-15)

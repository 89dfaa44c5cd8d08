"""Seeded synthetic inputs shared by the tests, the smoke check and the
benchmark.  This module holds parameter values and random draws only -- no
arithmetic of the method -- so both the CUDA path and the oracle can take
their inputs from it.

The paper's workload is the differentially heated porous cavity of Sec. 4
(left wall hot, right wall cold, horizontal walls adiabatic, no-slip); there
is no public dataset, and these generators stand in for it.
"""
from __future__ import annotations

import numpy as np

# Physical parameters common to the CUDA binding and the oracle (same names
# in both parameter records).  ``ergun`` selects the Ergun permeability.
C1_PLAIN_64 = dict(nx=64, ny=64, Ra=1e4, Pr=1.0, Da=1e-2, porosity=0.6, H=10.0, gamma_sf=1.0,
                   sigma=1.0, T_hot=1.0, T_cold=0.0, T_ref=0.5, ergun=False, steps=10_000)

C2_THROUGHPUT = dict(Ra=1e6, Pr=1.0, Da=1e-3, H=100.0, gamma_sf=10.0, sigma=1.0, T_hot=1.0,
                     T_cold=0.0, T_ref=0.5, ergun=True, phi_lo=0.3, phi_hi=0.9, seed=2,
                     warmup=500, steps=2000)

C4_ADJOINT = dict(nx=256, ny=256, Ra=1e5, Pr=1.0, Da=1e-3, H=50.0, gamma_sf=1.0, sigma=1.0,
                  T_hot=1.0, T_cold=0.0, T_ref=0.5, ergun=True, phi_lo=0.4, phi_hi=0.8, seed=4,
                  steps=4000, fd_nodes=32, fd_seed=40)

C5_REDUCED = dict(nx=8192, ny=8192, Ra=1e6, Pr=1.0, Da=1e-2, porosity=0.6, H=1000.0,
                  gamma_sf=1.0, sigma=1.0, T_hot=1.0, T_cold=0.0, T_ref=0.5, ergun=False,
                  steps=2000, parity_n=512)


def porosity_field(nx, ny, lo, hi, seed):
    """Per-node porosity drawn i.i.d. uniform in [lo, hi], shape (ny, nx)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(ny, nx))


def batch_cavities(count=256, seed=3):
    """Independent cavities of uneven size and parameters: side drawn from
    {64, 96, ..., 512}, aspect ratio nx/ny from {1, 2}; Ra log-uniform in
    [1e3, 1e6], Da log-uniform in [1e-4, 1e-1], porosity uniform in
    [0.3, 0.9], H log-uniform in [1, 1000], conductivity ratio log-uniform
    in [0.1, 100]."""
    rng = np.random.default_rng(seed)
    sides = np.arange(64, 513, 32)
    out = []
    for _ in range(count):
        ny = int(rng.choice(sides))
        aspect = int(rng.choice([1, 2]))
        out.append(dict(
            nx=aspect * ny, ny=ny,
            Ra=float(10 ** rng.uniform(3, 6)), Da=float(10 ** rng.uniform(-4, -1)),
            porosity=float(rng.uniform(0.3, 0.9)), H=float(10 ** rng.uniform(0, 3)),
            gamma_sf=float(10 ** rng.uniform(-1, 2)), Pr=1.0, sigma=1.0,
            T_hot=1.0, T_cold=0.0, T_ref=0.5))
    return out


def fd_nodes(nx, ny, count, seed, margin=2):
    """Distinct interior nodes at distance >= margin from every wall, as
    flat indices y*nx + x."""
    rng = np.random.default_rng(seed)
    xs = np.arange(margin, nx - margin)
    ys = np.arange(margin, ny - margin)
    flat = (ys[:, None] * nx + xs[None, :]).reshape(-1)
    return np.sort(rng.choice(flat, size=count, replace=False))


def random_fields(nx, ny, seed, du=0.01, dT=0.3):
    """Smooth-ish random initial fields (rho, ux, uy, Tf, Ts) for parity
    tests that start away from rest."""
    rng = np.random.default_rng(seed)
    n = nx * ny
    return dict(rho=1.0 + 0.01 * rng.standard_normal(n), ux=du * rng.standard_normal(n),
                uy=du * rng.standard_normal(n), T_f=0.5 + dT * rng.uniform(-1, 1, n),
                T_s=0.5 + dT * rng.uniform(-1, 1, n))


RATE_KEYS = ("s_e", "s_eps", "s_q", "zeta_e", "zeta_nu", "eta_e", "eta_nu")


def random_params(seed, nx, ny):
    """Random but stable cavity parameters for brute-force parity.  The
    non-hydrodynamic relaxation rates (s_e, s_eps, s_q of Eq. 17; zeta_e,
    zeta_nu, eta_e, eta_nu of Eqs. 39-40) are drawn independently in
    [0.8, 1.9] and varpi in [0.2, 0.8], so that a rate applied to the wrong
    moment, or a varpi-dependent constant taken at the default 2/5, changes
    the result."""
    rng = np.random.default_rng(seed)
    d = dict(nx=nx, ny=ny, Ra=float(10 ** rng.uniform(3, 5)), Pr=float(rng.uniform(0.7, 2)),
             Da=float(10 ** rng.uniform(-3, -1)), porosity=float(rng.uniform(0.35, 0.9)),
             H=float(10 ** rng.uniform(0, 3)), gamma_sf=float(10 ** rng.uniform(-1, 1.5)),
             sigma=float(rng.uniform(0.5, 2)), J_e=float(rng.uniform(0.8, 1.5)),
             T_hot=1.0, T_cold=0.0, T_ref=0.5, Ma=0.1)
    rr = np.random.default_rng([seed, 7])  # a second stream: the draws above are unchanged
    for k in RATE_KEYS:
        d[k] = float(rr.uniform(0.8, 1.9))
    d["varpi"] = float(rr.uniform(0.2, 0.8))
    return d

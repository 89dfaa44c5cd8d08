"""Shared test plumbing: map one physical parameter dict onto the oracle's
record and the CUDA binding's record, and compare fields."""
import numpy as np

PHYS_KEYS = ("Ra", "Pr", "Da", "porosity", "H", "gamma_sf", "sigma", "J_e", "T_hot", "T_cold",
             "T_ref", "Ma", "F_phi", "d_p", "qf", "qs", "s_e", "s_eps", "s_q", "zeta_e",
             "zeta_nu", "eta_e", "eta_nu", "varpi", "ext_ax", "ext_ay", "nu_override",
             "hv_local", "Dp_over_L", "thermal_correction")


def phys(d):
    return {k: v for k, v in d.items() if k in PHYS_KEYS}


def oracle_for(cfg, phi=None, bc=0):
    from oracle import Oracle, OracleParams

    p = OracleParams.make(cfg["nx"], cfg["ny"], bc=bc, ergun_K=int(bool(cfg.get("ergun"))),
                          **phys(cfg))
    return Oracle(p, phi=phi)


def cavity_for(cfg, storage="f32", phi=None, bc=0):
    from paper_1608_04118_gb300.ltne import Cavity, LTNE_K_DARCY, LTNE_K_ERGUN

    return Cavity(cfg["nx"], cfg["ny"], storage=storage, bc=bc,
                  permeability=LTNE_K_ERGUN if cfg.get("ergun") else LTNE_K_DARCY,
                  porosity_field=1 if phi is not None else 0, **phys(cfg))


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def field_errors(gpu, orc):
    """rel-L2 of u (vector), T_f, T_s and rho between two field dicts."""
    u_g = np.stack([gpu["ux"], gpu["uy"]])
    u_o = np.stack([orc["ux"], orc["uy"]])
    return dict(u=rel_l2(u_g, u_o), Tf=rel_l2(gpu["Tf"], orc["Tf"]),
                Ts=rel_l2(gpu["Ts"], orc["Ts"]),
                rho=rel_l2(gpu["rho"] - 1.0, orc["rho"] - 1.0),
                rho_abs=float(np.abs(gpu["rho"] - orc["rho"]).max()))


def golden(name):
    """The "name = value" lines of tests/golden/<name>.txt as floats (the
    values the paper prints; each file cites its passage)."""
    import os

    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name + ".txt")
    out = {}
    with open(path) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = (t.strip() for t in line.split("=", 1))
                out[k] = float(v)
    return out

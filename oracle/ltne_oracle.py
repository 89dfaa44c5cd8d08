"""ctypes front end of the FP64 C oracle (``ltne_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
CPU-baseline leg of the benchmark, never by the product path.  The
parameter record below is this module's own; it is not shared with the CUDA
library's binding.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ltne_oracle.c")
_LIB = os.path.join(_HERE, "libltne_oracle.so")
_lock = threading.Lock()
_lib = None

BC_CAVITY, BC_PERIODIC, BC_CHANNEL = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle (real and complex-step variants) into one .so."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    flags = ["-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-std=gnu11"]
    tmp = _LIB + ".%d.tmp" % os.getpid()
    o1 = _LIB + ".%d.r.o" % os.getpid()
    o2 = _LIB + ".%d.c.o" % os.getpid()
    try:
        subprocess.run(["gcc", *flags, "-c", _SRC, "-o", o1], check=True)
        subprocess.run(["gcc", *flags, "-DORC_COMPLEX", "-c", _SRC, "-o", o2], check=True)
        subprocess.run(["gcc", "-shared", "-fopenmp", o1, o2, "-lm", "-o", tmp], check=True)
        os.replace(tmp, _LIB)
    finally:
        for f in (o1, o2, tmp):
            if os.path.exists(f):
                os.remove(f)
    return _LIB


class OracleParams(C.Structure):
    """Problem statement (Sec. 2 groups, Sec. 4 rates) for the oracle."""

    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("bc", C.c_int32), ("ergun_K", C.c_int32),
        ("Ra", C.c_double), ("Pr", C.c_double), ("Da", C.c_double), ("porosity", C.c_double),
        ("H", C.c_double), ("gamma_sf", C.c_double), ("sigma", C.c_double), ("J_e", C.c_double),
        ("T_hot", C.c_double), ("T_cold", C.c_double), ("T_ref", C.c_double), ("Ma", C.c_double),
        ("F_phi", C.c_double), ("d_p", C.c_double), ("qf", C.c_double), ("qs", C.c_double),
        ("s_e", C.c_double), ("s_eps", C.c_double), ("s_q", C.c_double),
        ("zeta_e", C.c_double), ("zeta_nu", C.c_double), ("eta_e", C.c_double),
        ("eta_nu", C.c_double), ("varpi", C.c_double),
        ("ext_ax", C.c_double), ("ext_ay", C.c_double), ("nu_override", C.c_double),
        ("hv_local", C.c_int32), ("thermal_correction", C.c_int32), ("Dp_over_L", C.c_double),
        ("L_ref", C.c_double),
    ]

    # Defaults: relaxation rates and varpi from Sec. 4; T_0 midway between
    # the wall temperatures; Ergun F_phi (negative value); Ma = 0.1.
    DEFAULTS = dict(
        bc=BC_CAVITY, ergun_K=0, Ra=1e4, Pr=1.0, Da=1e-2, porosity=0.6, H=10.0,
        gamma_sf=1.0, sigma=1.0, J_e=1.0, T_hot=1.0, T_cold=0.0, T_ref=0.5, Ma=0.1,
        F_phi=-1.0, d_p=0.0, qf=0.0, qs=0.0, s_e=1.1, s_eps=1.1, s_q=1.2,
        zeta_e=1.1, zeta_nu=1.1, eta_e=1.1, eta_nu=1.1, varpi=0.4,
        ext_ax=0.0, ext_ay=0.0, nu_override=0.0, hv_local=0, thermal_correction=0, Dp_over_L=0.0135,
        L_ref=0.0,
    )

    @classmethod
    def make(cls, nx, ny, **kw):
        v = dict(cls.DEFAULTS)
        unknown = set(kw) - set(v)
        if unknown:
            raise KeyError("unknown oracle parameter(s): %s" % sorted(unknown))
        v.update(kw)
        p = cls()
        p.nx, p.ny = int(nx), int(ny)
        for k, val in v.items():
            setattr(p, k, val)
        return p


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        P = C.POINTER(OracleParams)
        dp = C.POINTER(C.c_double)
        for pre in ("orc_", "orc_cs_"):
            getattr(lib, pre + "create").restype = C.c_void_p
            getattr(lib, pre + "create").argtypes = [P, dp]
            getattr(lib, pre + "destroy").argtypes = [C.c_void_p]
            getattr(lib, pre + "init").argtypes = [C.c_void_p, dp, dp, dp, dp, dp]
            getattr(lib, pre + "step").argtypes = [C.c_void_p, C.c_long]
            getattr(lib, pre + "get_step").restype = C.c_long
            getattr(lib, pre + "get_step").argtypes = [C.c_void_p]
            getattr(lib, pre + "macros").argtypes = [C.c_void_p, dp, dp, dp, dp, dp]
            getattr(lib, pre + "observables").argtypes = [C.c_void_p, dp]
            getattr(lib, pre + "objective").argtypes = [C.c_void_p, dp, dp]
            getattr(lib, pre + "get_pops").argtypes = [C.c_void_p, dp, dp, dp]
            getattr(lib, pre + "set_pops").argtypes = [C.c_void_p, dp, dp, dp]
        lib.orc_cs_perturb.argtypes = [C.c_void_p, C.c_int, C.c_double]
        lib.orc_derived.argtypes = [C.c_void_p, dp]
        lib.orc_medium.argtypes = [C.c_void_p, dp, dp]
        lib.orc_lattice_tables.argtypes = [dp] * 6
        lib.orc_node.argtypes = [C.c_void_p, C.c_int] + [dp] * 9
        lib.orc_equilibria.argtypes = [C.c_void_p] + [C.c_double] * 8 + [dp] * 5
        lib.orc_num_threads.restype = C.c_int
        lib.orc_set_num_threads.argtypes = [C.c_int]
        lib.orc_ergun_diameter.restype = C.c_double
        lib.orc_ergun_diameter.argtypes = [dp, C.c_long, C.c_double, C.c_double]
        _lib = lib
        return lib


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a, n=None):
    if a is None:
        return None
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None and a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's node loops from now on (timing only)."""
    _load().orc_set_num_threads(int(n))


def ergun_diameter(phi, L, Da) -> float:
    """Particle diameter giving mean(K)/L^2 = Da over the porosities phi."""
    a = _f64(phi)
    return float(_load().orc_ergun_diameter(_ptr(a), a.size, float(L), float(Da)))


def lattice_tables():
    """e (2x9), w (9), M, Minv (9x9), N, Ninv (5x5) as built by the oracle."""
    lib = _load()
    e = np.zeros(18); w = np.zeros(9); M = np.zeros(81); Mi = np.zeros(81)
    N = np.zeros(25); Ni = np.zeros(25)
    lib.orc_lattice_tables(_ptr(e), _ptr(w), _ptr(M), _ptr(Mi), _ptr(N), _ptr(Ni))
    return (e.reshape(2, 9).astype(int), w, M.reshape(9, 9), Mi.reshape(9, 9),
            N.reshape(5, 5), Ni.reshape(5, 5))


class Oracle:
    """One cavity (or periodic / channel test box) advanced by the oracle."""

    _pre = "orc_"

    def __init__(self, params: OracleParams, phi=None):
        self.lib = _load()
        self.p = params
        self.nx, self.ny = params.nx, params.ny
        self.nn = self.nx * self.ny
        self._phi = _f64(phi, self.nn)
        h = getattr(self.lib, self._pre + "create")(C.byref(params), _ptr(self._phi))
        if not h:
            raise ValueError("oracle rejected the parameters")
        self.h = C.c_void_p(h)

    def _fn(self, name):
        return getattr(self.lib, self._pre + name)

    def close(self):
        if self.h:
            self._fn("destroy")(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, rho=None, ux=None, uy=None, Tf=None, Ts=None):
        arrs = [_f64(a, self.nn) for a in (rho, ux, uy, Tf, Ts)]
        self._fn("init")(self.h, *[_ptr(a) for a in arrs])
        return self

    def step(self, n: int):
        self._fn("step")(self.h, int(n))
        return self

    @property
    def steps(self) -> int:
        return int(self._fn("get_step")(self.h))

    def macros(self):
        """dict of (ny, nx) arrays: rho, ux, uy, Tf, Ts of the current state."""
        out = {k: np.zeros(self.nn) for k in ("rho", "ux", "uy", "Tf", "Ts")}
        self._fn("macros")(self.h, *[_ptr(out[k]) for k in ("rho", "ux", "uy", "Tf", "Ts")])
        return {k: v.reshape(self.ny, self.nx) for k, v in out.items()}

    OBS_KEYS = ("Nu_f_hot", "Nu_s_hot", "Nu_f_cold", "Nu_s_cold", "mass", "energy",
                "max_u", "max_dT", "mean_Tf", "mean_Ts", "Fo", "nonfinite")

    def observables(self):
        out = np.zeros(12)
        self._fn("observables")(self.h, _ptr(out))
        return dict(zip(self.OBS_KEYS, out.tolist()))

    def objective(self):
        re, im = C.c_double(), C.c_double()
        self._fn("objective")(self.h, C.byref(re), C.byref(im))
        return re.value, im.value

    def get_pops(self):
        """(f (ny,nx,9), gf (ny,nx,5), gs (ny,nx,5)) of the current state."""
        f = np.zeros(9 * self.nn); gf = np.zeros(5 * self.nn); gs = np.zeros(5 * self.nn)
        self._fn("get_pops")(self.h, _ptr(f), _ptr(gf), _ptr(gs))
        return (f.reshape(self.ny, self.nx, 9), gf.reshape(self.ny, self.nx, 5),
                gs.reshape(self.ny, self.nx, 5))

    def set_pops(self, f, gf, gs):
        f = _f64(f, 9 * self.nn); gf = _f64(gf, 5 * self.nn); gs = _f64(gs, 5 * self.nn)
        self._fn("set_pops")(self.h, _ptr(f), _ptr(gf), _ptr(gs))

    # --- real-only introspection used by the pins ---
    DERIVED_KEYS = ("L", "nu_f", "nu_e", "alpha_f", "alpha_s", "gbeta", "s_nu", "zeta_alpha",
                    "eta_alpha", "d_ergun", "csT2", "hv_over_rhoc_f", "s_e", "s_eps", "s_q", "cs2")

    def derived(self):
        out = np.zeros(16)
        self.lib.orc_derived(self.h, _ptr(out))
        return dict(zip(self.DERIVED_KEYS, out.tolist()))

    def medium(self):
        K = np.zeros(self.nn); F = np.zeros(self.nn)
        self.lib.orc_medium(self.h, _ptr(K), _ptr(F))
        return K.reshape(self.ny, self.nx), F.reshape(self.ny, self.nx)

    def node(self, n, f, gf, gs):
        """Collide one node's populations with node n's medium.

        Returns (f*, gf*, gs*, macro dict, S~, m^eq)."""
        f = _f64(f, 9); gf = _f64(gf, 5); gs = _f64(gs, 5)
        fo = np.zeros(9); gfo = np.zeros(5); gso = np.zeros(5)
        mac = np.zeros(11); St = np.zeros(9); me = np.zeros(9)
        self.lib.orc_node(self.h, int(n), _ptr(f), _ptr(gf), _ptr(gs), _ptr(fo), _ptr(gfo),
                          _ptr(gso), _ptr(mac), _ptr(St), _ptr(me))
        keys = ("rho", "ux", "uy", "Tf", "Ts", "Gx", "Gy", "Fx", "Fy", "a", "b")
        return fo, gfo, gso, dict(zip(keys, mac.tolist())), St, me

    def equilibria(self, rho, ux, uy, Tf, Ts, phi, Fx=0.0, Fy=0.0):
        fe = np.zeros(9); gfe = np.zeros(5); gse = np.zeros(5); me = np.zeros(9); S = np.zeros(9)
        self.lib.orc_equilibria(self.h, rho, ux, uy, Tf, Ts, phi, Fx, Fy, _ptr(fe), _ptr(gfe),
                                _ptr(gse), _ptr(me), _ptr(S))
        return fe, gfe, gse, me, S


class ComplexOracle(Oracle):
    """Complex-step variant: exact directional derivatives of the objective."""

    _pre = "orc_cs_"

    def perturb(self, node: int, h: float):
        """node >= 0: phi[node] += i h;  node == -1: H += i h.  Call before init."""
        self.lib.orc_cs_perturb(self.h, int(node), float(h))
        return self

"""Python binding of the ``ltne_*`` C ABI (include/ltne.h).

Argument marshalling only: every step of the method runs in the CUDA
kernels of ``libltne.so``.  PyTorch provides the device workspace and the
stream.  If the library has not been built this module raises on load; there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libltne.so")

LTNE_OK = 0
LTNE_ERR_INVALID_ARG = 1
LTNE_ERR_UNSTABLE_TAU = 2
LTNE_ERR_CUDA = 3
LTNE_ERR_NONFINITE = 4
LTNE_ERR_TIMEOUT = 5
LTNE_ERR_STATE = 6
LTNE_ERR_WORKSPACE = 7

LTNE_F64, LTNE_F32, LTNE_F16DEV, LTNE_BF16DEV = 0, 1, 2, 3
LTNE_BC_CAVITY, LTNE_BC_PERIODIC, LTNE_BC_CHANNEL = 0, 1, 2
LTNE_ADJ_AUTO, LTNE_ADJ_ONE_WAVE, LTNE_ADJ_CAPPED = 0, 1, 2
LTNE_HOST_IO_AUTO, LTNE_HOST_IO_STAGED, LTNE_HOST_IO_DIRECT = 0, 1, 2
LTNE_K_DARCY, LTNE_K_ERGUN = 0, 1

STORAGE = {"f64": LTNE_F64, "f32": LTNE_F32, "f16": LTNE_F16DEV, "bf16": LTNE_BF16DEV}


class LtneError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        msg = _lib().ltne_error_string(code).decode() if _lib_obj else "code %d" % code
        super().__init__("%s%s" % (what + ": " if what else "", msg))


class ltne_params(C.Structure):
    """Mirror of ``struct ltne_params`` (field order and types as in ltne.h)."""

    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("storage", C.c_int32), ("bc", C.c_int32),
        ("permeability", C.c_int32), ("porosity_field", C.c_int32),
        ("Ra", C.c_double), ("Pr", C.c_double), ("Da", C.c_double), ("porosity", C.c_double),
        ("H", C.c_double), ("gamma_sf", C.c_double), ("sigma", C.c_double), ("J_e", C.c_double),
        ("T_hot", C.c_double), ("T_cold", C.c_double), ("T_ref", C.c_double), ("Ma", C.c_double),
        ("F_phi", C.c_double), ("d_p", C.c_double), ("qf", C.c_double), ("qs", C.c_double),
        ("s_e", C.c_double), ("s_eps", C.c_double), ("s_q", C.c_double),
        ("zeta_e", C.c_double), ("zeta_nu", C.c_double), ("eta_e", C.c_double),
        ("eta_nu", C.c_double), ("varpi", C.c_double),
        ("ext_ax", C.c_double), ("ext_ay", C.c_double), ("nu_override", C.c_double),
        ("hv_local", C.c_int32), ("thermal_correction", C.c_int32), ("Dp_over_L", C.c_double),
    ]


class ltne_obs(C.Structure):
    _fields_ = [
        ("Nu_f_hot", C.c_double), ("Nu_s_hot", C.c_double), ("Nu_f_cold", C.c_double),
        ("Nu_s_cold", C.c_double), ("residual", C.c_double), ("mass", C.c_double),
        ("energy", C.c_double), ("max_u", C.c_double), ("max_dT", C.c_double),
        ("mean_Tf", C.c_double), ("mean_Ts", C.c_double), ("Fo", C.c_double),
        ("step", C.c_int64), ("nonfinite", C.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib_obj = None
_lock = threading.Lock()

# Every symbol include/ltne.h declares, with (restype, argtypes).
_vp, _dp = C.c_void_p, C.POINTER(C.c_double)
SIGNATURES = {
    "ltne_default_params": (None, [C.POINTER(ltne_params), C.c_int32, C.c_int32]),
    "ltne_create": (C.c_int, [C.POINTER(ltne_params), _vp, C.POINTER(_vp)]),
    "ltne_workspace_bytes": (C.c_size_t, [_vp]),
    "ltne_bind_workspace": (C.c_int, [_vp, _vp, C.c_size_t]),
    "ltne_set_fields": (C.c_int, [_vp, _dp, _dp, _dp, _dp, _dp, _dp]),
    "ltne_step": (C.c_int, [_vp, C.c_int64]),
    "ltne_observables": (C.c_int, [_vp, C.POINTER(ltne_obs)]),
    "ltne_get_fields": (C.c_int, [_vp, _dp, _dp, _dp, _dp, _dp]),
    "ltne_state_bytes": (C.c_size_t, [_vp]),
    "ltne_get_state": (C.c_int, [_vp, _vp, C.c_size_t]),
    "ltne_set_state": (C.c_int, [_vp, _vp, C.c_size_t]),
    "ltne_launch_count": (C.c_int64, [_vp]),
    "ltne_set_schedule": (C.c_int, [_vp, C.c_int32, C.c_int32, C.c_int32]),
    "ltne_get_schedule": (C.c_int, [_vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                    C.POINTER(C.c_int32)]),
    "ltne_set_staging": (C.c_int, [_vp, C.c_int32]),
    "ltne_slab_scratch_bytes": (C.c_size_t, [_vp, C.c_int32]),
    "ltne_step_slabs": (C.c_int, [_vp, C.c_int32, C.c_int64, _vp, C.c_size_t]),
    "ltne_check_bounded_wait": (C.c_int, [_vp, C.c_int32, C.POINTER(C.c_int32)]),
    "ltne_get_staging": (C.c_int, [_vp, C.POINTER(C.c_int32)]),
    "ltne_set_host_io": (C.c_int, [_vp, C.c_int32]),
    "ltne_get_host_io": (C.c_int, [_vp, C.POINTER(C.c_int32)]),
    "ltne_observables_static": (C.c_int, [C.POINTER(ltne_params), _vp, C.c_int64, _vp, C.c_int64,
                                          _vp, C.POINTER(ltne_obs)]),
    "ltne_set_adjoint_schedule": (C.c_int, [_vp, C.c_int32]),
    "ltne_get_adjoint_schedule": (C.c_int, [_vp, C.POINTER(C.c_int32)]),
    "ltne_adjoint_workspace_bytes": (C.c_size_t, [_vp, C.c_int64, C.c_int32]),
    "ltne_adjoint": (C.c_int, [_vp, _dp, _dp, _dp, _dp, C.c_int64, C.c_int32, _vp, C.c_size_t, _vp,
                               _dp, _dp]),
    "ltne_destroy": (None, [_vp]),
    "ltne_error_string": (C.c_char_p, [C.c_int]),
    "ltne_slab_rows": (C.c_int, [C.c_int32, C.c_int32, C.c_int32] + [C.POINTER(C.c_int32)] * 4),
    "ltne_create_slab": (C.c_int, [C.POINTER(ltne_params), C.c_int32, C.c_int32, _vp,
                                   C.POINTER(_vp)]),
    "ltne_halo_buffers": (C.c_int, [_vp] + [C.POINTER(_vp)] * 4 + [C.POINTER(C.c_size_t)]),
    "ltne_step_slab": (C.c_int, [_vp, C.c_int32]),
    "ltne_halo_pack": (C.c_int, [_vp]),
    "ltne_halo_unpack": (C.c_int, [_vp]),
    "ltne_slab_accumulators": (C.c_int, [_vp, _dp, C.c_int32]),
    "ltne_accumulators_combine": (C.c_int, [_dp, _dp, C.c_int32]),
    "ltne_observables_from_accumulators": (C.c_int, [C.POINTER(ltne_params), C.c_int64,
                                                     C.c_int32, _dp, C.c_int32,
                                                     C.POINTER(ltne_obs)]),
    "ltne_ergun_diameter": (C.c_int, [_dp, C.c_int64, C.c_double, C.c_double, _dp]),
    "ltne_batch_create": (C.c_int, [C.POINTER(ltne_params), C.c_int32, _vp, C.POINTER(_vp)]),
    "ltne_batch_workspace_bytes": (C.c_size_t, [_vp]),
    "ltne_batch_nodes": (C.c_int64, [_vp]),
    "ltne_batch_bind_workspace": (C.c_int, [_vp, _vp, C.c_size_t]),
    "ltne_batch_set_schedule": (C.c_int, [_vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32]),
    "ltne_batch_set_fields": (C.c_int, [_vp]),
    "ltne_batch_step": (C.c_int, [_vp, C.c_int64]),
    "ltne_batch_observables": (C.c_int, [_vp, C.POINTER(ltne_obs)]),
    "ltne_batch_get_fields": (C.c_int, [_vp, C.c_int32, _dp, _dp, _dp, _dp, _dp]),
    "ltne_batch_launch_count": (C.c_int64, [_vp]),
    "ltne_batch_destroy": (None, [_vp]),
}


def _lib():
    global _lib_obj
    with _lock:
        if _lib_obj is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(
                    "libltne.so is not built (%s); run __graft_entry__.build() or "
                    "python -m paper_1608_04118_gb300.build -- there is no CPU fallback" % LIB_PATH)
            lib = C.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib_obj = lib
        return _lib_obj


def load():
    """Load libltne.so (raises ImportError if it is missing)."""
    return _lib()


def _check(code, what):
    if code != LTNE_OK:
        raise LtneError(code, what)


def _f64(a, n):
    if a is None:
        return None
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64)).reshape(-1)
    if a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_dp)


# ---- thin wrappers with the C names ---------------------------------------

def ltne_default_params(nx, ny, **overrides) -> ltne_params:
    p = ltne_params()
    _lib().ltne_default_params(C.byref(p), int(nx), int(ny))
    names = {f for f, _ in ltne_params._fields_}
    for k, v in overrides.items():
        if k == "storage" and isinstance(v, str):
            v = STORAGE[v]
        if k not in names:
            raise KeyError("unknown parameter %r" % k)
        setattr(p, k, v)
    return p


def ltne_create(params: ltne_params, stream=None):
    h = _vp()
    s = _vp(int(stream) if stream is not None else 0)
    _check(_lib().ltne_create(C.byref(params), s, C.byref(h)), "ltne_create")
    return h


def ltne_workspace_bytes(h) -> int:
    return int(_lib().ltne_workspace_bytes(h))


def ltne_bind_workspace(h, device_ptr: int, nbytes: int):
    _check(_lib().ltne_bind_workspace(h, _vp(int(device_ptr)), int(nbytes)), "ltne_bind_workspace")


def ltne_set_fields(h, nn, porosity=None, rho=None, ux=None, uy=None, T_f=None, T_s=None):
    arrs = [_f64(a, nn) for a in (porosity, rho, ux, uy, T_f, T_s)]
    _check(_lib().ltne_set_fields(h, *[_ptr(a) for a in arrs]), "ltne_set_fields")


def ltne_step(h, n: int):
    _check(_lib().ltne_step(h, int(n)), "ltne_step")


def ltne_observables(h, allow_nonfinite=False) -> dict:
    o = ltne_obs()
    rc = _lib().ltne_observables(h, C.byref(o))
    if not (rc == LTNE_OK or (allow_nonfinite and rc == LTNE_ERR_NONFINITE)):
        raise LtneError(rc, "ltne_observables")
    return o.as_dict()


FIELD_KEYS = ("rho", "ux", "uy", "Tf", "Ts")


def ltne_get_fields(h, nx, ny, out=None) -> dict:
    """The five fields as (ny, nx) float64 arrays; ``out`` may hold arrays of
    that shape and type (C-contiguous) to be filled instead of new ones."""
    if out is None:
        out = {k: np.empty((ny, nx)) for k in FIELD_KEYS}
    else:
        for k in FIELD_KEYS:
            a = out[k]
            if (not isinstance(a, np.ndarray) or a.dtype != np.float64 or a.shape != (ny, nx)
                    or not a.flags.c_contiguous or not a.flags.writeable):
                raise ValueError("out[%r] must be a writeable C-contiguous float64 array of "
                                 "shape (%d, %d)" % (k, ny, nx))
    _check(_lib().ltne_get_fields(h, *[_ptr(out[k]) for k in FIELD_KEYS]), "ltne_get_fields")
    return {k: out[k] for k in FIELD_KEYS}


def ltne_state_bytes(h) -> int:
    return int(_lib().ltne_state_bytes(h))


def ltne_get_state(h) -> bytes:
    n = ltne_state_bytes(h)
    buf = (C.c_char * n)()
    _check(_lib().ltne_get_state(h, C.cast(buf, _vp), n), "ltne_get_state")
    return bytes(buf)


def ltne_set_state(h, blob: bytes):
    buf = C.create_string_buffer(blob, len(blob))
    _check(_lib().ltne_set_state(h, C.cast(buf, _vp), len(blob)), "ltne_set_state")


def ltne_launch_count(h) -> int:
    return int(_lib().ltne_launch_count(h))


def ltne_set_schedule(h, block_x, block_y, nodes_per_thread):
    _check(_lib().ltne_set_schedule(h, int(block_x), int(block_y), int(nodes_per_thread)),
           "ltne_set_schedule")


def ltne_set_staging(h, staged):
    _check(_lib().ltne_set_staging(h, int(staged)), "ltne_set_staging")


def ltne_slab_scratch_bytes(h, nslabs) -> int:
    return int(_lib().ltne_slab_scratch_bytes(h, int(nslabs)))


def ltne_step_slabs(h, nslabs, n, scratch_ptr, nbytes):
    _check(_lib().ltne_step_slabs(h, int(nslabs), int(n), _vp(int(scratch_ptr)), int(nbytes)),
           "ltne_step_slabs")


def ltne_check_bounded_wait(stream_ptr, spins) -> int:
    v = C.c_int32()
    _check(_lib().ltne_check_bounded_wait(_vp(int(stream_ptr)), int(spins), C.byref(v)),
           "ltne_check_bounded_wait")
    return v.value


def ltne_set_adjoint_schedule(h, mode):
    _check(_lib().ltne_set_adjoint_schedule(h, int(mode)), "ltne_set_adjoint_schedule")


def ltne_get_adjoint_schedule(h) -> int:
    v = C.c_int32()
    _check(_lib().ltne_get_adjoint_schedule(h, C.byref(v)), "ltne_get_adjoint_schedule")
    return v.value


def ltne_get_staging(h) -> int:
    v = C.c_int32()
    _check(_lib().ltne_get_staging(h, C.byref(v)), "ltne_get_staging")
    return v.value


def ltne_set_host_io(h, mode):
    _check(_lib().ltne_set_host_io(h, int(mode)), "ltne_set_host_io")


def ltne_get_host_io(h) -> int:
    v = C.c_int32()
    _check(_lib().ltne_get_host_io(h, C.byref(v)), "ltne_get_host_io")
    return v.value


def ltne_get_schedule(h):
    bx, by, npt = C.c_int32(), C.c_int32(), C.c_int32()
    _check(_lib().ltne_get_schedule(h, C.byref(bx), C.byref(by), C.byref(npt)),
           "ltne_get_schedule")
    return bx.value, by.value, npt.value


def ltne_adjoint_workspace_bytes(h, n_steps, segment) -> int:
    return int(_lib().ltne_adjoint_workspace_bytes(h, int(n_steps), int(segment)))


def ltne_adjoint(h, nn, porosity, n_steps, segment, adj_ptr, adj_bytes, dJ_dphi_ptr,
                 rho=None, T_f=None, T_s=None):
    """Returns (J, dJ/dH); dJ/dphi is written to the device buffer."""
    arrs = [_f64(a, nn) for a in (porosity, rho, T_f, T_s)]
    J, dH = C.c_double(), C.c_double()
    _check(_lib().ltne_adjoint(h, *[_ptr(a) for a in arrs], int(n_steps), int(segment),
                               _vp(int(adj_ptr)), int(adj_bytes),
                               _vp(int(dJ_dphi_ptr)) if dJ_dphi_ptr else None,
                               C.byref(J), C.byref(dH)), "ltne_adjoint")
    return J.value, dH.value


def ltne_destroy(h):
    if h:
        _lib().ltne_destroy(h)


def ltne_error_string(code: int) -> str:
    return _lib().ltne_error_string(int(code)).decode()


LTNE_NACC = 18


def ltne_slab_rows(ny, nslabs, index):
    """(y0, rows, halo_lo, halo_hi) of slab `index` of `nslabs`."""
    v = [C.c_int32() for _ in range(4)]
    _check(_lib().ltne_slab_rows(int(ny), int(nslabs), int(index), *[C.byref(x) for x in v]),
           "ltne_slab_rows")
    return tuple(x.value for x in v)


def ltne_create_slab(params: ltne_params, nslabs, index, stream=None):
    h = _vp()
    s = _vp(int(stream) if stream is not None else 0)
    _check(_lib().ltne_create_slab(C.byref(params), int(nslabs), int(index), s, C.byref(h)),
           "ltne_create_slab")
    return h


def ltne_halo_buffers(h):
    """(send_lo, send_hi, recv_lo, recv_hi, bytes): device addresses (None
    on a side without a neighbour) and the message size."""
    v = [_vp() for _ in range(4)]
    nb = C.c_size_t()
    _check(_lib().ltne_halo_buffers(h, *[C.byref(x) for x in v], C.byref(nb)),
           "ltne_halo_buffers")
    return tuple(x.value for x in v) + (nb.value,)


def ltne_step_slab(h, write_macros):
    _check(_lib().ltne_step_slab(h, int(write_macros)), "ltne_step_slab")


def ltne_halo_pack(h):
    _check(_lib().ltne_halo_pack(h), "ltne_halo_pack")


def ltne_halo_unpack(h):
    _check(_lib().ltne_halo_unpack(h), "ltne_halo_unpack")


def ltne_slab_accumulators(h) -> np.ndarray:
    acc = np.zeros(LTNE_NACC)
    _check(_lib().ltne_slab_accumulators(h, _ptr(acc), LTNE_NACC), "ltne_slab_accumulators")
    return acc


def ltne_accumulators_combine(acc, other) -> np.ndarray:
    a = np.array(acc, dtype=np.float64)
    b = _f64(other, LTNE_NACC)
    _check(_lib().ltne_accumulators_combine(_ptr(a), _ptr(b), LTNE_NACC),
           "ltne_accumulators_combine")
    return a


def ltne_observables_from_accumulators(params: ltne_params, step, have_prev, acc,
                                       allow_nonfinite=False) -> dict:
    a = _f64(acc, LTNE_NACC)
    o = ltne_obs()
    rc = _lib().ltne_observables_from_accumulators(C.byref(params), int(step), int(have_prev),
                                                   _ptr(a), LTNE_NACC, C.byref(o))
    if not (rc == LTNE_OK or (allow_nonfinite and rc == LTNE_ERR_NONFINITE)):
        raise LtneError(rc, "ltne_observables_from_accumulators")
    return o.as_dict()


def ltne_ergun_diameter(porosity, L, Da) -> float:
    a = np.ascontiguousarray(np.asarray(porosity, dtype=np.float64)).reshape(-1)
    d = C.c_double()
    _check(_lib().ltne_ergun_diameter(_ptr(a), a.size, float(L), float(Da), C.byref(d)),
           "ltne_ergun_diameter")
    return d.value


# ---- convenience object ----------------------------------------------------

class Cavity:
    """One lattice on the current CUDA device with a torch-owned workspace.

    ``Cavity(nx, ny, storage="f32", Ra=1e6, ...)`` takes any ltne_params
    field as a keyword.  All device work runs on the current torch stream
    unless ``stream`` is given.
    """

    def __init__(self, nx, ny, stream=None, device=None, **params):
        import torch

        self.nx, self.ny = int(nx), int(ny)
        self.params = ltne_default_params(nx, ny, **params)
        dev = torch.device(device) if device is not None else torch.device("cuda",
                                                                          torch.cuda.current_device())
        if stream is None:
            stream = torch.cuda.current_stream(dev)
        self.stream = stream
        self.h = ltne_create(self.params, stream.cuda_stream)
        nbytes = ltne_workspace_bytes(self.h)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        ltne_bind_workspace(self.h, self.workspace.data_ptr(), nbytes)

    @property
    def nodes(self):
        return self.nx * self.ny

    @property
    def storage(self):
        """Population storage type: "f64", "f32", "f16" or "bf16"."""
        return {v: k for k, v in STORAGE.items()}[int(self.params.storage)]

    def set_fields(self, porosity=None, rho=None, ux=None, uy=None, T_f=None, T_s=None):
        ltne_set_fields(self.h, self.nodes, porosity, rho, ux, uy, T_f, T_s)
        return self

    def step(self, n):
        ltne_step(self.h, n)
        return self

    def observables(self, allow_nonfinite=False):
        return ltne_observables(self.h, allow_nonfinite)

    def fields(self, out=None):
        """The fields as (ny, nx) float64 arrays (into ``out`` if given)."""
        return ltne_get_fields(self.h, self.nx, self.ny, out)

    def get_state(self):
        return ltne_get_state(self.h)

    def set_state(self, blob):
        ltne_set_state(self.h, blob)
        return self

    @property
    def launches(self):
        return ltne_launch_count(self.h)

    def set_schedule(self, block_x, block_y, nodes_per_thread):
        """Block shape and nodes per thread (1, or 2 in paired FP32) of the
        step kernel."""
        ltne_set_schedule(self.h, block_x, block_y, nodes_per_thread)
        return self

    @property
    def schedule(self):
        return ltne_get_schedule(self.h)

    def step_slabs(self, nslabs, n):
        """Advance n steps as nslabs row slabs with halo exchanges (the same
        bits as step(n)); the slab buffers are a temporary torch tensor."""
        import torch

        nb = ltne_slab_scratch_bytes(self.h, nslabs)
        if nb == 0:
            raise LtneError(LTNE_ERR_INVALID_ARG, "ltne_slab_scratch_bytes")
        buf = torch.empty(nb + 256, dtype=torch.uint8, device=self.workspace.device)
        ptr = (buf.data_ptr() + 255) // 256 * 256
        ltne_step_slabs(self.h, nslabs, n, ptr, nb)
        self.stream.synchronize()  # the slab buffers are released on return
        return self

    def set_staging(self, staged):
        """Step from TMA-staged shared-memory tiles (1) or direct loads (0)."""
        ltne_set_staging(self.h, staged)
        return self

    @property
    def staging(self):
        return ltne_get_staging(self.h)

    def set_host_io(self, mode):
        """How set_fields / fields move host arrays: LTNE_HOST_IO_AUTO,
        _STAGED (pinned buffers, host conversion) or _DIRECT (kernels read
        and write the host arrays)."""
        ltne_set_host_io(self.h, mode)
        return self

    @property
    def host_io(self):
        """The host I/O form in use (LTNE_HOST_IO_STAGED or _DIRECT)."""
        return ltne_get_host_io(self.h)

    def set_adjoint_schedule(self, mode):
        """Register budget of the adjoint's transposed collision: 0 by lattice
        size, 1 all registers (one wave), 2 capped (64 registers)."""
        ltne_set_adjoint_schedule(self.h, mode)
        return self

    @property
    def adjoint_schedule(self):
        return ltne_get_adjoint_schedule(self.h)

    def adjoint(self, porosity, n_steps, segment=None, rho=None, T_f=None, T_s=None):
        """Run n_steps from the given initial fields (fluid at rest) and return
        (J, dJ/dphi as a (ny, nx) device tensor, dJ/dH) with J = (Nu_f,hot +
        Nu_s,hot)/2 at the last step.  segment defaults to ceil(sqrt(n))."""
        import math

        import torch

        if segment is None:
            segment = max(1, int(math.ceil(math.sqrt(n_steps))))
        nbytes = ltne_adjoint_workspace_bytes(self.h, n_steps, segment)
        ws = torch.empty(nbytes, dtype=torch.uint8, device=self.workspace.device)
        dt = torch.float64 if self.params.storage == LTNE_F64 else torch.float32
        g = torch.empty((self.ny, self.nx), dtype=dt, device=self.workspace.device)
        J, dH = ltne_adjoint(self.h, self.nodes, porosity, n_steps, segment, ws.data_ptr(), nbytes,
                             g.data_ptr(), rho=rho, T_f=T_f, T_s=T_s)
        return J, g, dH

    def close(self):
        if getattr(self, "h", None):
            ltne_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SlabCavity:
    """One row slab of a cavity, advanced by this process, on the current
    CUDA device.  ``SlabCavity(nx, ny, nslabs, index, **params)``: nx, ny and
    the parameters describe the whole cavity.  The halo exchange between
    steps is the caller's (``paper_1608_04118_gb300.slabs`` moves it with
    torch.distributed)."""

    def __init__(self, nx, ny, nslabs, index, stream=None, device=None, **params):
        import torch

        self.nx, self.ny_global = int(nx), int(ny)
        self.nslabs, self.index = int(nslabs), int(index)
        self.params = ltne_default_params(nx, ny, **params)
        self.y0, self.rows, self.halo_lo, self.halo_hi = ltne_slab_rows(ny, nslabs, index)
        self.ny = self.rows + self.halo_lo + self.halo_hi  # local rows
        dev = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        if stream is None:
            stream = torch.cuda.current_stream(dev)
        self.stream = stream
        self.h = ltne_create_slab(self.params, nslabs, index, stream.cuda_stream)
        nbytes = ltne_workspace_bytes(self.h)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        ltne_bind_workspace(self.h, self.workspace.data_ptr(), nbytes)
        self.buffers = ltne_halo_buffers(self.h)
        self.have_prev = False

    @property
    def local_rows(self):
        """Rows [a, b) of the cavity that the local lattice covers (halos
        included)."""
        return self.y0 - self.halo_lo, self.y0 + self.rows + self.halo_hi

    def local(self, field):
        """The local lattice's part of a whole-cavity field (ny x nx)."""
        if field is None:
            return None
        a, b = self.local_rows
        return np.asarray(field, dtype=np.float64).reshape(self.ny_global, self.nx)[a:b]

    def set_fields(self, porosity=None, rho=None, ux=None, uy=None, T_f=None, T_s=None):
        """Initial fields given for the WHOLE cavity (any may be None)."""
        ltne_set_fields(self.h, self.nx * self.ny, *[self.local(f) for f in
                                                      (porosity, rho, ux, uy, T_f, T_s)])
        self.have_prev = False
        return self

    def step(self, write_macros):
        ltne_step_slab(self.h, write_macros)
        return self

    def pack(self):
        ltne_halo_pack(self.h)
        return self

    def unpack(self):
        ltne_halo_unpack(self.h)
        return self

    def accumulators(self):
        return ltne_slab_accumulators(self.h)

    def fields(self):
        """Macroscopic fields of the slab's computed rows (rows x nx)."""
        f = ltne_get_fields(self.h, self.nx, self.ny)
        a = self.halo_lo
        return {k: v[a:a + self.rows] for k, v in f.items()}

    def get_state(self):
        return ltne_get_state(self.h)

    def set_state(self, blob):
        ltne_set_state(self.h, blob)
        return self

    @property
    def launches(self):
        return ltne_launch_count(self.h)

    def close(self):
        if getattr(self, "h", None):
            ltne_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- batched form -----------------------------------------------------------

def ltne_batch_create(params_list, stream=None):
    arr = (ltne_params * len(params_list))(*params_list)
    h = _vp()
    s = _vp(int(stream) if stream is not None else 0)
    _check(_lib().ltne_batch_create(arr, len(params_list), s, C.byref(h)), "ltne_batch_create")
    return h


def ltne_batch_workspace_bytes(b) -> int:
    return int(_lib().ltne_batch_workspace_bytes(b))


def ltne_batch_nodes(b) -> int:
    return int(_lib().ltne_batch_nodes(b))


def ltne_batch_bind_workspace(b, device_ptr: int, nbytes: int):
    _check(_lib().ltne_batch_bind_workspace(b, _vp(int(device_ptr)), int(nbytes)),
           "ltne_batch_bind_workspace")


def ltne_batch_set_schedule(b, tile_x, tile_y, blocks, nodes_per_thread=1):
    _check(_lib().ltne_batch_set_schedule(b, int(tile_x), int(tile_y), int(blocks),
                                          int(nodes_per_thread)),
           "ltne_batch_set_schedule")


def ltne_batch_set_fields(b):
    _check(_lib().ltne_batch_set_fields(b), "ltne_batch_set_fields")


def ltne_batch_step(b, n):
    _check(_lib().ltne_batch_step(b, int(n)), "ltne_batch_step")


def ltne_batch_observables(b, count, allow_nonfinite=False):
    out = (ltne_obs * count)()
    rc = _lib().ltne_batch_observables(b, out)
    if not (rc == LTNE_OK or (allow_nonfinite and rc == LTNE_ERR_NONFINITE)):
        raise LtneError(rc, "ltne_batch_observables")
    return [o.as_dict() for o in out]


def ltne_batch_get_fields(b, index, nx, ny):
    out = {k: np.empty(nx * ny) for k in ("rho", "ux", "uy", "Tf", "Ts")}
    _check(_lib().ltne_batch_get_fields(b, int(index),
                                        *[_ptr(out[k]) for k in ("rho", "ux", "uy", "Tf", "Ts")]),
           "ltne_batch_get_fields")
    return {k: v.reshape(ny, nx) for k, v in out.items()}


def ltne_batch_launch_count(b) -> int:
    return int(_lib().ltne_batch_launch_count(b))


def ltne_batch_destroy(b):
    if b:
        _lib().ltne_batch_destroy(b)


class Batch:
    """Many independent FP32 cavities advanced together on one device.

    ``Batch([dict(nx=.., ny=.., Ra=.., ...), ...])``: each dict takes
    ltne_params fields (storage, bc and porosity_field are fixed)."""

    def __init__(self, cavities, stream=None, device=None):
        import torch

        self.shapes = [(int(c["nx"]), int(c["ny"])) for c in cavities]
        plist = []
        for c in cavities:
            kw = {k: v for k, v in c.items() if k not in ("nx", "ny")}
            plist.append(ltne_default_params(c["nx"], c["ny"], storage=LTNE_F32, **kw))
        dev = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        if stream is None:
            stream = torch.cuda.current_stream(dev)
        self.stream = stream
        self.b = ltne_batch_create(plist, stream.cuda_stream)
        nbytes = ltne_batch_workspace_bytes(self.b)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        ltne_batch_bind_workspace(self.b, self.workspace.data_ptr(), nbytes)
        self.schedule = (128, 2, 0, 1)

    @property
    def count(self):
        return len(self.shapes)

    @property
    def nodes(self):
        return ltne_batch_nodes(self.b)

    def set_schedule(self, tile_x, tile_y, blocks, nodes_per_thread=1):
        ltne_batch_set_schedule(self.b, tile_x, tile_y, blocks, nodes_per_thread)
        self.schedule = (tile_x, tile_y, blocks, nodes_per_thread)
        return self

    def set_fields(self):
        ltne_batch_set_fields(self.b)
        return self

    def step(self, n):
        ltne_batch_step(self.b, n)
        return self

    def observables(self, allow_nonfinite=False):
        return ltne_batch_observables(self.b, self.count, allow_nonfinite)

    def fields(self, index):
        nx, ny = self.shapes[index]
        return ltne_batch_get_fields(self.b, index, nx, ny)

    @property
    def launches(self):
        return ltne_batch_launch_count(self.b)

    def close(self):
        if getattr(self, "b", None):
            ltne_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

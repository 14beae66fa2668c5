"""ctypes binding of libpetto's C ABI (include/petto.h).  Argument marshalling only:
every step of the PeTTO path runs in the CUDA kernels of the shared library.

Functions keep the C names (``petto_create``, ``petto_pt_solve``, ...).  They raise
``PettoError`` when the library returns a status other than PETTO_OK (PETTO_ENOTCONV is
returned, not raised, by the solve calls).  The library must exist: there is no CPU
fallback, and loading fails loudly when it cannot be built or opened.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

PETTO_OK, PETTO_EINVAL, PETTO_ENOMEM, PETTO_ECUDA, PETTO_ENOTCONV, PETTO_EDIVERGED, PETTO_ETIMEOUT, \
    PETTO_EUNSUPPORTED = range(8)
PETTO_ELASTIC, PETTO_THERMAL = 0, 1
PETTO_SIMP_MODIFIED, PETTO_SIMP_PAPER = 0, 1
PETTO_F32, PETTO_F64, PETTO_BF16, PETTO_F16 = 0, 1, 2, 3
PETTO_VOL_PROJECTED, PETTO_VOL_PENALTY = 0, 1
PETTO_SOLVE_PAPER, PETTO_SOLVE_TOL = 0, 1
PETTO_SWEEP_APT, PETTO_SWEEP_PT = 0, 1
PETTO_LAYER_PHI, PETTO_LAYER_MU = 0, 1

_i64 = ctypes.c_int64
_dbl = ctypes.c_double
_int = ctypes.c_int
_vp = ctypes.c_void_p


class petto_grid(ctypes.Structure):
    _fields_ = [("dim", _int), ("nx", _i64), ("ny", _i64), ("nz", _i64), ("h", _dbl)]


class petto_materials(ctypes.Structure):
    _fields_ = [("physics", _int), ("n_phases", _int), ("modulus", ctypes.POINTER(_dbl)), ("e_min", _dbl),
                ("nu", _dbl), ("penal", _dbl), ("interp", _int)]


class petto_loads(ctypes.Structure):
    _fields_ = [("n", _i64), ("node", ctypes.POINTER(_i64)), ("comp", ctypes.POINTER(ctypes.c_int32)),
                ("value", ctypes.POINTER(_dbl)), ("rhs", ctypes.POINTER(ctypes.c_int32)), ("body_source", _dbl)]


class petto_bcs(ctypes.Structure):
    _fields_ = [("n_boxes", _int), ("box", ctypes.POINTER(_i64)), ("comp_mask", ctypes.POINTER(ctypes.c_uint32))]


class petto_options(ctypes.Structure):
    _fields_ = [("precision", _int), ("storage", _int), ("nrhs", _int), ("stream", _vp)]


class petto_solve_opts(ctypes.Structure):
    _fields_ = [("mode", _int), ("n_apt", _i64), ("n_pt", _i64), ("a", _dbl), ("b", _dbl), ("s1", _dbl),
                ("tol", _dbl), ("max_sweeps", _i64), ("check_every", _int), ("local_dt", _int),
                ("momentum", _int), ("refine", _int)]


class petto_solve_report(ctypes.Structure):
    _fields_ = [("sweeps", _i64), ("apt_sweeps", _i64), ("pt_sweeps", _i64), ("res_norm", _dbl), ("f_norm", _dbl),
                ("rel_res", _dbl), ("r_pde", _dbl), ("converged", _int), ("fell_back_to_pt", _int)]


class petto_pf_opts(ctypes.Structure):
    _fields_ = [("vol_mode", _int), ("alpha_h", _dbl), ("kappa_v", _dbl), ("kappa_1", _dbl), ("gamma_g", _dbl),
                ("tau", _dbl), ("ch_steps", _int), ("n_bisect", _int)]


petto_step_cb = ctypes.CFUNCTYPE(None, ctypes.POINTER(_dbl), _vp)
petto_exchange_fn = ctypes.CFUNCTYPE(_int, _vp, _vp)
petto_allreduce_fn = ctypes.CFUNCTYPE(_int, ctypes.POINTER(_dbl), _int, _vp)
petto_layer_exchange_fn = ctypes.CFUNCTYPE(_int, _vp, _int, _int, _vp)

_P = ctypes.POINTER
_SIGS = {
    "petto_create": (_int, [_P(petto_grid), _P(petto_materials), _P(petto_loads), _P(petto_bcs), _P(_dbl),
                            _P(petto_options), _P(_vp)]),
    "petto_destroy": (None, [_vp]),
    "petto_last_error": (ctypes.c_char_p, [_vp]),
    "petto_status_string": (ctypes.c_char_p, [_int]),
    "petto_set_design": (_int, [_vp, _vp, _int, _int]),
    "petto_get_design": (_int, [_vp, _vp, _int, _int]),
    "petto_set_state": (_int, [_vp, _vp, _vp, _int, _int]),
    "petto_get_state": (_int, [_vp, _vp, _vp, _int, _int]),
    "petto_get_modulus": (_int, [_vp, _vp, _int, _int]),
    "petto_sweep": (_int, [_vp, _int, _i64, _dbl, _dbl, _dbl, _int, _P(_dbl)]),
    "petto_set_wait_limit": (_int, [_vp, _int]),
    "petto_sweep_rhs": (_int, [_vp, _int, _i64, _dbl, _dbl, _dbl, _int, _vp, _int, _P(_dbl)]),
    "petto_residual": (_int, [_vp, _P(_dbl), _vp, _int, _int]),
    "petto_residual64": (_int, [_vp, _vp, _int, _P(_dbl), _vp]),
    "petto_pt_solve": (_int, [_vp, _P(petto_solve_opts), _P(petto_solve_report)]),
    "petto_sensitivity": (_int, [_vp, _P(_dbl), _P(_dbl), _vp, _int, _int]),
    "petto_design_update": (_int, [_vp, _P(petto_pf_opts), _P(_dbl)]),
    "petto_cahn_hilliard": (_int, [_vp, _P(petto_pf_opts)]),
    "petto_phase_field_step": (_int, [_vp, _P(petto_pf_opts), _P(_dbl)]),
    "petto_optimize": (_int, [_vp, _int, _P(petto_solve_opts), _P(petto_pf_opts), petto_step_cb, _vp]),
    "petto_save": (_int, [_vp, ctypes.c_char_p]),
    "petto_load": (_int, [_vp, ctypes.c_char_p]),
    "petto_synchronize": (_int, [_vp]),
    "petto_launch_count": (_i64, [_vp]),
    "petto_profile": (_int, [_vp, _int]),
    "petto_profile_read": (_int, [_vp, _P(_dbl), _P(_i64), _P(_i64)]),
    "petto_residual_norm_static": (_int, [_P(petto_grid), _dbl, _vp, _vp, _vp, _vp, _P(_dbl), _vp]),
    "petto_autotune": (_int, [_vp, _int, ctypes.c_char_p, _int]),
    "petto_select_kernel": (_int, [_vp, ctypes.c_char_p]),
    "petto_kernel_info": (_int, [_vp, ctypes.c_char_p, _int, _P(_int)]),
    "petto_set_owned_planes": (_int, [_vp, _i64, _i64, _i64]),
    "petto_slab_solve": (_int, [_vp, _P(petto_solve_opts), petto_exchange_fn, petto_allreduce_fn,
                                petto_allreduce_fn, _vp, _P(petto_solve_report)]),
    "petto_slab_design_step": (_int, [_vp, _P(petto_solve_opts), _P(petto_pf_opts), petto_exchange_fn,
                                      petto_layer_exchange_fn, petto_allreduce_fn, petto_allreduce_fn, _vp,
                                      _P(_dbl)]),
    "petto_layer_bytes": (_i64, [_vp, _int]),
    "petto_get_layer": (_int, [_vp, _int, _int, _i64, _vp, _int]),
    "petto_set_layer": (_int, [_vp, _int, _int, _i64, _vp, _int]),
    "petto_get_plane": (_int, [_vp, _i64, _vp, _int, _int]),
    "petto_set_plane": (_int, [_vp, _i64, _vp, _int, _int]),
    "petto_set_keepout": (_int, [_vp, _P(_i64), _P(_dbl), _dbl]),
    "petto_batch_create": (_int, [_int, _P(_vp), _P(_vp)]),
    "petto_batch_destroy": (None, [_vp]),
    "petto_batch_last_error": (ctypes.c_char_p, [_vp]),
    "petto_batch_launch_count": (_i64, [_vp]),
    "petto_batch_pt_solve": (_int, [_vp, _P(petto_solve_opts), _P(petto_solve_report)]),
    "petto_batch_optimize": (_int, [_vp, _int, _P(petto_solve_opts), _P(petto_pf_opts), _P(_dbl)]),
    "petto_batch_profile": (_int, [_vp, _int]),
    "petto_batch_profile_read": (_int, [_vp, _P(_dbl), _P(_i64)]),
}
EXPORTED = tuple(_SIGS)

_lock = threading.Lock()
_lib = None


class PettoError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{status_string(status)}: {message}")
        self.status = status


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libpetto.so (building it first when missing or stale and nvcc exists)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing:
                try:
                    path = _build.build()
                except RuntimeError:
                    if not os.path.exists(path):
                        raise
            if not os.path.exists(path):
                raise RuntimeError(f"libpetto.so is missing at {path}; run __graft_entry__.build() first")
            lib = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def status_string(s: int) -> str:
    try:
        return load().petto_status_string(int(s)).decode()
    except Exception:
        return f"status {s}"


def check(ctx, status: int, allow=(PETTO_OK,)) -> int:
    if status not in allow:
        msg = load().petto_last_error(ctx).decode() if ctx else ""
        raise PettoError(status, msg)
    return status


def check_batch(batch, status: int, allow=(PETTO_OK,)) -> int:
    if status not in allow:
        msg = load().petto_batch_last_error(batch).decode() if batch else ""
        raise PettoError(status, msg)
    return status

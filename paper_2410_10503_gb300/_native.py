"""ctypes declarations of libmc (include/mc.h).  Loading fails loudly if the
in-tree library has not been built: there is no fallback implementation."""
from __future__ import annotations

import ctypes
import os

from .build import CHECKED_LIB, LIB

MC_OK, MC_EINVAL, MC_ENOMEM, MC_ECUDA, MC_ETIMEOUT, MC_ESTATE, MC_EDEVICE = 0, -1, -2, -3, -4, -5, -6
STATUS_NAMES = {0: "MC_OK", -1: "MC_EINVAL", -2: "MC_ENOMEM", -3: "MC_ECUDA",
                -4: "MC_ETIMEOUT", -5: "MC_ESTATE", -6: "MC_EDEVICE"}
MC_MOTION_RIGID, MC_MOTION_FIELD = 0, 1
MC_OPT_GRAPH, MC_OPT_PROFILE, MC_OPT_TRACE_OBJECTIVE, MC_OPT_STORAGE, MC_OPT_TEST_STALL = 1, 2, 3, 4, 5
MC_OPT_SUBSET_BANDS, MC_OPT_SUBSET_ROWS, MC_OPT_FORWARD_LINES, MC_OPT_BACKPROJECT_ROWS = 6, 7, 8, 9
MC_STORE_F32, MC_STORE_F16, MC_STORE_BF16 = 0, 1, 2


class mc_geometry(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_angles", ctypes.c_int32), ("n_bins", ctypes.c_int32)]


class mc_motion(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("rigid", ctypes.c_void_p), ("field", ctypes.c_void_p)]


class mc_sampling(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("stream", ctypes.c_uint32), ("p", ctypes.c_void_p)]


# name -> (restype, argtypes); every declaration of include/mc.h
_VP, _I32, _I64, _U64, _D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
SIGNATURES = {
    "mc_create": (_I32, [ctypes.POINTER(mc_geometry), _I32, ctypes.POINTER(mc_motion), _VP,
                         ctypes.POINTER(_VP)]),
    "mc_destroy": (None, [_VP]),
    "mc_last_error": (ctypes.c_char_p, [_VP]),
    "mc_set_data": (_I32, [_VP, _VP, _D]),
    "mc_stage_data": (_I32, [_VP, _VP]),
    "mc_commit_data": (_I32, [_VP, _D]),
    "mc_forward": (_I32, [_VP, _I32, _VP, _VP]),
    "mc_adjoint": (_I32, [_VP, _I32, _VP, _VP]),
    "mc_project": (_I32, [_VP, _VP, _VP]),
    "mc_backproject": (_I32, [_VP, _VP, _VP]),
    "mc_warp": (_I32, [_VP, _I32, _VP, _VP]),
    "mc_warp_adjoint": (_I32, [_VP, _I32, _VP, _VP]),
    "mc_set_subsets": (_I32, [_VP, _I32]),
    "mc_autotune": (_I32, [_VP, _I32, _VP]),
    "mc_set_field": (_I32, [_VP, _I32, _VP]),
    "mc_vjp": (_I32, [_VP, _I32, _VP, _VP, _VP, _VP]),
    "mc_norms": (_I32, [_VP, _I32, _D, _VP]),
    "mc_set_norms": (_I32, [_VP, _VP]),
    "mc_get_steps": (_I32, [_VP, _I32, _VP]),
    "mc_set_reference": (_I32, [_VP, _VP]),
    "mc_reset": (_I32, [_VP]),
    "mc_solve_normal": (_I32, [_VP, _I32, _D, _VP, _VP]),
    "mc_spdhg_run": (_I32, [_VP, _I32, ctypes.POINTER(mc_sampling), _VP, _VP]),
    "mc_pdhg_run": (_I32, [_VP, _I32, _VP, _VP]),
    "mc_batch_create": (_I32, [_VP, _I32, _VP, ctypes.POINTER(_VP)]),
    "mc_batch_run": (_I32, [_VP, _I32, _VP, _VP]),
    "mc_batch_last_error": (ctypes.c_char_p, [_VP]),
    "mc_batch_destroy": (None, [_VP]),
    "mc_batch_spdhg_run": (_I32, [_VP, _I32, _I32, _VP, _VP]),
    "mc_draw_gates": (_I32, [_VP, ctypes.POINTER(mc_sampling), _U64, _I32, _VP]),
    "mc_objective": (_I32, [_VP, _VP, _VP]),
    "mc_set_option": (_I32, [_VP, _I32, _I64]),
    "mc_profile_read": (_I32, [_VP, _I32, _VP, _VP, _VP, _VP]),
    "mc_profile_reset": (_I32, [_VP]),
    "mc_iteration": (_I32, [_VP, _VP]),
    "mc_sync": (_I32, [_VP]),
    "mc_state_size": (_I32, [_VP, _VP]),
    "mc_save_state": (_I32, [_VP, _VP, _U64]),
    "mc_load_state": (_I32, [_VP, _VP, _U64]),
    "mc_version": (ctypes.c_char_p, []),
    "mc_plan_shapes": (_I32, [ctypes.POINTER(mc_geometry), _I32, _VP]),
    "mc_get_shapes": (_I32, [_VP, _VP]),
    "mc_measure_shared_load_peak": (_I32, [_I32, _VP]),
    "mc_forward_static": (_I32, [ctypes.POINTER(mc_geometry), _VP, _VP, _VP, _VP, ctypes.c_char_p, _I32]),
    "mc_forward_static_status": (_I32, [_VP, ctypes.c_char_p, _I32]),
}

_lib = None


def lib_path() -> str:
    """The library this process loads: the checked flavour under MC_CHECKED=1."""
    return CHECKED_LIB if os.environ.get("MC_CHECKED") == "1" else LIB


def load() -> ctypes.CDLL:
    """Load the in-tree libmc.so (built by __graft_entry__.build())."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libmc is not built ({path} missing): run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib

"""ctypes binding of libgnep (include/gnep.h): argument marshalling only.

The shared library is built in-tree by ``paper_2507_00528_gb300.build`` into
``_build/libgnep.so``.  Loading fails loudly when it is missing: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

GNEP_OK = 0
STATUS = {
    0: "GNEP_OK", -1: "GNEP_ERR_INVALID_ARG", -2: "GNEP_ERR_OOM", -3: "GNEP_ERR_CUDA",
    -4: "GNEP_ERR_NEIGHBOR_OVERFLOW", -5: "GNEP_ERR_NONFINITE", -6: "GNEP_ERR_TIMEOUT",
    -7: "GNEP_ERR_CHECKPOINT_CORRUPT", -8: "GNEP_ERR_UNSUPPORTED",
}
PREC = {"fp32": 0, "tf32": 1, "bf16": 2}
LOSS_MSE, LOSS_RMSE = 0, 1
LIST_RADIAL, LIST_ANGULAR = 0, 1

# Every entry point declared in include/gnep.h.
EXPORTS = [
    "gnep_create", "gnep_destroy", "gnep_set_precision", "gnep_num_params", "gnep_num_descriptors",
    "gnep_get_params", "gnep_set_params", "gnep_set_descriptor_scale", "gnep_get_descriptor_scale",
    "gnep_compute_descriptor_scale", "gnep_build_neighbors", "gnep_rebuild_neighbors",
    "gnep_nlist_destroy", "gnep_nlist_info", "gnep_nlist_export", "gnep_descriptors", "gnep_forward",
    "gnep_loss_grad", "gnep_adam_step", "gnep_adam_step_scheduled", "gnep_get_step",
    "gnep_lr_schedule", "gnep_graph_create", "gnep_graph_launch", "gnep_graph_destroy",
    "gnep_graph_kernel_count", "gnep_graph_create_steps", "gnep_save",
    "gnep_load", "gnep_sync_status", "gnep_last_error", "gnep_abi_version", "gnep_profile_step",
    "gnep_profile_stage_name", "gnep_descriptors_noalloc", "gnep_loss", "gnep_get_grad", "gnep_set_grad",
    "gnep_autotune", "gnep_tuning_get", "gnep_tuning_set", "gnep_md_verlet", "gnep_shard_loss_weights",
    "gnep_shard_mse_partials", "gnep_shard_mse_total", "gnep_selftest_wait_timeout",
]


class GnepError(RuntimeError):
    def __init__(self, code: int, msg: str):
        self.code = code
        super().__init__(f"{STATUS.get(code, code)}: {msg}")


class Batch(C.Structure):
    _fields_ = [("n_struct", C.c_int32), ("n_atoms", C.c_int32), ("struct_off", C.c_void_p),
                ("pos", C.c_void_p), ("type", C.c_void_p), ("cell", C.c_void_p)]


class Labels(C.Structure):
    _fields_ = [("energy", C.c_void_p), ("force", C.c_void_p), ("virial", C.c_void_p),
                ("lambda_e", C.c_double), ("lambda_f", C.c_double), ("lambda_v", C.c_double),
                ("lambda_l2", C.c_double), ("loss_form", C.c_int32)]


_vp = C.c_void_p
_SIGS = {
    "gnep_create": [C.POINTER(_vp), C.c_int, _vp, C.c_double, C.c_double, C.c_int, C.c_int, C.c_int,
                    C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_int],
    "gnep_destroy": [_vp],
    "gnep_set_precision": [_vp, C.c_int],
    "gnep_num_params": [_vp, C.POINTER(C.c_int64)],
    "gnep_num_descriptors": [_vp, C.POINTER(C.c_int32)],
    "gnep_get_params": [_vp, _vp, C.c_int64, _vp],
    "gnep_set_params": [_vp, _vp, C.c_int64, _vp],
    "gnep_set_descriptor_scale": [_vp, _vp, C.c_int32, _vp],
    "gnep_get_descriptor_scale": [_vp, _vp, C.c_int32, _vp],
    "gnep_compute_descriptor_scale": [_vp, _vp, _vp],
    "gnep_build_neighbors": [_vp, C.POINTER(Batch), C.POINTER(_vp), _vp],
    "gnep_rebuild_neighbors": [_vp, C.POINTER(Batch), _vp, _vp],
    "gnep_nlist_destroy": [_vp],
    "gnep_nlist_info": [_vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)],
    "gnep_nlist_export": [_vp, C.c_int, _vp, _vp, _vp, _vp],
    "gnep_descriptors": [_vp, _vp, _vp, _vp],
    "gnep_descriptors_noalloc": [_vp, _vp, _vp, _vp],
    "gnep_forward": [_vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "gnep_loss_grad": [_vp, _vp, C.POINTER(Labels), _vp, _vp, _vp],
    "gnep_loss": [_vp, _vp, C.POINTER(Labels), _vp, _vp],
    "gnep_get_grad": [_vp, _vp, C.c_int64, _vp],
    "gnep_set_grad": [_vp, _vp, C.c_int64, _vp],
    "gnep_autotune": [_vp, _vp, C.POINTER(Labels), C.c_int, _vp],
    "gnep_md_verlet": [_vp, _vp, _vp, _vp, _vp, _vp, C.c_double, _vp, _vp],
    "gnep_tuning_get": [_vp, _vp, _vp],
    "gnep_tuning_set": [_vp, _vp, _vp, _vp],
    "gnep_adam_step": [_vp, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, _vp],
    "gnep_adam_step_scheduled": [_vp, C.c_double, C.c_double, C.c_int64, C.c_int64, C.c_double,
                                 C.c_double, C.c_double, C.c_double, _vp],
    "gnep_get_step": [_vp, C.POINTER(C.c_int64), _vp],
    "gnep_lr_schedule": [C.c_double, C.c_double, C.c_int64, C.c_int64, C.c_int64],
    "gnep_graph_create": [_vp, _vp, C.POINTER(Labels), _vp, C.c_double, C.c_double, C.c_int64,
                          C.c_int64, C.c_double, C.c_double, C.c_double, C.c_double, _vp,
                          C.POINTER(_vp)],
    "gnep_graph_create_steps": [_vp, _vp, C.POINTER(Labels), C.c_int32, _vp, C.c_double, C.c_double, C.c_int64,
                                C.c_int64, C.c_double, C.c_double, C.c_double, C.c_double, _vp, C.POINTER(_vp)],
    "gnep_graph_launch": [_vp, _vp],
    "gnep_graph_destroy": [_vp],
    "gnep_graph_kernel_count": [_vp, _vp],
    "gnep_save": [_vp, C.c_char_p],
    "gnep_load": [_vp, C.c_char_p],
    "gnep_sync_status": [_vp, _vp],
    "gnep_last_error": [],
    "gnep_profile_step": [_vp, _vp, C.POINTER(Labels), _vp, C.c_int32, C.POINTER(C.c_int32), _vp],
    "gnep_profile_stage_name": [C.c_int32],
    "gnep_abi_version": [],
    "gnep_shard_loss_weights": [C.c_double, C.c_double, C.c_double, C.c_double, C.c_int32, C.c_int64,
                                C.c_int64, C.c_int64, C.c_int64, _vp, C.c_int32, _vp],
    "gnep_shard_mse_partials": [_vp, C.c_int64, C.c_int64, _vp],
    "gnep_shard_mse_total": [_vp, _vp],
    "gnep_selftest_wait_timeout": [_vp, C.c_int64, _vp],
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libgnep.so (optionally building it first).  Raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(
                f"libgnep.so is not built ({path}); run paper_2507_00528_gb300.build.build() "
                "(there is no CPU fallback)")
        _build.build()
    L = C.CDLL(path)
    for name, args in _SIGS.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int
    L.gnep_lr_schedule.restype = C.c_double
    L.gnep_last_error.restype = C.c_char_p
    L.gnep_profile_stage_name.restype = C.c_char_p
    _lib = L
    return L


def check(rc: int):
    if rc != GNEP_OK:
        msg = load().gnep_last_error().decode(errors="replace")
        raise GnepError(rc, msg)
    return rc

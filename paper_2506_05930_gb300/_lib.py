"""ctypes view of include/nvc.h: structures, prototypes and library loading.

The library is required: importing this module on a machine where
libnvc.so has not been built raises with instructions, there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import (POINTER, Structure, c_char_p, c_double, c_float, c_int32, c_int64,
                    c_uint32, c_uint64, c_void_p)

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libnvc.so")

NVC_OK = 0
NVC_ERR_INVALID_ARG = 1
NVC_ERR_UNSUPPORTED = 2
NVC_ERR_CUDA = 3
NVC_ERR_NONFINITE = 4
NVC_ERR_TIMEOUT = 5
STATUS_NAMES = {0: "NVC_OK", 1: "NVC_ERR_INVALID_ARG", 2: "NVC_ERR_UNSUPPORTED",
                3: "NVC_ERR_CUDA", 4: "NVC_ERR_NONFINITE", 5: "NVC_ERR_TIMEOUT"}

PRECISIONS = {"fp32": 0, "fp16": 1, "bf16": 2, "fp8": 3}
LOSSES = {"l2": 0, "bce": 1}
LR_SCHEDULES = {"constant": 0, "paper_ramp": 1, "ramp": 1}


class NvcConfig(Structure):
    _fields_ = [
        ("n_levels", c_int32), ("n_features", c_int32), ("log2_table_size", c_int32),
        ("base_resolution", c_int32), ("growth", c_double), ("n_hidden", c_int32),
        ("hidden_width", c_int32), ("n_outputs", c_int32), ("leaky_slope", c_float),
        ("precision", c_int32), ("train_precision", c_int32), ("loss", c_int32),
        ("lr_schedule", c_int32), ("lr", c_float), ("lr_end", c_float),
        ("lr_ramp_steps", c_int32), ("beta1", c_float), ("beta2", c_float), ("eps", c_float),
        ("loss_scale", c_float), ("batch_positions", c_int32), ("bounds_min", c_float * 3),
        ("bounds_max", c_float * 3)]


class NvcScene(Structure):
    _fields_ = [
        ("lights", c_void_p), ("n_lights", c_int32), ("spheres", c_void_p),
        ("n_spheres", c_int32), ("boxes", c_void_p), ("n_boxes", c_int32),
        ("world_min", c_float * 3), ("world_max", c_float * 3)]


CLUSTER_WEIGHTS = {"sum": 0, "visibility": 1}


class NvcClusters(Structure):
    _fields_ = [("k", c_int32), ("offsets", c_void_p), ("members", c_void_p),
                ("weights", c_int32)]


class NvcShadePlan(Structure):
    _fields_ = [("variant", c_int32), ("ctas_per_sm", c_int32)]


class NvcCounters(Structure):
    _fields_ = [("step", c_int32), ("skipped", c_int32), ("error_flags", c_int32),
                ("frames", c_int32)]


class NvcView(Structure):
    _fields_ = [
        ("pos", c_void_p), ("nrm", c_void_p), ("n_pixels", c_int64), ("view_id", c_uint32),
        ("idx", c_void_p), ("pdf", c_void_p), ("wsum", c_void_p), ("radiance", c_void_p)]


_cfgp = POINTER(NvcConfig)
_scp = POINTER(NvcScene)
_clp = POINTER(NvcClusters)
_vp = c_void_p

PROTOTYPES = {
    "nvc_create": (c_int32, [_cfgp, POINTER(c_void_p)]),
    "nvc_destroy": (None, [_vp]),
    "nvc_last_error": (c_char_p, [_vp]),
    "nvc_param_count": (c_int64, [_cfgp]),
    "nvc_level_resolution": (c_int32, [_cfgp, c_int32]),
    "nvc_set_state": (c_int32, [_vp, _vp, _vp, _vp, c_int32, _vp]),
    "nvc_get_state": (c_int32, [_vp, _vp, _vp, _vp, _vp]),
    "nvc_set_staging": (c_int32, [_vp, c_int64]),
    "nvc_sync_status": (c_int32, [_vp, _vp, POINTER(NvcCounters)]),
    "nvc_encode": (c_int32, [_vp, _vp, c_int64, _vp, _vp]),
    "nvc_infer": (c_int32, [_vp, _vp, c_int64, _vp, _vp]),
    "nvc_light_weights": (c_int32, [_scp, _vp, _vp, _vp, c_int64, _vp, _vp, _vp]),
    "nvc_wrs_from_weights": (c_int32, [_vp, c_int64, c_int32, c_uint64, c_uint32, c_uint32,
                                       c_int64, _vp, _vp, _vp, _vp]),
    "nvc_wrs_sample": (c_int32, [_vp, _scp, _vp, _vp, c_int64, c_uint64, c_uint32, c_uint32,
                                 c_int64, _vp, _vp, _vp, _vp]),
    "nvc_direct_illum": (c_int32, [_vp, _scp, _vp, _vp, c_int64, _vp, _vp]),
    "nvc_shade": (c_int32, [_vp, _scp, _vp, _vp, c_int64, c_uint64, c_uint32, c_uint32, c_int64,
                            _vp, _vp, _vp, _vp, c_int32, _vp]),
    "nvc_sampler_weights": (c_int32, [_vp, _scp, _vp, _vp, c_int64, _vp, _vp]),
    "nvc_autotune_shade": (c_int32, [_vp, _scp, _vp, _vp, c_int64, _vp, _vp, _vp, _vp, c_int32,
                                     POINTER(c_int32), POINTER(c_double), _vp]),
    "nvc_set_shade_variant": (c_int32, [_vp, c_int32]),
    "nvc_mlp_infer_features": (c_int32, [_vp, _vp, c_int64, c_int32, _vp, _vp]),
    "nvc_set_shade_plan": (c_int32, [_vp, POINTER(NvcShadePlan)]),
    "nvc_autotune_shade_plan": (c_int32, [_vp, _scp, _vp, _vp, c_int64, _vp, _vp, _vp, _vp, c_int32,
                                          POINTER(NvcShadePlan), POINTER(NvcShadePlan),
                                          POINTER(c_double), c_int32, POINTER(c_int32), _vp]),
    "nvc_shade_phases": (c_int32, [_vp, _scp, _vp, _vp, c_int64, c_uint64, c_uint32, _vp, _vp,
                                   _vp, _vp, POINTER(c_double), _vp]),
    "nvc_gather_bench": (c_int32, [_vp, c_int64, c_int32, c_int64, c_int32, c_uint32, _vp, _vp]),
    "nvc_set_params": (c_int32, [_vp, _vp, _vp]),
    "nvc_set_table_precision": (c_int32, [_vp, c_int32, _vp]),
    "nvc_autotune_infer": (c_int32, [_vp, _vp, c_int64, _vp, c_int32, _vp, _vp, _vp]),
    "nvc_calibrate": (c_int32, [_vp, _vp, c_int64, _vp]),
    "nvc_trace_visibility": (c_int32, [_scp, _vp, c_int64, _vp, _vp]),
    "nvc_training_positions": (c_int32, [_scp, _vp, c_int64, c_int64, c_uint64, c_uint32, _vp,
                                         _vp]),
    "nvc_training_positions_split": (c_int32, [_scp, _vp, c_int64, c_int64, c_int64, c_uint64,
                                               c_uint32, _vp, _vp]),
    "nvc_set_training_placement": (c_int32, [_vp, c_int64]),
    "nvc_set_training_data_fused": (c_int32, [_vp, c_int32]),
    "nvc_training_batch": (c_int32, [_vp, _vp, _vp, _vp]),
    "nvc_train_step": (c_int32, [_vp, _scp, _vp, c_int64, c_uint64, c_uint32, _vp, _vp]),
    "nvc_train_gradient": (c_int32, [_vp, _scp, _vp, c_int64, c_uint64, c_uint32, _vp, _vp,
                                     _vp]),
    "nvc_mlp_forward": (c_int32, [_vp, _vp, c_int64, _vp, _vp]),
    "nvc_mlp_backward": (c_int32, [_vp, _vp, c_int64, _vp, _vp, _vp]),
    "nvc_frame": (c_int32, [_vp, _scp, POINTER(NvcView), c_int32, c_int32, c_uint64, c_uint32,
                            _vp, c_int32, _vp]),
    "nvc_frame_host": (c_int32, [_vp, _scp, POINTER(NvcView), c_int32, c_int32, c_uint64,
                                 c_uint32, _vp, c_int32, _vp]),
    "nvc_host_frames_wait": (c_int32, [_vp, _vp]),
    "nvc_shade_estimate": (c_int32, [_scp, _vp, _vp, c_int64, _vp, _vp, _vp, _vp, c_uint32, _vp]),
    "nvc_exact_di": (c_int32, [_scp, _vp, _vp, c_int64, _vp, _vp]),
    "nvc_kmeans_lights": (c_int32, [_vp, c_int32, _vp, c_int32, c_int32, _vp, _vp]),
    "nvc_train_step_clustered": (c_int32, [_vp, _scp, _clp, _vp, c_int64, c_uint64, c_uint32,
                                           _vp, _vp]),
    "nvc_cluster_targets": (c_int32, [_scp, _clp, _vp, c_int64, c_uint64, c_uint32, _vp, _vp]),
    "nvc_sample_clustered": (c_int32, [_scp, _clp, _vp, _vp, _vp, c_int64, c_int64, c_uint64,
                                       c_uint32, c_uint32, _vp, _vp, _vp, _vp]),
    "nvc_temporal_merge": (c_int32, [_scp, _vp, _vp, c_int64, c_int64, c_uint64, c_uint32, c_uint32,
                                     _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "nvc_infer_noalloc": (c_int32, [_cfgp, _vp, _vp, c_int64, _vp, _vp]),
    "nvc_set_profiling": (c_int32, [_vp, c_int32]),
    "nvc_stage_times": (c_int32, [_vp, POINTER(c_double), c_int32, POINTER(c_int64)]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libnvc.so once and attach the prototypes."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build it with `python -c \"import __graft_entry__ as g; "
            f"g.build()\"` (needs nvcc); there is no CPU fallback")
    lib = ctypes.CDLL(path)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class NVCError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def check(status: int, handle=None):
    if status != NVC_OK:
        msg = _lib.nvc_last_error(handle).decode(errors="replace")
        raise NVCError(status, msg)

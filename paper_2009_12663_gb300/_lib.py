"""ctypes binding of the gbfwi C ABI (include/gbfwi.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Arrays may be torch tensors (CUDA or CPU) or numpy arrays; device
tensors are passed as device pointers and the work is queued on the current
torch CUDA stream, host arrays are staged by the library.  A missing or
unloadable library raises at import of the first call: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

GBFWI_OK = 0
ERRORS = {
    -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ECFL", -5: "ECURV",
    -6: "ENONFINITE", -8: "ENOMODEL", -9: "ESCRATCH",
}

#: every symbol declared in include/gbfwi.h
ABI_SYMBOLS = (
    "gbfwi_mesh_create", "gbfwi_mesh_destroy", "gbfwi_mesh_dims", "gbfwi_node_coords",
    "gbfwi_num_tiles", "gbfwi_tile_shape", "gbfwi_get_schedule", "gbfwi_set_schedule",
    "gbfwi_set_model", "gbfwi_forward", "gbfwi_misfit", "gbfwi_adjoint_gradient", "gbfwi_precond_diag",
    "gbfwi_bfgs_create", "gbfwi_bfgs_update", "gbfwi_bfgs_count", "gbfwi_bfgs_apply",
    "gbfwi_lowrank_invhess", "gbfwi_lowrank_twopass", "gbfwi_lowrank_exact", "gbfwi_bfgs_destroy", "gbfwi_launch_count", "gbfwi_enable_timing",
    "gbfwi_last_phase_times", "gbfwi_misfit_noalloc", "gbfwi_strerror",
    "gbfwi_unet_create", "gbfwi_unet_destroy", "gbfwi_unet_num_params", "gbfwi_unet_layer_info",
    "gbfwi_unet_set_params", "gbfwi_unet_get_params", "gbfwi_unet_forward", "gbfwi_unet_gradient",
    "gbfwi_unet_train_step", "gbfwi_unet_features", "gbfwi_resample", "gbfwi_precond_from_hessian",
)


class GbfwiError(RuntimeError):
    def __init__(self, code: int, what: str, msg: str):
        super().__init__(f"{what}: {ERRORS.get(code, code)} ({msg})")
        self.code = code
        self.name = ERRORS.get(code, str(code))


class MeshDesc(ctypes.Structure):
    _fields_ = [("nex", ctypes.c_int), ("nez", ctypes.c_int), ("h", ctypes.c_double),
                ("ngll", ctypes.c_int), ("free_surface_top", ctypes.c_int),
                ("dt", ctypes.c_double), ("nt", ctypes.c_int), ("precision", ctypes.c_int)]


class Source(ctypes.Structure):
    _fields_ = [("x", ctypes.c_double), ("z", ctypes.c_double), ("type", ctypes.c_int),
                ("f0", ctypes.c_double), ("t0", ctypes.c_double), ("amp", ctypes.c_double)]


class UnetDesc(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("base", ctypes.c_int), ("cin", ctypes.c_int), ("cout", ctypes.c_int),
                ("height", ctypes.c_int), ("width", ctypes.c_int)]


class Schedule(ctypes.Structure):
    _fields_ = [("shots_per_launch", ctypes.c_int), ("tile", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("ckpt_every", ctypes.c_int), ("streams", ctypes.c_int)]


_LIB = None


def lib(path: str | None = None):
    """Load (building it first if needed) the in-tree libgbfwi.so."""
    global _LIB
    if _LIB is None:
        so = path or os.environ.get("GBFWI_LIB") or _build.build()
        _LIB = ctypes.CDLL(so)
        L = _LIB
        vp = ctypes.c_void_p
        L.gbfwi_strerror.restype = ctypes.c_char_p
        L.gbfwi_strerror.argtypes = [ctypes.c_int]
        L.gbfwi_mesh_create.argtypes = [ctypes.POINTER(MeshDesc), ctypes.POINTER(Source), ctypes.c_int,
                                        vp, ctypes.c_int, ctypes.POINTER(vp)]
        L.gbfwi_mesh_destroy.argtypes = [vp]
        L.gbfwi_mesh_dims.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        L.gbfwi_node_coords.argtypes = [vp, vp, vp]
        L.gbfwi_num_tiles.argtypes = []
        L.gbfwi_tile_shape.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        L.gbfwi_get_schedule.argtypes = [vp, ctypes.POINTER(Schedule)]
        L.gbfwi_set_schedule.argtypes = [vp, ctypes.POINTER(Schedule)]
        L.gbfwi_set_model.argtypes = [vp, vp, vp, vp, vp]
        L.gbfwi_forward.argtypes = [vp, vp, ctypes.c_int, vp, vp]
        L.gbfwi_misfit.argtypes = [vp, vp, ctypes.c_int, vp, ctypes.POINTER(ctypes.c_double), vp]
        L.gbfwi_adjoint_gradient.argtypes = [vp, vp, ctypes.c_int, vp, ctypes.POINTER(ctypes.c_double), vp,
                                             ctypes.c_int, vp]
        L.gbfwi_precond_diag.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                         vp, vp, vp]
        L.gbfwi_bfgs_create.argtypes = [ctypes.c_longlong, ctypes.c_int, vp, ctypes.POINTER(vp)]
        L.gbfwi_bfgs_update.argtypes = [vp, vp, vp, vp]
        L.gbfwi_bfgs_count.argtypes = [vp]
        L.gbfwi_bfgs_apply.argtypes = [vp, vp, ctypes.c_int, vp, ctypes.c_double, ctypes.c_int, vp]
        L.gbfwi_lowrank_invhess.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_ulonglong,
                                            ctypes.c_double, vp, vp, vp, vp]
        L.gbfwi_lowrank_twopass.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_ulonglong,
                                            ctypes.c_double, vp, vp, vp, vp]
        L.gbfwi_lowrank_exact.argtypes = [vp, ctypes.c_int, ctypes.c_double, vp, vp, vp, vp]
        L.gbfwi_bfgs_destroy.argtypes = [vp]
        L.gbfwi_misfit_noalloc.argtypes = [vp, vp, ctypes.c_int, ctypes.c_longlong, ctypes.c_double, vp, vp]
        L.gbfwi_launch_count.restype = ctypes.c_longlong
        L.gbfwi_launch_count.argtypes = []
        L.gbfwi_enable_timing.argtypes = [vp, ctypes.c_int]
        L.gbfwi_last_phase_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
        L.gbfwi_unet_create.argtypes = [ctypes.POINTER(UnetDesc), ctypes.POINTER(vp)]
        L.gbfwi_unet_destroy.argtypes = [vp]
        L.gbfwi_unet_num_params.restype = ctypes.c_longlong
        L.gbfwi_unet_num_params.argtypes = [vp]
        L.gbfwi_unet_layer_info.argtypes = [vp, ctypes.c_int, vp]
        L.gbfwi_unet_set_params.argtypes = [vp, vp, vp]
        L.gbfwi_unet_get_params.argtypes = [vp, vp, vp]
        L.gbfwi_unet_forward.argtypes = [vp, vp, vp, vp]
        L.gbfwi_unet_gradient.argtypes = [vp, vp, vp, vp, vp]
        L.gbfwi_unet_train_step.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_double,
                                            ctypes.POINTER(ctypes.c_double), vp]
        L.gbfwi_unet_features.argtypes = [vp, vp, vp, vp, ctypes.c_double, ctypes.c_int, ctypes.c_int, vp, vp]
        L.gbfwi_resample.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, vp]
        L.gbfwi_precond_from_hessian.argtypes = [vp, vp, ctypes.c_double, ctypes.c_double, vp, vp]
    return _LIB


def check(rc: int, what: str) -> int:
    if rc < 0:
        raise GbfwiError(rc, what, lib().gbfwi_strerror(rc).decode())
    return rc


# ---------------------------------------------------------------------------
# array marshalling
# ---------------------------------------------------------------------------

def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def ptr(a, dtype):
    """Data pointer of a contiguous torch tensor / numpy array of `dtype`."""
    if a is None:
        return None
    if _is_torch(a):
        import torch
        want = {np.float32: torch.float32, np.float64: torch.float64, np.int32: torch.int32}[dtype]
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"expected a contiguous {want} tensor")
        return ctypes.c_void_p(a.data_ptr())
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags.c_contiguous:
        raise TypeError(f"expected a contiguous numpy array of {np.dtype(dtype)}")
    return ctypes.c_void_p(a.ctypes.data)


def stream_of(*arrays):
    """The current torch CUDA stream when any array lives on the GPU, else NULL."""
    for a in arrays:
        if a is not None and _is_torch(a) and a.is_cuda:
            import torch
            return ctypes.c_void_p(torch.cuda.current_stream(a.device).cuda_stream)
    return None

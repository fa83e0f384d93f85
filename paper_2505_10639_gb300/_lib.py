"""ctypes declarations of the C ABI in ``include/mfbd.h`` and
``include/mfbd_testing.h``. Loading fails loudly when the library is missing:
there is no fallback implementation."""

import ctypes
import os

from . import build as _build

MFBD_OK = 0
MFBD_ERR_INVALID_ARG = 1
MFBD_ERR_UNSUPPORTED = 2
MFBD_ERR_OOM = 3
MFBD_ERR_CUDA = 4
MFBD_ERR_STATE = 5
MFBD_ERR_TIMEOUT = 6

MFBD_BASIS_ZERNIKE = 0
MFBD_BASIS_KL = 1
MFBD_BASIS_USER = 2
MFBD_PREC_FP32 = 0
MFBD_PREC_BF16_PHASE = 1
MFBD_FLAG_FULL_SPECTRUM = 0x1
MFBD_FLAG_SIMT_PROJECTION = 0x2
MFBD_FLAG_RECOMPUTE_BACKWARD = 0x4
MFBD_FLAG_GENERIC_KERNELS = 0x8
MFBD_FLAG_SPLIT_PASSES = 0x10
MFBD_BATCH_ONE_LAUNCH = 0
MFBD_BATCH_STAGED = 1


class PlanDesc(ctypes.Structure):
    _fields_ = [
        ("n_pix", ctypes.c_int),
        ("n_patches", ctypes.c_int),
        ("n_objects", ctypes.c_int),
        ("n_frames", ctypes.c_int),
        ("n_modes", ctypes.c_int),
        ("pupil_diam_px", ctypes.POINTER(ctypes.c_float)),
        ("wavelength", ctypes.POINTER(ctypes.c_double)),
        ("central_obscuration", ctypes.c_float),
        ("basis", ctypes.c_int),
        ("user_basis", ctypes.POINTER(ctypes.c_float)),
        ("gamma", ctypes.c_double),
        ("frame_weight", ctypes.POINTER(ctypes.c_float)),
        ("precision", ctypes.c_int),
        ("flags", ctypes.c_uint),
    ]


class PlanInfo(ctypes.Structure):
    _fields_ = [
        ("n_pix", ctypes.c_int),
        ("n_patches", ctypes.c_int),
        ("n_objects", ctypes.c_int),
        ("n_frames", ctypes.c_int),
        ("n_modes", ctypes.c_int),
        ("pupil_pixels", ctypes.c_int * 8),
        ("pupil_box", ctypes.c_int * 8),
        ("workspace_bytes", ctypes.c_size_t),
        ("slots_per_cta", ctypes.c_int),
        ("ctas", ctypes.c_int),
        ("reduction_split", ctypes.c_int),
        ("fused_ctas", ctypes.c_int),
        ("tc_projection", ctypes.c_int),
        ("tc_adjoint", ctypes.c_int),
    ]


class DictDesc(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int),
        ("n_patches", ctypes.c_int),
        ("n_objects", ctypes.c_int),
        ("n_frames", ctypes.c_int),
        ("n_atoms", ctypes.c_int),
    ]


class BatchInfo(ctypes.Structure):
    _fields_ = [
        ("n_problems", ctypes.c_int),
        ("n_patches", ctypes.c_longlong),
        ("n_units", ctypes.c_longlong),
        ("n_items", ctypes.c_longlong),
        ("coeff_floats", ctypes.c_longlong),
        ("spectra_complex", ctypes.c_longlong),
        ("loss_doubles", ctypes.c_longlong),
        ("object_complex", ctypes.c_longlong),
        ("workspace_bytes", ctypes.c_size_t),
        ("mode", ctypes.c_int),
        ("window_units", ctypes.c_int),
        ("ctas_per_sm", ctypes.c_int),
        ("max_ctas_per_sm", ctypes.c_int),
        ("ctas", ctypes.c_int),
        ("smem_bytes", ctypes.c_int),
        ("variant", ctypes.c_int),
    ]


_VP = ctypes.c_void_p
_SIGNATURES = {
    "mfbd_plan_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.POINTER(PlanDesc), _VP]),
    "mfbd_plan_destroy": (ctypes.c_int, [_VP]),
    "mfbd_plan_get_info": (ctypes.c_int, [_VP, ctypes.POINTER(PlanInfo)]),
    "mfbd_forward": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "mfbd_backward": (ctypes.c_int, [_VP, _VP, _VP]),
    "mfbd_loss_grad": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "mfbd_loss_grad_host": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, ctypes.c_int, _VP]),
    "mfbd_otf": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "mfbd_describe_object": (ctypes.c_int, [ctypes.POINTER(PlanDesc), ctypes.c_int, _VP, _VP, _VP, _VP]),
    "mfbd_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "mfbd_last_error": (ctypes.c_char_p, []),
    "mfbd_test_fft_host": (ctypes.c_int, [ctypes.c_int, _VP, _VP]),
    "mfbd_plan_set_profiling": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int]),
    "mfbd_plan_read_profile": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int]),
    "mfbd_phase_loss_grad_noalloc": (ctypes.c_int, [ctypes.POINTER(PlanDesc), _VP, _VP, _VP, _VP, _VP, _VP]),
    "mfbd_plan_set_diversity": (ctypes.c_int, [_VP, _VP, _VP]),
    "mfbd_dict_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(DictDesc)]),
    "mfbd_dict_loss_grad": (ctypes.c_int, [ctypes.POINTER(DictDesc), _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP,
                                           _VP]),
    "mfbd_spectra_from_frames": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                _VP, _VP]),
    "mfbd_filter_objects": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "mfbd_loss_grad_explicit": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "mfbd_ls_filter_objects": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_float, _VP, _VP, _VP]),
    "mfbd_merge_objects": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP,
                                          _VP]),
    "mfbd_batch_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.POINTER(PlanDesc), ctypes.c_int, _VP]),
    "mfbd_batch_destroy": (ctypes.c_int, [_VP]),
    "mfbd_batch_get_info": (ctypes.c_int, [_VP, ctypes.POINTER(BatchInfo)]),
    "mfbd_batch_get_offsets": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "mfbd_batch_set_schedule": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "mfbd_batch_loss_grad": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "mfbd_batch_otf": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "mfbd_batch_check": (ctypes.c_int, [_VP, _VP]),
    "mfbd_batch_autotune": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, ctypes.c_int, _VP]),
    "mfbd_test_batch_items": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, ctypes.c_longlong,
                                             _VP]),
    "mfbd_probe_fma_rate": (ctypes.c_int, [ctypes.c_int, ctypes.c_longlong, _VP, _VP, _VP]),
    "mfbd_plan_check": (ctypes.c_int, [_VP, _VP]),
}

_lib = None


def lib_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load (building first if needed) the shared library."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError("libmfbd.so is not built (run __graft_entry__.build())")
        _build.build()
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class MFBDError(RuntimeError):
    def __init__(self, status, where):
        lib = load()
        msg = "%s failed: %s (%s)" % (where, lib.mfbd_status_string(status).decode(),
                                      lib.mfbd_last_error().decode())
        super().__init__(msg)
        self.status = status


def check(status, where):
    if status != MFBD_OK:
        raise MFBDError(status, where)

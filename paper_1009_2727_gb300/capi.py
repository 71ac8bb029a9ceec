"""ctypes binding of include/pic.h (argument marshalling only).

Every function here forwards to the CUDA library libpicgb.so; no step of the
method runs in Python. PyTorch supplies the device memory (its caching
allocator, through the pic_alloc_fn callback) and the CUDA stream.
The library is loaded on first use and the import fails loudly when it cannot
be built or loaded: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
API_VERSION = 1

PIC_OK, PIC_EINVAL, PIC_ENOMEM, PIC_ECFL, PIC_EOVERFLOW, PIC_ECUDA, PIC_ETIMEOUT, PIC_ENAN, PIC_ESTATE = \
    0, -1, -2, -3, -4, -5, -6, -7, -8
PIC_FP64, PIC_MIXED = 0, 1
EX, EY, EZ, BX, BY, BZ, JX, JY, JZ, RHO = range(10)
ELECTRONS, BEAM = 0, 2

STATUS_NAMES = {0: "PIC_OK", -1: "PIC_EINVAL", -2: "PIC_ENOMEM", -3: "PIC_ECFL", -4: "PIC_EOVERFLOW",
                -5: "PIC_ECUDA", -6: "PIC_ETIMEOUT", -7: "PIC_ENAN", -8: "PIC_ESTATE"}

# every symbol include/pic.h declares
EXPORTS = ("pic_init", "pic_load_plasma", "pic_inject_laser", "pic_step", "pic_sync", "pic_boosted_to_lab_diag",
           "pic_free", "pic_get_field", "pic_set_field", "pic_get_particles", "pic_get_stats",
           "pic_get_particles_y", "pic_last_error",
           "pic_kernel_launches", "pic_kernel_timing", "pic_get_rho_noalloc", "pic_autotune",
           "pic_autotune_window",
           "pic_ensemble_create", "pic_ensemble_step", "pic_ensemble_sync", "pic_ensemble_size",
           "pic_ensemble_member", "pic_ensemble_free", "pic_ensemble_autotune",
           "pic_mlp_create", "pic_mlp_free", "pic_mlp_param_count", "pic_mlp_get_params", "pic_mlp_set_params",
           "pic_mlp_infer", "pic_mlp_grad", "pic_mlp_train", "pic_mlp_use_tensor_cores", "pic_mlp_use_graphs",
           "pic_mlp_status",
           "pic_measure_fp32_peak", "pic_beam_self_field", "pic_ensemble_batched", "pic_ensemble_use_graphs",
           "pic_ensemble_launches")
NOALLOC_MAX_NZ = 16384

_D = ctypes.POINTER(ctypes.c_double)


class PicConfig(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32), ("version", ctypes.c_uint32),
        ("dim", ctypes.c_int32), ("nx", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("dz_lab", ctypes.c_double), ("dx", ctypes.c_double), ("gamma_boost", ctypes.c_double),
        ("courant", ctypes.c_double), ("dt", ctypes.c_double),
        ("ck_alpha", ctypes.c_double), ("ck_beta", ctypes.c_double), ("ck_gamma", ctypes.c_double),
        ("theta", ctypes.c_double),
        ("pml_cells", ctypes.c_int32), ("pml_sigma_max", ctypes.c_double), ("pml_delta", ctypes.c_double),
        ("pml_power", ctypes.c_double), ("pml_xi_exp", ctypes.c_int32),
        ("filter_passes", ctypes.c_int32), ("filter_stride", ctypes.c_int32), ("filter_compensate", ctypes.c_int32),
        ("filter_J", ctypes.c_int32), ("filter_gather", ctypes.c_int32),
        ("shape_order", ctypes.c_int32), ("particle_guard", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("moving_window", ctypes.c_int32), ("window_beta", ctypes.c_double),
        ("tile_x", ctypes.c_int32), ("tile_z", ctypes.c_int32), ("sort_every", ctypes.c_int32),
        ("ny", ctypes.c_int32), ("gather_scheme", ctypes.c_int32), ("dy", ctypes.c_double),
        ("filter_stride_set", ctypes.c_int32 * 4),
    ]


class PicPlasma(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32), ("version", ctypes.c_uint32),
        ("n0", ctypes.c_double), ("z_start_lab", ctypes.c_double), ("ramp_lab", ctypes.c_double),
        ("length_lab", ctypes.c_double), ("ppc_x", ctypes.c_int32), ("ppc_z", ctypes.c_int32),
        ("ions", ctypes.c_int32),
        ("beam_n", ctypes.c_int64),
        ("beam_x", _D), ("beam_z", _D), ("beam_ux", _D), ("beam_uy", _D), ("beam_uz", _D),
        ("beam_t_lab", ctypes.c_double), ("beam_z_plane_lab", ctypes.c_double),
        ("beam_y", _D), ("ppc_y", ctypes.c_int32), ("beam_self", ctypes.c_int32), ("beam_w", _D),
        ("reserved", ctypes.c_int32 * 2),
    ]


class PicLaser(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32), ("version", ctypes.c_uint32),
        ("lambda0", ctypes.c_double), ("a0", ctypes.c_double), ("w0", ctypes.c_double),
        ("tau_fwhm", ctypes.c_double), ("t_peak", ctypes.c_double), ("x_center", ctypes.c_double),
        ("phase", ctypes.c_double), ("z_antenna", ctypes.c_double), ("beta_s", ctypes.c_double),
        ("y_center", ctypes.c_double), ("reserved", ctypes.c_int32 * 6),
    ]


class PicBtdReq(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("version", ctypes.c_uint32), ("n_rows", ctypes.c_int64),
                ("z_lab", _D), ("t_lab", _D)]


class PicBtdOut(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("version", ctypes.c_uint32), ("data", ctypes.c_void_p),
                ("done", ctypes.POINTER(ctypes.c_int32)), ("on_device", ctypes.c_int32),
                ("n_rows_filled", ctypes.c_int64)]


class PicStats(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32), ("version", ctypes.c_uint32),
        ("step", ctypes.c_int64), ("t", ctypes.c_double),
        ("dt", ctypes.c_double), ("dx", ctypes.c_double), ("dz", ctypes.c_double),
        ("gamma", ctypes.c_double), ("beta", ctypes.c_double),
        ("n_electrons", ctypes.c_int64), ("n_beam_active", ctypes.c_int64),
        ("beam_gamma_lab", ctypes.c_double), ("beam_spread", ctypes.c_double), ("field_energy", ctypes.c_double),
        ("gx_lo", ctypes.c_int32), ("gx_hi", ctypes.c_int32), ("gz_lo", ctypes.c_int32), ("gz_hi", ctypes.c_int32),
        ("sorts", ctypes.c_int64), ("overflow_chunks", ctypes.c_int64),
        ("z0", ctypes.c_double),
        ("trap_gamma_lab", ctypes.c_double), ("trapped_charge", ctypes.c_double),
    ]


TUNE_MAX_TRIALS = 16


class PicTuneResult(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32), ("version", ctypes.c_uint32),
        ("tile_x", ctypes.c_int32), ("tile_z", ctypes.c_int32), ("sort_every", ctypes.c_int32),
        ("ms_per_step", ctypes.c_double), ("n_trials", ctypes.c_int32),
        ("trial_tile_x", ctypes.c_int32 * TUNE_MAX_TRIALS), ("trial_tile_z", ctypes.c_int32 * TUNE_MAX_TRIALS),
        ("trial_sort_every", ctypes.c_int32 * TUNE_MAX_TRIALS), ("trial_ms", ctypes.c_double * TUNE_MAX_TRIALS),
        ("cached", ctypes.c_int32),
    ]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return os.path.join(HERE, "_build", "libpicgb.so")


def load(build_if_missing: bool = True):
    """Load libpicgb.so (building it with nvcc first when it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import build as _b
        path = library_path()
        if build_if_missing and not _b.up_to_date():
            path = _b.build()
        if not os.path.exists(path):
            raise RuntimeError("libpicgb.so is not built; run paper_1009_2727_gb300/build.py")
        L = ctypes.CDLL(path)
        vp = ctypes.c_void_p
        L.pic_init.argtypes = [ctypes.POINTER(PicConfig), ALLOC_FN, FREE_FN, vp, vp, ctypes.POINTER(vp)]
        L.pic_load_plasma.argtypes = [vp, ctypes.POINTER(PicPlasma)]
        L.pic_inject_laser.argtypes = [vp, ctypes.POINTER(PicLaser)]
        L.pic_step.argtypes = [vp, ctypes.c_int]
        L.pic_sync.argtypes = [vp]
        L.pic_boosted_to_lab_diag.argtypes = [vp, ctypes.POINTER(PicBtdReq), ctypes.POINTER(PicBtdOut)]
        L.pic_free.argtypes = [vp]
        L.pic_get_field.argtypes = [vp, ctypes.c_int, _D, ctypes.c_int]
        L.pic_set_field.argtypes = [vp, ctypes.c_int, _D]
        L.pic_get_particles.argtypes = [vp, ctypes.c_int, _D, _D, _D, _D, _D, _D,
                                        ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(ctypes.c_int64)]
        L.pic_get_stats.argtypes = [vp, ctypes.POINTER(PicStats)]
        L.pic_get_particles_y.argtypes = [vp, ctypes.c_int, _D, ctypes.POINTER(ctypes.c_int64)]
        L.pic_last_error.argtypes = [vp]
        L.pic_last_error.restype = ctypes.c_char_p
        L.pic_kernel_launches.argtypes = [vp]
        L.pic_kernel_launches.restype = ctypes.c_int64
        L.pic_kernel_timing.argtypes = [vp, ctypes.c_int, ctypes.c_int, _D, ctypes.POINTER(ctypes.c_int64)]
        L.pic_get_rho_noalloc.argtypes = [vp, _D]
        L.pic_ensemble_create.argtypes = [ctypes.c_int, ctypes.POINTER(PicConfig), ctypes.POINTER(PicPlasma),
                                          ctypes.POINTER(PicLaser), ALLOC_FN, FREE_FN, vp, vp, ctypes.POINTER(vp)]
        L.pic_ensemble_step.argtypes = [vp, ctypes.c_int]
        L.pic_ensemble_sync.argtypes = [vp]
        L.pic_ensemble_size.argtypes = [vp]
        L.pic_ensemble_member.argtypes = [vp, ctypes.c_int]
        L.pic_ensemble_member.restype = vp
        L.pic_ensemble_free.argtypes = [vp]
        L.pic_ensemble_autotune.argtypes = [ctypes.c_int, ctypes.POINTER(PicConfig), ctypes.POINTER(PicPlasma),
                                            ctypes.POINTER(PicLaser), ctypes.c_int, ALLOC_FN, FREE_FN, vp, vp,
                                            ctypes.POINTER(PicTuneResult)]
        _F = ctypes.POINTER(ctypes.c_float)
        L.pic_mlp_create.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_uint64, ALLOC_FN, FREE_FN,
                                     vp, vp, ctypes.POINTER(vp)]
        L.pic_mlp_free.argtypes = [vp]
        L.pic_mlp_param_count.argtypes = [vp]
        L.pic_mlp_param_count.restype = ctypes.c_int64
        L.pic_mlp_get_params.argtypes = [vp, _F]
        L.pic_mlp_set_params.argtypes = [vp, _F]
        L.pic_mlp_infer.argtypes = [vp, vp, ctypes.c_int64, vp]
        L.pic_mlp_use_tensor_cores.argtypes = [vp, ctypes.c_int]
        L.pic_mlp_use_graphs.argtypes = [vp, ctypes.c_int]
        L.pic_mlp_status.argtypes = [vp]
        L.pic_mlp_grad.argtypes = [vp, vp, vp, ctypes.c_int, _F, _F]
        L.pic_mlp_train.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                    ctypes.c_float, ctypes.c_uint64, _F]
        L.pic_autotune.argtypes = [ctypes.POINTER(PicConfig), ctypes.POINTER(PicPlasma), ctypes.POINTER(PicLaser),
                                   ctypes.c_int, ALLOC_FN, FREE_FN, vp, vp, ctypes.POINTER(PicTuneResult)]
        L.pic_autotune_window.argtypes = [ctypes.POINTER(PicConfig), ctypes.POINTER(PicPlasma),
                                          ctypes.POINTER(PicLaser), ctypes.c_int, ctypes.c_int, ALLOC_FN, FREE_FN,
                                          vp, vp, ctypes.POINTER(PicTuneResult)]
        L.pic_measure_fp32_peak.argtypes = [_D, _D]
        L.pic_beam_self_field.argtypes = [vp]
        L.pic_ensemble_batched.argtypes = [vp]
        L.pic_ensemble_use_graphs.argtypes = [vp, ctypes.c_int]
        L.pic_ensemble_launches.argtypes = [vp]
        L.pic_ensemble_launches.restype = ctypes.c_int64
        _lib = L
        return L

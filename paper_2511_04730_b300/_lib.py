"""ctypes declarations of the C ABI in include/lloid.h.

Loading fails loudly when the shared library is missing: there is no
fallback path.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblloid_b300.so")

LLOID_OK = 0
STATUS_NAMES = {
    0: "LLOID_OK", -1: "LLOID_EINVAL", -2: "LLOID_ENOMEM", -3: "LLOID_EBUDGET", -4: "LLOID_EGAP",
    -5: "LLOID_ENOTREADY", -6: "LLOID_ETIMEOUT", -7: "LLOID_ECUDA", -8: "LLOID_ERANGE", -9: "LLOID_EEXPIRED",
}
PRECISIONS = {"fp32": 0, "fp16_split": 1, "bf16_split": 2}


class LloidConfig(ctypes.Structure):
    _fields_ = [
        ("f0", ctypes.c_int32), ("n_detectors", ctypes.c_int32), ("n_down", ctypes.c_int32),
        ("n_up", ctypes.c_int32), ("window_samples", ctypes.c_int64), ("window_overlap", ctypes.c_int64),
        ("snr_threshold", ctypes.c_float), ("precision", ctypes.c_int32), ("max_block", ctypes.c_int64),
        ("max_history", ctypes.c_int64), ("min_rate", ctypes.c_int32), ("device", ctypes.c_int32),
        ("hbm_budget_bytes", ctypes.c_size_t), ("cuda_stream", ctypes.c_void_p), ("flags", ctypes.c_uint32),
        ("coinc_window", ctypes.c_int32), ("form_ratio", ctypes.c_float), ("fir_ctas", ctypes.c_int32),
    ]


class LloidTuning(ctypes.Structure):
    _fields_ = [
        ("form_ratio", ctypes.c_float), ("flags_form", ctypes.c_uint32), ("fir_ctas", ctypes.c_int32),
        ("n_tried", ctypes.c_int32), ("best", ctypes.c_int32), ("ms", ctypes.c_float * 16),
        ("cand_ratio", ctypes.c_float * 16), ("cand_flags", ctypes.c_uint32 * 16), ("cand_ctas", ctypes.c_int32 * 16),
    ]


class LloidSlice(ctypes.Structure):
    _fields_ = [
        ("rate", ctypes.c_int32), ("n_taps", ctypes.c_int32), ("j_start", ctypes.c_int64),
        ("n_basis", ctypes.c_int32), ("pad0", ctypes.c_int32),
        ("bases", ctypes.POINTER(ctypes.c_double)), ("coeffs", ctypes.POINTER(ctypes.c_double)),
    ]


class LloidBankDesc(ctypes.Structure):
    _fields_ = [("n_templates", ctypes.c_int32), ("n_slices", ctypes.c_int32),
                ("slices", ctypes.POINTER(LloidSlice)), ("ac_half", ctypes.c_int32), ("pad1", ctypes.c_int32),
                ("autocorr", ctypes.POINTER(ctypes.c_double))]


class LloidTrigger(ctypes.Structure):
    _fields_ = [
        ("detector", ctypes.c_int32), ("bank", ctypes.c_int32), ("tmpl", ctypes.c_int32),
        ("is_bank_max", ctypes.c_int32), ("window", ctypes.c_int64), ("sample", ctypes.c_int64),
        ("snr", ctypes.c_float), ("phase", ctypes.c_float), ("re", ctypes.c_float), ("im", ctypes.c_float),
        ("xi2", ctypes.c_float), ("pad", ctypes.c_int32),
    ]


class LloidEvent(ctypes.Structure):
    _fields_ = [
        ("window", ctypes.c_int64), ("bank", ctypes.c_int32), ("tmpl", ctypes.c_int32), ("n_ifo", ctypes.c_int32),
        ("ifo_mask", ctypes.c_uint32), ("net_snr", ctypes.c_float), ("ref_detector", ctypes.c_int32),
        ("ref_sample", ctypes.c_int64),
    ]


class LloidWhitenerConfig(ctypes.Structure):
    _fields_ = [
        ("rate_in", ctypes.c_int32), ("rate_out", ctypes.c_int32), ("n_fft", ctypes.c_int32), ("z_pad", ctypes.c_int32),
        ("n_med", ctypes.c_int32), ("n_avg", ctypes.c_int32), ("n_detectors", ctypes.c_int32), ("device", ctypes.c_int32),
        ("max_push", ctypes.c_int64), ("cuda_stream", ctypes.c_void_p),
    ]


# (name, restype, argtypes) for every entry point of include/lloid.h
SIGNATURES = [
    ("lloid_config_default", None, [ctypes.POINTER(LloidConfig)]),
    ("lloid_create", ctypes.c_int, [ctypes.POINTER(LloidConfig), ctypes.POINTER(ctypes.c_void_p)]),
    ("lloid_destroy", None, [ctypes.c_void_p]),
    ("lloid_strerror", ctypes.c_char_p, [ctypes.c_int]),
    ("lloid_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    ("lloid_load_bank", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(LloidBankDesc), ctypes.POINTER(ctypes.c_int32)]),
    ("lloid_unload_bank", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    ("lloid_push_strain", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p,
                                         ctypes.c_int64, ctypes.c_int]),
    ("lloid_push_strain_all", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                             ctypes.c_int]),
    ("lloid_pull_triggers", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(LloidTrigger),
                                           ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32]),
    ("lloid_set_background_bins", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float), ctypes.c_int32,
                                                 ctypes.POINTER(ctypes.c_float), ctypes.c_int32]),
    ("lloid_get_background", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_uint32),
                                            ctypes.c_int64]),
    ("lloid_whitener_config_default", None, [ctypes.POINTER(LloidWhitenerConfig)]),
    ("lloid_whitener_create", ctypes.c_int, [ctypes.POINTER(LloidWhitenerConfig), ctypes.POINTER(ctypes.c_void_p)]),
    ("lloid_whitener_destroy", None, [ctypes.c_void_p]),
    ("lloid_whiten", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                    ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), ctypes.c_int]),
    ("lloid_whitener_psd", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_float),
                                          ctypes.c_int64]),
    ("lloid_pull_events", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                         ctypes.POINTER(LloidEvent), ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                                         ctypes.c_int32]),
    ("lloid_pull_triggers_range", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                                 ctypes.POINTER(LloidTrigger), ctypes.c_int64,
                                                 ctypes.POINTER(ctypes.c_int64), ctypes.c_int32]),
    ("lloid_pull_submit", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                         ctypes.POINTER(ctypes.c_int32)]),
    ("lloid_pull_collect", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(LloidTrigger),
                                          ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32]),
    ("lloid_snr_block", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    ("lloid_synchronize", ctypes.c_int, [ctypes.c_void_p]),
    ("lloid_save_state", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    ("lloid_restore_state", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    ("lloid_launch_count", ctypes.c_int64, [ctypes.c_void_p]),
    ("lloid_bytes_in_use", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t),
                                          ctypes.POINTER(ctypes.c_size_t)]),
    ("lloid_stream", ctypes.c_void_p, [ctypes.c_void_p]),
    ("lloid_triggers_from_snr_noalloc", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_float,
      ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]),
    ("lloid_stage_times", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_int64), ctypes.c_int]),
    ("lloid_bank_form", ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32]),
    ("lloid_inject_fault", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64]),
    ("lloid_autotune", ctypes.c_int, [ctypes.POINTER(LloidConfig), ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                      ctypes.c_int32, ctypes.POINTER(LloidTuning)]),
    ("lloid_clear_error", ctypes.c_int, [ctypes.c_void_p]),
]

FLAG_STAGE_TIMING = 1
FORM_FLAGS = {None: 0, "ladder": 2, "f0": 4}     # LLOID_FLAG_FORM_LADDER, LLOID_FLAG_FORM_F0
FLAG_FILL_GAPS = 8
FAULTS = {"alloc": 1, "drop_block": 2, "delay": 3, "wait_expiry": 4}   # LLOID_FAULT_*
N_STAGES = 7
STAGE_NAMES = ("ingest", "downsample", "fir", "upsample", "recon", "finalize", "gather")

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the library (once) and declare every entry point."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"LLOID CUDA library not built: {path} is missing "
                           "(run paper_2511_04730_b300/build.py or __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib

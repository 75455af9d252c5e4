"""ctypes declarations of libwskpn.so (include/wskpn.h).  Marshalling only."""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libwskpn.so")

MAX_LAYERS = 8
MAX_KERNELS = 8
MAX_BATCH = 16

OK, EINVAL, ENOMEM, ECUDA, EUNSUPPORTED, EBUSY, ETIMEOUT, ENUMERIC = range(8)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "EUNSUPPORTED", "EBUSY", "ETIMEOUT", "ENUMERIC"]
FP32, BF16, FP8 = 0, 1, 2
TUNE_TC_SPLIT = 2
TUNE_TRAIN_RECOMPUTE = 3
TUNE_TC_SPLIT_LAYERS = 8
TUNE_FP8_SPLIT = 4
TUNE_HOST_BANDS = 5
TUNE_HOST_FIRST_BAND = 6
TUNE_HOST_LAST_BAND = 7
TUNE_WAIT_LIMIT_US = 9
TUNE_WAIT_PROBE = 10
TUNE_TRAIN_KEEP = 11
TUNE_FUSED_PREP = 12


class Config(ctypes.Structure):
    _fields_ = [
        ("n_layers", ctypes.c_int),
        ("widths", ctypes.c_int * (MAX_LAYERS + 1)),
        ("conv_ks", ctypes.c_int),
        ("n_kernels", ctypes.c_int),
        ("ksizes", ctypes.c_int * MAX_KERNELS),
        ("prec", ctypes.c_int),
        ("albedo_eps", ctypes.c_float),
        ("gamma", ctypes.c_float),
        ("depth_near", ctypes.c_float),
        ("depth_far", ctypes.c_float),
        ("max_batch", ctypes.c_int),
        ("max_h", ctypes.c_int),
        ("max_w", ctypes.c_int),
    ]


class Frame(ctypes.Structure):
    _fields_ = [("radiance", ctypes.c_void_p), ("albedo", ctypes.c_void_p),
                ("normal", ctypes.c_void_p), ("depth", ctypes.c_void_p)]


class TemporalConfig(ctypes.Structure):
    _fields_ = [("alpha_min", ctypes.c_float), ("tau_pos", ctypes.c_float), ("tau_normal", ctypes.c_float),
                ("min_weight", ctypes.c_float)]


class MrConfig(ctypes.Structure):
    _fields_ = [("max_h", ctypes.c_int), ("max_w", ctypes.c_int), ("albedo_eps", ctypes.c_float),
                ("gamma", ctypes.c_float), ("depth_near", ctypes.c_float), ("depth_far", ctypes.c_float),
                ("prec", ctypes.c_int)]


class ServeConfig(ctypes.Structure):
    _fields_ = [("n_workers", ctypes.c_int), ("max_batch", ctypes.c_int), ("max_queue", ctypes.c_int),
                ("mem_budget", ctypes.c_size_t), ("use_graphs", ctypes.c_int), ("batch_window_us", ctypes.c_int),
                ("temporal", TemporalConfig)]


class ServeStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("batches", ctypes.c_uint64), ("graph_launches", ctypes.c_uint64),
                ("graph_captures", ctypes.c_uint64), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("max_ms", ctypes.c_double), ("fps", ctypes.c_double),
                ("mean_batch", ctypes.c_double), ("mem_in_use", ctypes.c_size_t), ("mem_peak", ctypes.c_size_t),
                ("temporal_frames", ctypes.c_uint64), ("temporal_streams", ctypes.c_uint64),
                ("temporal_bytes", ctypes.c_size_t)]


class ServeTicketInfo(ctypes.Structure):
    _fields_ = [("h", ctypes.c_int), ("w", ctypes.c_int), ("worker", ctypes.c_int), ("batch", ctypes.c_int),
                ("submit_ms", ctypes.c_double), ("dispatch_ms", ctypes.c_double), ("done_ms", ctypes.c_double)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_F = ctypes.c_float
_SZ = ctypes.c_size_t
_FR = ctypes.POINTER(Frame)

# name -> (argtypes, restype): the exported C ABI, in header order
SIGNATURES = {
    "wskpn_version": ([], ctypes.c_char_p),
    "wskpn_config_default": ([ctypes.POINTER(Config)], _I),
    "wskpn_n_weights": ([ctypes.POINTER(Config)], _SZ),
    "wskpn_create": ([ctypes.POINTER(Config), _P, _SZ, ctypes.POINTER(_P)], _I),
    "wskpn_destroy": ([_P], None),
    "wskpn_last_error": ([_P], ctypes.c_char_p),
    "wskpn_set_weights": ([_P, _P, _SZ, _I, _P], _I),
    "wskpn_get_weights": ([_P, _P, _SZ, _P], _I),
    "wskpn_denoise": ([_P, _FR, _I, _I, _I, _P, _P], _I),
    "wskpn_denoise_host": ([_P, _FR, _I, _I, _I, _P, _P], _I),
    "wskpn_denoise_host_async": ([_P, _FR, _I, _I, _I, _P, _P], _I),
    "wskpn_logits": ([_P, _FR, _I, _I, _I, _P, _P], _I),
    "wskpn_prep": ([_FR, _I, _I, _I, _F, _F, _F, _P, _P], _I),
    "wskpn_decode_fuse_fwd": ([_P, _P, _P, _I, _I, _I, _I, ctypes.POINTER(_I), _F, _P, _P, _P], _I),
    "wskpn_calibrate": ([_P, _FR, _I, _I, _I, _F, _P], _I),
    "wskpn_decode_fuse_bwd_scratch_floats": ([_I, _I, _I, _I], _SZ),
    "wskpn_decode_fuse_bwd": ([_P, _P, _P, _P, _I, _I, _I, _I, ctypes.POINTER(_I), _F, _P, _P, _P, _P], _I),
    "wskpn_forward_train": ([_P, _FR, _I, _I, _I, _P, _P, _P], _I),
    "wskpn_backward": ([_P, _FR, _I, _I, _I, _P, _P, _P, _P, _P], _I),
    "wskpn_l1_loss": ([_P, _P, _P, _SZ, _P, _P, _P], _I),
    "wskpn_adam_step": ([_P, _P, _F, _F, _F, _F, _I, _P], _I),
    "wskpn_repvgg_fold": ([_P, _P, _P, _P, _P, _P, _I, _I, _I, _P, _P, _P], _I),
    "wskpn_repvgg_fold_grad": ([_P, _I, _I, _P, _P, _P, _P], _I),
    "wskpn_temporal_config_default": ([_P], None),
    "wskpn_temporal_create": ([_P, _I, _I, _P], _I),
    "wskpn_temporal_step": ([_P, _P, _P, _P, _P, _P, _P], _I),
    "wskpn_temporal_history": ([_P, _P, _P], _I),
    "wskpn_temporal_reset": ([_P, _P], _I),
    "wskpn_temporal_destroy": ([_P], None),
    "wskpn_mr_config_default": ([_P], None),
    "wskpn_mr_n_weights": ([], _SZ),
    "wskpn_mr_create": ([_P, _P, _SZ, _P], _I),
    "wskpn_mr_denoise": ([_P, _FR, _I, _I, _P, _P], _I),
    "wskpn_mr_logits": ([_P, _FR, _I, _I, _P, _P, _P, _P], _I),
    "wskpn_mr_last_error": ([_P], ctypes.c_char_p),
    "wskpn_mr_destroy": ([_P], None),
    "wskpn_serve_config_default": ([ctypes.POINTER(ServeConfig)], _I),
    "wskpn_serve_start": ([ctypes.POINTER(Config), _P, _SZ, ctypes.POINTER(ServeConfig), ctypes.POINTER(_P)], _I),
    "wskpn_serve_submit": ([_P, _I, _FR, _I, _I, _P, ctypes.POINTER(ctypes.c_uint64)], _I),
    "wskpn_serve_submit_temporal": ([_P, _I, _FR, _P, _P, _I, _I, _I, _P, ctypes.POINTER(ctypes.c_uint64)], _I),
    "wskpn_serve_wait": ([_P, ctypes.c_uint64, _I], _I),
    "wskpn_serve_wait_info": ([_P, ctypes.c_uint64, _I, ctypes.POINTER(ServeTicketInfo)], _I),
    "wskpn_serve_pause": ([_P, _I], _I),
    "wskpn_serve_stats_get": ([_P, ctypes.POINTER(ServeStats)], _I),
    "wskpn_serve_stop": ([_P], None),
    "wskpn_numeric_fallbacks": ([_P, ctypes.POINTER(ctypes.c_uint64)], _I),
    "wskpn_profile_enable": ([_P, _I], _I),
    "wskpn_profile_read": ([_P, ctypes.POINTER(_F), _I, ctypes.POINTER(_I), ctypes.POINTER(_I)], _I),
    "wskpn_set_tuning": ([_P, _I, _I], _I),
    "wskpn_device_status": ([_P, ctypes.POINTER(ctypes.c_uint32)], _I),
    "wskpn_denoise_static": ([ctypes.POINTER(Config), _P, _FR, _I, _I, _I, _P, _P], _I),
}

_lib = None


class WskpnError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"wskpn {name}: {msg}")


def load() -> ctypes.CDLL:
    """Loads the in-tree libwskpn.so; raises ImportError when it is missing
    (there is no fallback implementation)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is not built: run `python -m paper_2202_05977_b300.build`")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
    return _lib


def check(status: int, ctx=None) -> None:
    if status != OK:
        msg = load().wskpn_last_error(ctx)
        raise WskpnError(status, msg.decode() if msg else "")

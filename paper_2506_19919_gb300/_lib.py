"""ctypes binding of the C ABI in include/sps.h (argument marshalling only).

Every compute step runs in the CUDA library; this module only declares the
structs and prototypes and loads the in-tree shared library.  It raises if
the library is missing: there is no CPU fallback."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libsps_gb300.so")

NPARAM = 12
MAX_BANDS = 32

SPS_OK = 0
STATUS_NAMES = {0: "SPS_OK", 1: "SPS_E_INVALID_ARG", 2: "SPS_E_SHAPE", 3: "SPS_E_NONFINITE",
                4: "SPS_E_CUDA", 5: "SPS_E_TIMEOUT", 6: "SPS_E_UNSUPPORTED", 7: "SPS_E_STATE",
                8: "SPS_E_NOMEM"}
SPS_EXACT, SPS_APPROX = 0, 1
SPS_FP32, SPS_BF16, SPS_TF32X3 = 0, 1, 2


class sps_tables(C.Structure):
    _fields_ = [("n_age", C.c_int32), ("n_met", C.c_int32), ("n_lam", C.c_int32),
                ("n_band", C.c_int32), ("age_yr", C.c_void_p), ("lgZ", C.c_void_p),
                ("lam_ang", C.c_void_p), ("ssp", C.c_void_p), ("band_kind", C.c_void_p),
                ("band_p0", C.c_void_p), ("band_p1", C.c_void_p), ("band_tab_n", C.c_void_p),
                ("band_tab_T", C.c_void_p), ("mdf_offset", C.c_void_p)]


class sps_config(C.Structure):
    _fields_ = [("h0_kms_mpc", C.c_double), ("omega_m", C.c_double),
                ("prior_lo", C.c_double * NPARAM), ("prior_hi", C.c_double * NPARAM),
                ("device", C.c_int32), ("sfh_gl_order", C.c_int32), ("sfh_panel", C.c_double),
                ("sigmoid_k", C.c_double * NPARAM), ("sigmoid_x0", C.c_double * NPARAM), ("prior", C.c_int32),
                ("skew_xi", C.c_double * NPARAM), ("skew_omega", C.c_double * NPARAM),
                ("skew_s", C.c_double * NPARAM)]


class sps_hmc_config(C.Structure):
    _fields_ = [("chains_per_gal", C.c_int32), ("n_warm", C.c_int32), ("n_samp", C.c_int32),
                ("L_min", C.c_int32), ("L_max", C.c_int32), ("target_accept", C.c_float),
                ("eps0", C.c_float), ("seed", C.c_uint64), ("mode", C.c_int32),
                ("prec", C.c_int32), ("use_graph", C.c_int32), ("autotune", C.c_int32),
                ("adapt_mass", C.c_int32), ("sampler", C.c_int32), ("max_depth", C.c_int32)]


class sps_hmc_stats(C.Structure):
    _fields_ = [("accept_prob", C.c_void_p), ("step_size", C.c_void_p),
                ("divergences", C.c_void_p), ("grad_evals", C.c_void_p), ("status", C.c_void_p)]


class sps_info(C.Structure):
    _fields_ = [("n_age", C.c_int32), ("n_met", C.c_int32), ("n_lam", C.c_int32),
                ("n_band", C.c_int32), ("k_pad", C.c_int32), ("n_gal", C.c_int64),
                ("has_approx", C.c_int32), ("device", C.c_int32), ("sfh_gl_order", C.c_int32),
                ("max_panels", C.c_int32), ("hmc_launches", C.c_int32)]


_P = C.c_void_p
_PROTOS = {
    "sps_config_default": (C.c_int, [C.POINTER(sps_config)]),
    "sps_hmc_config_default": (C.c_int, [C.POINTER(sps_hmc_config)]),
    "sps_create": (C.c_int, [C.POINTER(_P), C.POINTER(sps_tables), C.POINTER(sps_config)]),
    "sps_destroy": (C.c_int, [_P]),
    "sps_set_galaxies": (C.c_int, [_P, _P, C.c_int64, C.c_int32, _P]),
    "sps_photometry": (C.c_int, [_P, _P, _P, C.c_int64, C.c_int, C.c_int, _P, _P]),
    "sps_loglike_grad": (C.c_int, [_P, _P, _P, C.c_int64, _P, _P, _P, C.c_int, C.c_int, _P, _P,
                                   _P]),
    "sps_loglike_grad_z": (C.c_int, [_P, _P, _P, C.c_int64, _P, _P, _P, C.c_int, C.c_int, _P, _P,
                                   _P]),
    "sps_loglike_grad_forward_mode": (C.c_int, [_P, _P, _P, C.c_int64, _P, _P, _P, _P, _P, _P]),
    "sps_wait_probe": (C.c_int, [_P, C.c_int32, C.c_uint32, _P]),
    "sps_hmc_run": (C.c_int, [_P, C.POINTER(sps_hmc_config), _P, _P, _P, _P, _P,
                              C.POINTER(sps_hmc_stats), _P]),
    "sps_hmc_run_forward_mode": (C.c_int, [_P, C.POINTER(sps_hmc_config), _P, _P, _P, _P, _P,
                                           C.POINTER(sps_hmc_stats), _P]),
    "sps_leapfrog": (C.c_int, [_P, _P, _P, _P, _P, _P, C.c_int64, _P, _P, _P, _P, _P, _P, _P]),
    "sps_philox": (C.c_int, [_P, _P, C.c_int64, C.c_uint64, _P, _P]),
    "sps_weights": (C.c_int, [_P, _P, _P, C.c_int64, _P, _P, _P]),
    "sps_diagnostics": (C.c_int, [_P, C.c_int64, C.c_int32, C.c_int32, C.c_int32, _P, _P]),
    "sps_partition_galaxies": (C.c_int, [_P, C.c_int64, C.c_int32, C.c_int32, _P]),
    "sps_get_info": (C.c_int, [_P, C.POINTER(sps_info)]),
    "sps_gl_rule": (C.c_int, [_P, _P, _P]),
    "sps_photometry_exact_noalloc": (C.c_int, [_P, _P, _P, C.c_int64, _P, _P]),
    "sps_error_string": (C.c_char_p, [C.c_int]),
    "sps_last_error_message": (C.c_char_p, []),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the shared library (once) and declare its prototypes."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} is missing "
                          "(run `python -c 'import __graft_entry__ as g; g.build()'`)")
    lib = C.CDLL(path)
    for name, (res, args) in _PROTOS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class SpsError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load()
        msg = lib.sps_last_error_message().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)} ({msg})")
        self.status = status


def check(status: int, where: str):
    if status != SPS_OK:
        raise SpsError(status, where)

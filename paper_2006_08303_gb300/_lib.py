"""ctypes loader for libcip.so (the sm_103a CUDA library).

Fails loudly when the library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcip.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "cip.h")

c_int, c_double, c_size_t, c_void_p, c_char_p = ctypes.c_int, ctypes.c_double, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_char_p
P_int = ctypes.POINTER(ctypes.c_int)
P_double = ctypes.POINTER(ctypes.c_double)
P_size = ctypes.POINTER(ctypes.c_size_t)


class cip_options(ctypes.Structure):
    _fields_ = [("col_tile", c_int), ("check_every", c_int), ("column_pass", c_int), ("precision", c_int),
                ("prior_fft", c_int), ("reserved", c_int * 11)]


class cip_request(ctypes.Structure):
    _fields_ = [("N", c_int), ("K", c_int), ("M", c_int), ("prior", c_int), ("lam", c_double), ("rho", c_double),
                ("beta", c_double), ("h", c_void_p), ("y", c_void_p), ("x_out", c_void_p), ("tol", c_double),
                ("max_iter", c_int), ("psf_key", ctypes.c_ulonglong), ("rho_tau", c_double), ("rho_mu", c_double)]


class cip_result(ctypes.Structure):
    _fields_ = [("state", c_int), ("status", c_int), ("iterations", c_int), ("r_rel", c_double),
                ("s_rel", c_double), ("t_submit", c_double), ("t_admit", c_double), ("t_done", c_double)]


P_ull = ctypes.POINTER(ctypes.c_ulonglong)

# name -> (restype, argtypes)
SIGNATURES = {
    "cip_plan_create_on_stream": (c_int, [ctypes.POINTER(c_void_p), c_int, c_int, c_int, c_int,
                                          ctypes.POINTER(cip_options), c_void_p]),
    "cip_server_create": (c_int, [ctypes.POINTER(c_void_p), c_size_t, c_int, c_int]),
    "cip_server_submit": (c_int, [c_void_p, ctypes.POINTER(cip_request), P_ull]),
    "cip_server_poll": (c_int, [c_void_p, ctypes.c_ulonglong, ctypes.POINTER(cip_result)]),
    "cip_server_wait": (c_int, [c_void_p, ctypes.c_ulonglong, ctypes.POINTER(cip_result), c_double]),
    "cip_server_cancel": (c_int, [c_void_p, ctypes.c_ulonglong]),
    "cip_server_stats": (c_int, [c_void_p, P_double, P_int, P_int, P_size, P_int, P_int]),
    "cip_server_destroy": (c_int, [c_void_p]),
    "cip_version": (c_char_p, []),
    "cip_status_string": (c_char_p, [c_int]),
    "cip_wavelet_lowpass": (c_int, [c_int, P_double]),
    "cip_last_error": (c_char_p, [c_void_p]),
    "cip_plan_create": (c_int, [ctypes.POINTER(c_void_p), c_int, c_int, c_int, c_int, ctypes.POINTER(cip_options)]),
    "cip_plan_destroy": (c_int, [c_void_p]),
    "cip_plan_bytes": (c_size_t, [c_int, c_int, c_int, c_int, c_int]),
    "cip_set_prior": (c_int, [c_void_p, c_int, c_double, c_double, c_double, c_void_p]),
    "cip_set_psfs": (c_int, [c_void_p, c_void_p, c_void_p]),
    "cip_set_measurements": (c_int, [c_void_p, c_void_p, c_void_p]),
    "cip_reset_state": (c_int, [c_void_p, c_void_p]),
    "cip_iterate": (c_int, [c_void_p, c_int, c_double, P_int, c_void_p]),
    "cip_get_x": (c_int, [c_void_p, c_void_p, c_void_p]),
    "cip_get_u": (c_int, [c_void_p, c_void_p, c_void_p]),
    "cip_get_residuals": (c_int, [c_void_p, P_double, P_double]),
    "cip_get_iteration": (c_int, [c_void_p, P_int]),
    "cip_state_import": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "cip_state_size": (c_int, [c_void_p, P_size]),
    "cip_state_export": (c_int, [c_void_p, c_void_p, c_void_p]),
    "cip_state_restore": (c_int, [c_void_p, c_void_p, c_void_p]),
    "cip_set_timing": (c_int, [c_void_p, c_int]),
    "cip_set_test_fault": (c_int, [c_void_p, c_int]),
    "cip_get_timing": (c_int, [c_void_p, P_double, P_int, P_double, P_int]),
    "cip_get_config": (c_int, [c_void_p, P_int, P_int, P_int, P_int, P_int]),
    "cip_get_launches": (c_int, [c_void_p, ctypes.POINTER(ctypes.c_ulonglong)]),
    "cip_batch_create": (c_int, [ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p), c_int, c_int]),
    "cip_batch_iterate": (c_int, [c_void_p, c_int, c_void_p]),
    "cip_batch_last_error": (c_char_p, [c_void_p]),
    "cip_batch_destroy": (c_int, [c_void_p]),
    "cip_set_dictionary": (c_int, [c_void_p, c_void_p, c_int, c_int, c_void_p]),
    "cip_set_dictionary_3d": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_void_p]),
    "cip_set_code_gradient_weight": (c_int, [c_void_p, c_double]),
    "cip_set_dictionary_learning": (c_int, [c_void_p, c_double, c_void_p]),
    "cip_get_dictionary": (c_int, [c_void_p, c_void_p, c_void_p]),
    "cip_get_prior_fft": (c_int, [c_void_p, ctypes.POINTER(c_int)]),
    "cip_set_sigma_adaptation": (c_int, [c_void_p, c_double, c_double]),
    "cip_get_sigma": (c_int, [c_void_p, P_double]),
    "cip_set_rho_adaptation": (c_int, [c_void_p, c_double, c_double]),
    "cip_get_rho": (c_int, [c_void_p, P_double]),
    "cip_get_coefficients": (c_int, [c_void_p, c_void_p, c_void_p]),
    "cip_state_import_coefficients": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "cip_shrink_dual_noalloc": (c_int, [c_int, c_int, c_int, c_int, c_double, c_double, c_void_p, c_void_p,
                                        c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
}

_LIB = None


def header_symbols(path: str = HEADER):
    """Function names declared in include/cip.h."""
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(cip_[a-z0-9_]+)\s*\(", txt)))


def load(path: str = LIB_PATH):
    """Load libcip.so and declare every signature (no CUDA call is made)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()'); there is no CPU fallback")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib

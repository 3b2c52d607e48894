"""The C-ABI library builds, loads and exports every symbol include/cip.h
declares; argument checks and host-side logic that need no GPU.  CPU only (no device
compute call)."""
import ctypes

import numpy as np
import pytest

from paper_2006_08303_gb300 import _lib, build


@pytest.fixture(scope="module")
def L():
    build.build()
    return _lib.load()


def test_exports_every_declared_symbol(L):
    syms = _lib.header_symbols()
    assert len(syms) >= 20
    missing = [s for s in syms if not hasattr(L, s)]
    assert not missing, missing
    assert set(syms) == set(_lib.SIGNATURES), "binding and header disagree"


def test_status_strings_and_version(L):
    assert L.cip_version().startswith(b"cip")
    for s in range(8):
        assert len(L.cip_status_string(s)) > 0


def test_invalid_sizes_rejected_before_device_use(L):
    h = ctypes.c_void_p()
    opt = _lib.cip_options()
    assert L.cip_plan_create(ctypes.byref(h), 100, 3, 3, 0, ctypes.byref(opt)) == 2   # not a power of two
    assert b"power of two" in L.cip_last_error(None)
    assert L.cip_plan_create(ctypes.byref(h), 4096, 3, 3, 0, ctypes.byref(opt)) == 2
    assert L.cip_plan_create(ctypes.byref(h), 64, 3, 17, 0, ctypes.byref(opt)) == 2  # M > 16
    assert L.cip_plan_create(None, 64, 3, 3, 0, ctypes.byref(opt)) == 1
    assert L.cip_plan_create(ctypes.byref(h), 64, 3, 3, 7, ctypes.byref(opt)) == 1   # bad dtype
    assert L.cip_set_code_gradient_weight(None, 0.01) == 1                            # null plan
    assert L.cip_set_dictionary_learning(None, 1.0, None) == 1                         # null plan
    assert L.cip_get_dictionary(None, None, None) == 1


def test_plan_bytes_accounts_for_factor_and_state(L):
    # 512^2 x 10, f32, DCT: packed factor (55 planes of N*(N/2+4) complex64), its FP64 copy
    # and the kept FP64 PSF spectra (100 maps of N*(N/2+4) complex128) dominate
    b = L.cip_plan_bytes(512, 10, 10, 0, 1)
    factor = 55 * 512 * 260 * 8
    lam64 = 100 * 512 * 260 * 16
    assert 3 * factor + lam64 < b < 1.5 * (3 * factor + lam64)
    assert L.cip_plan_bytes(100, 1, 1, 0, 0) == 0
    assert L.cip_plan_bytes(512, 10, 10, 1, 1) > b
    # the wavelet prior adds its work planes: x / q and the coefficients (N^2 each) and two
    # lowpass bands of (N/2)^2 per channel, plus the M x M channel DCT
    assert L.cip_plan_bytes(512, 10, 10, 0, 5) - b == 10 * 512 * 512 * 4 * 5 // 2 + 100 * 4


def test_wavelet_filter_of_the_library_matches_the_oracle(L):
    """Host logic of the wavelet prior: the library builds its Symmlet filter itself (Aberth root
    finding and its own phase-linearity selection); it must agree with the oracle's independent
    construction (numpy roots, reading R24) for every supported number of vanishing moments."""
    from oracle import admm
    for p in range(1, 9):
        h = (ctypes.c_double * (2 * p))()
        assert L.cip_wavelet_lowpass(p, h) == 0
        assert np.abs(np.array(h[:]) - admm.symlet_lowpass(p)).max() < 1e-12, p
    h = (ctypes.c_double * 2)()
    assert L.cip_wavelet_lowpass(0, h) == 1 and L.cip_wavelet_lowpass(9, h) == 1
    assert L.cip_wavelet_lowpass(8, None) == 1

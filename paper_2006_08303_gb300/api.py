"""Python binding of the cip C ABI (include/cip.h), argument marshalling only.

Arrays may be CUDA torch tensors (device pointers), CPU torch tensors
(pinned or not) or numpy arrays (host pointers); every step of the
reconstruction runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Tuple

import numpy as np

from . import _lib

PRIORS = {"tv": 0, "dct8": 1, "l1": 2, "convdict": 3, "tv_iso": 4, "wdct": 5}
DTYPES = {"f32": 0, "f64": 1}
NP_DTYPE = {"f32": np.float32, "f64": np.float64}


class CipError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"cip error {status}: {msg}")
        self.status = status


def _torch():
    import torch
    return torch


def _ptr_and_check(a, dtype: str, shape: Tuple[int, ...]):
    """Return (pointer, keepalive) for a contiguous array of the plan dtype and shape."""
    want = NP_DTYPE[dtype]
    if isinstance(a, np.ndarray):
        if a.dtype != want:
            raise TypeError(f"expected {np.dtype(want)}, got {a.dtype}")
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        if tuple(a.shape) != tuple(shape):
            raise ValueError(f"expected shape {shape}, got {a.shape}")
        return a.ctypes.data, a
    torch = _torch()
    if isinstance(a, torch.Tensor):
        tdt = torch.float32 if dtype == "f32" else torch.float64
        if a.dtype != tdt:
            raise TypeError(f"expected {tdt}, got {a.dtype}")
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if tuple(a.shape) != tuple(shape):
            raise ValueError(f"expected shape {shape}, got {tuple(a.shape)}")
        return a.data_ptr(), a
    raise TypeError(f"unsupported array type {type(a)}")


def _stream_ptr(stream):
    if stream is None:
        torch = _torch()
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        return ctypes.c_void_p(0)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def version() -> str:
    return _lib.load().cip_version().decode()


def wavelet_lowpass(p: int = 8) -> np.ndarray:
    """Lowpass taps of the wavelet prior's filter with p vanishing moments (cip_wavelet_lowpass)."""
    h = (ctypes.c_double * (2 * p))()
    st = _lib.load().cip_wavelet_lowpass(p, h)
    if st != 0:
        raise CipError(st, "cip_wavelet_lowpass: p must be in [1, 8]")
    return np.array(h[:], dtype=np.float64)


def plan_bytes(N: int, K: int, M: int, dtype: str = "f32", prior: str = "tv") -> int:
    return int(_lib.load().cip_plan_bytes(N, K, M, DTYPES[dtype], PRIORS[prior]))


class Plan:
    """One reconstruction instance held on the device (cip_plan)."""

    def __init__(self, N: int, K: int, M: int, dtype: str = "f32", col_tile: int = 0, check_every: int = 0,
                 column_pass: int = 0, plain_fp32: bool = False, prior_fft: int = 0):
        self._L = _lib.load()
        self.N, self.K, self.M, self.dtype = N, K, M, dtype
        self.prior: Optional[str] = None
        opt = _lib.cip_options()
        opt.col_tile = col_tile
        opt.check_every = check_every
        opt.column_pass = column_pass
        opt.precision = 1 if plain_fp32 else 0
        opt.prior_fft = prior_fft
        h = ctypes.c_void_p()
        st = self._L.cip_plan_create(ctypes.byref(h), N, K, M, DTYPES[dtype], ctypes.byref(opt))
        if st != 0:
            raise CipError(st, self._L.cip_last_error(None).decode())
        self._h = h

    # -- helpers
    def _check(self, st: int):
        if st != 0:
            raise CipError(st, self._L.cip_last_error(self._h).decode())

    @property
    def ncomp(self) -> int:
        return 2 if self.prior in ("tv", "tv_iso") else 1

    @property
    def state_shape(self):
        """Shape of t and u: [M][ncomp][N][N], or [M][L][N][N] for the convolutional dictionary."""
        if self.prior == "convdict":
            return (self.M, self.L, self.N, self.N)
        return (self.M, self.ncomp, self.N, self.N)

    def set_dictionary(self, filters, stream=None):
        """Filters [L][P][P] of the convolutional dictionary (after set_prior('convdict', ...))."""
        L, P = int(filters.shape[0]), int(filters.shape[-1])
        p, keep = _ptr_and_check(filters, self.dtype, (L, P, P))
        self._check(self._L.cip_set_dictionary(self._h, ctypes.c_void_p(p), L, P, _stream_ptr(stream)))
        self.L = L
        self.filter_size = P

    def set_dictionary_3d(self, filters, stream=None):
        """3D filters [L][Q][P][P] of the convolutional dictionary (Section IV-B, 3D case;
        cip_set_dictionary_3d), after set_prior('convdict', ...)."""
        L, Q, P = int(filters.shape[0]), int(filters.shape[1]), int(filters.shape[-1])
        p, keep = _ptr_and_check(filters, self.dtype, (L, Q, P, P))
        self._check(self._L.cip_set_dictionary_3d(self._h, ctypes.c_void_p(p), L, Q, P, _stream_ptr(stream)))
        self.L = L
        self.filter_size = P
        self.filter_depth = Q

    def set_rho_adaptation(self, tau: float = 2.0, mu: float = 10.0):
        """Adaptive penalty of Eq. paramS at the residual checks (tau = 0: off); call before
        set_measurements."""
        self._check(self._L.cip_set_rho_adaptation(self._h, ctypes.c_double(tau), ctypes.c_double(mu)))

    @property
    def rho(self) -> float:
        v = ctypes.c_double()
        self._check(self._L.cip_get_rho(self._h, ctypes.byref(v)))
        return v.value

    def set_code_gradient_weight(self, mu: float):
        """Gradient (Tikhonov) penalty mu on the dictionary codes (cip_set_code_gradient_weight)."""
        self._check(self._L.cip_set_code_gradient_weight(self._h, ctypes.c_double(mu)))

    def set_dictionary_learning(self, sigma: float, stream=None):
        """Online dictionary update with filter-ADMM penalty sigma (cip_set_dictionary_learning);
        0 turns it off."""
        self._check(self._L.cip_set_dictionary_learning(self._h, ctypes.c_double(sigma), _stream_ptr(stream)))

    def set_sigma_adaptation(self, tau: float = 2.0, mu: float = 10.0):
        """Adaptation of the filter ADMM's sigma by the rule of Eq. paramS (cip_set_sigma_adaptation;
        tau = 0: off)."""
        self._check(self._L.cip_set_sigma_adaptation(self._h, ctypes.c_double(tau), ctypes.c_double(mu)))

    @property
    def sigma(self) -> float:
        v = ctypes.c_double()
        self._check(self._L.cip_get_sigma(self._h, ctypes.byref(v)))
        return v.value

    def get_dictionary(self, out=None, stream=None):
        """Learnt filters [L, P, P] (cip_get_dictionary)."""
        shape = (self.L, self.filter_size, self.filter_size)
        if out is None:
            torch = _torch()
            out = torch.empty(shape, device="cuda", dtype=torch.float32 if self.dtype == "f32" else torch.float64)
        p, keep = _ptr_and_check(out, self.dtype, shape)
        self._check(self._L.cip_get_dictionary(self._h, ctypes.c_void_p(p), _stream_ptr(stream)))
        return out

    def get_coefficients(self, out=None, stream=None):
        shape = (self.M, self.L, self.N, self.N)
        if out is None:
            torch = _torch()
            out = torch.empty(shape, device="cuda", dtype=torch.float32 if self.dtype == "f32" else torch.float64)
        p, keep = _ptr_and_check(out, self.dtype, shape)
        self._check(self._L.cip_get_coefficients(self._h, ctypes.c_void_p(p), _stream_ptr(stream)))
        return out

    def state_import_coefficients(self, z, t, u, stream=None):
        shape = (self.M, self.L, self.N, self.N)
        pz, k0 = _ptr_and_check(z, self.dtype, shape)
        pt, k1 = _ptr_and_check(t, self.dtype, shape)
        pu, k2 = _ptr_and_check(u, self.dtype, shape)
        self._check(self._L.cip_state_import_coefficients(self._h, ctypes.c_void_p(pz), ctypes.c_void_p(pt),
                                                          ctypes.c_void_p(pu), _stream_ptr(stream)))

    def close(self):
        if getattr(self, "_h", None):
            self._L.cip_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- ABI calls
    def set_prior(self, prior: str, lam: float, rho: float, beta: float = 1.0, stream=None):
        self._check(self._L.cip_set_prior(self._h, PRIORS[prior], lam, rho, beta, _stream_ptr(stream)))
        self.prior = prior

    def set_psfs(self, h, stream=None):
        p, keep = _ptr_and_check(h, self.dtype, (self.K, self.M, self.N, self.N))
        self._check(self._L.cip_set_psfs(self._h, ctypes.c_void_p(p), _stream_ptr(stream)))

    def set_measurements(self, y, stream=None):
        p, keep = _ptr_and_check(y, self.dtype, (self.K, self.N, self.N))
        self._check(self._L.cip_set_measurements(self._h, ctypes.c_void_p(p), _stream_ptr(stream)))

    def reset_state(self, stream=None):
        self._check(self._L.cip_reset_state(self._h, _stream_ptr(stream)))

    def iterate(self, n: int, tol: float = 0.0, stream=None) -> int:
        done = ctypes.c_int(0)
        self._check(self._L.cip_iterate(self._h, n, tol, ctypes.byref(done), _stream_ptr(stream)))
        return done.value

    def get_x(self, out=None, stream=None):
        if out is None:
            torch = _torch()
            out = torch.empty((self.M, self.N, self.N), device="cuda",
                              dtype=torch.float32 if self.dtype == "f32" else torch.float64)
        p, keep = _ptr_and_check(out, self.dtype, (self.M, self.N, self.N))
        self._check(self._L.cip_get_x(self._h, ctypes.c_void_p(p), _stream_ptr(stream)))
        return out

    def get_u(self, out=None, stream=None):
        shape = self.state_shape
        if out is None:
            torch = _torch()
            out = torch.empty(shape, device="cuda", dtype=torch.float32 if self.dtype == "f32" else torch.float64)
        p, keep = _ptr_and_check(out, self.dtype, shape)
        self._check(self._L.cip_get_u(self._h, ctypes.c_void_p(p), _stream_ptr(stream)))
        return out

    def residuals(self) -> Tuple[float, float]:
        r, s = ctypes.c_double(), ctypes.c_double()
        self._check(self._L.cip_get_residuals(self._h, ctypes.byref(r), ctypes.byref(s)))
        return r.value, s.value

    def iteration(self) -> int:
        v = ctypes.c_int()
        self._check(self._L.cip_get_iteration(self._h, ctypes.byref(v)))
        return v.value

    def state_import(self, t, u, stream=None):
        shape = self.state_shape
        pt, k1 = _ptr_and_check(t, self.dtype, shape)
        pu, k2 = _ptr_and_check(u, self.dtype, shape)
        self._check(self._L.cip_state_import(self._h, ctypes.c_void_p(pt), ctypes.c_void_p(pu), _stream_ptr(stream)))

    def state_size(self) -> int:
        n = ctypes.c_size_t()
        self._check(self._L.cip_state_size(self._h, ctypes.byref(n)))
        return n.value

    def state_export(self, buf=None, stream=None):
        n = self.state_size()
        if buf is None:
            buf = np.empty(n, dtype=np.uint8)
        ptr = buf.ctypes.data if isinstance(buf, np.ndarray) else buf.data_ptr()
        self._check(self._L.cip_state_export(self._h, ctypes.c_void_p(ptr), _stream_ptr(stream)))
        return buf

    def state_restore(self, buf, stream=None):
        ptr = buf.ctypes.data if isinstance(buf, np.ndarray) else buf.data_ptr()
        self._check(self._L.cip_state_restore(self._h, ctypes.c_void_p(ptr), _stream_ptr(stream)))

    def set_timing(self, on: bool):
        self._check(self._L.cip_set_timing(self._h, 1 if on else 0))

    def set_test_fault(self, kind: int):
        """Test-only fault switch (cip_set_test_fault): 1 = the prior pass's staged-copy wait can
        never complete and gives up after a few polls; 0 = off."""
        self._check(self._L.cip_set_test_fault(self._h, int(kind)))

    def get_timing(self):
        a, b = ctypes.c_double(), ctypes.c_double()
        na, nb = ctypes.c_int(), ctypes.c_int()
        self._check(self._L.cip_get_timing(self._h, ctypes.byref(a), ctypes.byref(na), ctypes.byref(b), ctypes.byref(nb)))
        return {"prior_pass_ms": a.value, "prior_pass_n": na.value, "column_pass_ms": b.value, "column_pass_n": nb.value}

    def launches(self) -> int:
        v = ctypes.c_ulonglong()
        self._check(self._L.cip_get_launches(self._h, ctypes.byref(v)))
        return int(v.value)

    def config(self):
        v = [ctypes.c_int() for _ in range(5)]
        self._check(self._L.cip_get_config(self._h, *[ctypes.byref(x) for x in v]))
        e = ctypes.c_int()
        self._check(self._L.cip_get_prior_fft(self._h, ctypes.byref(e)))
        return {"rows_per_tile": v[0].value, "col_tile": v[1].value, "prior_pass_blocks": v[2].value,
                "column_pass_blocks": v[3].value, "column_pass": {1: "fused", 2: "split"}.get(v[4].value, "?"),
                "prior_fft_elems": e.value}


class Batch:
    """cip_batch: iterate many plans together through one CUDA graph (one branch per plan)."""

    def __init__(self, plans, nstreams: int = 0):
        self._L = _lib.load()
        self.plans = list(plans)  # keeps the plans alive while the batch exists
        arr = (ctypes.c_void_p * len(self.plans))(*[p._h.value for p in self.plans])
        h = ctypes.c_void_p()
        st = self._L.cip_batch_create(ctypes.byref(h), arr, len(self.plans), nstreams)
        if st != 0:
            raise CipError(st, "cip_batch_create failed")
        self._h = h

    def iterate(self, n: int, stream=None):
        st = self._L.cip_batch_iterate(self._h, n, _stream_ptr(stream))
        if st != 0:
            raise CipError(st, self._L.cip_batch_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._L.cip_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


RESULT_STATES = {0: "queued", 1: "running", 2: "done", 3: "failed", 4: "cancelled"}


class Server:
    """cip_server: continuous batching of reconstructions with admission by device-memory budget."""

    def __init__(self, hbm_budget: int, max_active: int = 16, check_every: int = 10):
        self._L = _lib.load()
        h = ctypes.c_void_p()
        st = self._L.cip_server_create(ctypes.byref(h), int(hbm_budget), max_active, check_every)
        if st != 0:
            raise CipError(st, "cip_server_create failed")
        self._h = h
        self._keep = {}

    def submit(self, h, y, prior: str, lam: float, rho: float, beta: float = 1.0, tol: float = 0.0,
               max_iter: int = 300, psf_key: int = 0, rho_tau: float = 0.0, rho_mu: float = 0.0):
        """Queue one reconstruction (float32 host arrays h [K][M][N][N], y [K][N][N]); returns (id, x_out).
        rho_tau > 1, rho_mu > 1: adaptive penalty of Eq. paramS at every check."""
        h = np.ascontiguousarray(h, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.float32)
        K, M, N = h.shape[0], h.shape[1], h.shape[-1]
        x_out = np.zeros((M, N, N), dtype=np.float32)
        req = _lib.cip_request(N, K, M, PRIORS[prior], lam, rho, beta, h.ctypes.data, y.ctypes.data,
                               x_out.ctypes.data, tol, max_iter, psf_key, rho_tau, rho_mu)
        rid = ctypes.c_ulonglong()
        st = self._L.cip_server_submit(self._h, ctypes.byref(req), ctypes.byref(rid))
        if st != 0:
            raise CipError(st, "cip_server_submit failed")
        self._keep[rid.value] = x_out
        return rid.value, x_out

    @staticmethod
    def _res(r):
        return {"state": RESULT_STATES.get(r.state, "?"), "status": r.status, "iterations": r.iterations,
                "r_rel": r.r_rel, "s_rel": r.s_rel, "t_submit": r.t_submit, "t_admit": r.t_admit, "t_done": r.t_done}

    def poll(self, rid: int):
        r = _lib.cip_result()
        st = self._L.cip_server_poll(self._h, rid, ctypes.byref(r))
        if st != 0:
            raise CipError(st, "cip_server_poll failed")
        return self._res(r)

    def wait(self, rid: int, timeout: float = 600.0):
        r = _lib.cip_result()
        st = self._L.cip_server_wait(self._h, rid, ctypes.byref(r), timeout)
        if st not in (0, 6):
            raise CipError(st, "cip_server_wait failed")
        return self._res(r)

    def cancel(self, rid: int):
        self._L.cip_server_cancel(self._h, rid)

    def stats(self):
        v, run, q, b, hit, miss = (ctypes.c_double(), ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t(), ctypes.c_int(),
                                   ctypes.c_int())
        self._L.cip_server_stats(self._h, *[ctypes.byref(x) for x in (v, run, q, b, hit, miss)])
        return {"voxel_iters": v.value, "running": run.value, "queued": q.value, "bytes_in_use": b.value,
                "cache_hits": hit.value, "cache_misses": miss.value}

    def close(self):
        if getattr(self, "_h", None):
            self._L.cip_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def shrink_dual_noalloc(prior: str, lam: float, rho: float, x, u_in, t_prev, u_out, resid_out, t_out=None,
                        stream=None):
    """cip_shrink_dual_noalloc: t/u update and relative residuals from device tensors the caller owns,
    with no device allocation by the library (for callers that cannot allocate, e.g. inside a
    stream capture or a fixed memory arena).  resid_out: 2 float64 (device tensor or numpy array)."""
    M, N = int(x.shape[0]), int(x.shape[-1])
    dtype = "f32" if str(x.dtype).endswith("float32") else "f64"
    ncomp = 2 if prior == "tv" else 1
    px, k0 = _ptr_and_check(x, dtype, (M, N, N))
    pu, k1 = _ptr_and_check(u_in, dtype, (M, ncomp, N, N))
    pt, k2 = _ptr_and_check(t_prev, dtype, (M, ncomp, N, N))
    po, k3 = _ptr_and_check(u_out, dtype, (M, ncomp, N, N))
    ptout = _ptr_and_check(t_out, dtype, (M, ncomp, N, N))[0] if t_out is not None else None
    pr = resid_out.ctypes.data if isinstance(resid_out, np.ndarray) else resid_out.data_ptr()
    L = _lib.load()
    st = L.cip_shrink_dual_noalloc(DTYPES[dtype], PRIORS[prior], N, M, lam, rho, ctypes.c_void_p(px),
                                   ctypes.c_void_p(pu), ctypes.c_void_p(pt), ctypes.c_void_p(po),
                                   ctypes.c_void_p(ptout), ctypes.c_void_p(pr), _stream_ptr(stream))
    if st != 0:
        raise CipError(st, L.cip_status_string(st).decode())


def reconstruct(problem, dtype: Optional[str] = None, iters: Optional[int] = None, tol: float = 0.0, stream=None):
    """Convenience: full reconstruction of an ``inputs.Problem`` with device-resident inputs."""
    torch = _torch()
    dt = dtype or problem.dtype
    tdt = torch.float32 if dt == "f32" else torch.float64
    P = Plan(problem.N, problem.K, problem.M, dt)
    P.set_prior(problem.prior, problem.lam, problem.rho, problem.beta, stream)
    P.set_psfs(torch.as_tensor(problem.h, dtype=tdt).cuda().contiguous(), stream)
    P.set_measurements(torch.as_tensor(problem.y, dtype=tdt).cuda().contiguous(), stream)
    n = P.iterate(iters if iters is not None else problem.iters, tol, stream)
    return P, P.get_x(stream=stream), n

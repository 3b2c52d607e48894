"""FP64 CPU oracle, fast form: the same steps as ``oracle.admm`` (Alg. 1 and
Alg. 2 of Dogan & Oktem, arXiv 2006.08303), with the naive DFT replaced by
scipy.fft's real FFT (pocketfft, all host cores) and the spatial convolution
never formed.  Used for image sizes the naive oracle cannot reach and as the
timed CPU baseline.  It is cross-checked against ``oracle.admm`` in the CPU
tests.

TEST INFRASTRUCTURE ONLY: imported by tests, the smoke check and the
benchmark's CPU-baseline leg, never by the library.  It shares no code with
the CUDA path and only reuses the operator definitions of ``oracle.admm``.
"""
from __future__ import annotations

import os
from dataclasses import dataclass

import numpy as np
import scipy.fft as sfft

from . import admm as ref

WORKERS = os.cpu_count() or 1


def rfft2(x):
    return sfft.rfft2(x, workers=WORKERS)


def irfft2(X, N):
    return sfft.irfft2(X, s=(N, N), workers=WORKERS)


def gram_eigenvalues_half(prior: str, N: int) -> np.ndarray:
    """g(w) on the half spectrum [N, N/2+1] (DFT of the kernel T^T T delta)."""
    if prior in ("dct8", "l1", "wdct"):
        return np.ones((N, N // 2 + 1))
    fwd, adj = ref.PRIORS[prior]
    delta = np.zeros((N, N))
    delta[0, 0] = 1.0
    return rfft2(adj(fwd(delta))).real


@dataclass
class FastAnalysis:
    N: int
    M: int
    prior: str
    lam: float
    rho: float
    beta: float
    Pinv: np.ndarray   # [N, N/2+1, M, M]
    bhat: np.ndarray   # [N, N/2+1, M]


def analysis_setup(h, y, prior, lam, rho, beta) -> FastAnalysis:
    """Alg. 1 setup on the half spectrum (same readings as oracle.admm)."""
    K, M, N, _ = h.shape
    Lam = np.moveaxis(rfft2(h), (0, 1), (2, 3))                 # [N, H, K, M]
    g = gram_eigenvalues_half(prior, N)
    Psi = rho * g[..., None, None] * np.eye(M) + beta * np.einsum("abki,abkj->abij", Lam.conj(), Lam)
    sing = g <= 1e-12 * g.max()
    Pinv = np.linalg.inv(np.where(sing[..., None, None], np.eye(M), Psi))
    for a, b in np.argwhere(sing):
        Pinv[a, b] = ref.pinv_hermitian(Psi[a, b])
    Y = np.moveaxis(rfft2(y), 0, 2)                             # [N, H, K]
    bhat = beta * np.einsum("abkm,abk->abm", Lam.conj(), Y)
    return FastAnalysis(N, M, prior, lam, rho, beta, Pinv, bhat)


def x_update(S: FastAnalysis, t, u):
    """Eq. solx_Trans_DFT on the half spectrum."""
    _, adj = ref.PRIORS[S.prior]
    Q = np.moveaxis(rfft2(adj(t - u)), 0, 2)                    # [N, H, M]
    X = np.matmul(S.Pinv, (S.bhat + S.rho * Q)[..., None])[..., 0]
    return irfft2(np.moveaxis(X, 2, 0), S.N)


def analysis_step(S: FastAnalysis, t, u):
    fwd, _ = ref.PRIORS[S.prior]
    x = x_update(S, t, u)
    w = fwd(x)
    t_new = ref.shrink(S.prior, w + u, S.lam / S.rho)
    return x, t_new, u + w - t_new, w


def run_analysis_adaptive(h, y, prior, lam, rho, beta, iters: int, check_every: int, tau: float = 2.0,
                          mu: float = 10.0, tol: float = 0.0):
    """Same schedule as oracle.admm.run_analysis_adaptive (Eq. paramS after every check_every-th
    iteration, u rescaled, factor formed again); with tol > 0 it also stops at the first check at
    which both relative residuals are below tol.  Returns (x, t, u, rhos, iterations_done)."""
    S = analysis_setup(h, y, prior, lam, rho, beta)
    ncomp = ref.ncomp_of(prior)
    t = np.zeros((S.M, ncomp, S.N, S.N))
    u = np.zeros_like(t)
    rhos = []
    x = None
    done = 0
    for it in range(iters):
        x, t_new, u_new, w = analysis_step(S, t, u)
        done = it + 1
        stop = False
        if (it + 1) % check_every == 0:
            r = float(np.linalg.norm(w - t_new))
            s = S.rho * float(np.linalg.norm(t_new - t))
            if tol > 0:
                r_rel = r / max(np.linalg.norm(w), np.linalg.norm(t_new), 1e-300)
                s_rel = s / max(S.rho * np.linalg.norm(u_new), 1e-300)
                stop = r_rel < tol and s_rel < tol
            rho_new = ref.adapt_rho(S.rho, r, s, tau, mu)
            if not stop and rho_new != S.rho:
                u_new = u_new * (S.rho / rho_new)
                S = analysis_setup(h, y, prior, lam, rho_new, beta)
        t, u = t_new, u_new
        rhos.append(S.rho)
        if stop:
            break
    return x, t, u, rhos, done


def run_analysis(S: FastAnalysis, iters: int, t0=None, u0=None, tol: float = 0.0):
    """Alg. 1; with tol > 0 stops when both relative residuals (reading R11) fall below tol.
    Returns (x, t, u, iterations_done, (r_rel, s_rel))."""
    ncomp = ref.ncomp_of(S.prior)
    t = np.zeros((S.M, ncomp, S.N, S.N)) if t0 is None else t0.copy()
    u = np.zeros_like(t) if u0 is None else u0.copy()
    x = None
    rr = (np.inf, np.inf)
    done = 0
    for it in range(iters):
        x, t_new, u_new, w = analysis_step(S, t, u)
        done = it + 1
        if tol > 0:
            r = np.linalg.norm(w - t_new)
            s = S.rho * np.linalg.norm(t_new - t)
            rr = (r / max(np.linalg.norm(w), np.linalg.norm(t_new), 1e-300),
                  s / max(S.rho * np.linalg.norm(u_new), 1e-300))
        t, u = t_new, u_new
        if tol > 0 and rr[0] < tol and rr[1] < tol:
            break
    return x, t, u, done, rr


@dataclass
class FastConvDict:
    N: int
    M: int
    L: int
    lam: float
    rho: float
    beta: float
    Pinv: np.ndarray   # [N, H, M, M]
    bhat: np.ndarray   # [N, H, M]
    theta: np.ndarray  # [N, H, L]
    rho_n: np.ndarray = None  # [N, H] rho + mu g(w) (gradient penalty on the codes)


def convdict_setup(h, y, d, lam, rho, beta, mu: float = 0.0) -> FastConvDict:
    K, M, N, _ = h.shape
    Lam = np.moveaxis(rfft2(h), (0, 1), (2, 3))
    Psi = np.eye(M) + beta * np.einsum("abki,abkj->abij", Lam.conj(), Lam)
    Pinv = np.linalg.inv(Psi)
    Y = np.moveaxis(rfft2(y), 0, 2)
    bhat = beta * np.einsum("abkm,abk->abm", Lam.conj(), Y)
    theta = np.moveaxis(rfft2(ref.embed_filters(d, N)), 0, 2)
    rho_n = rho + mu * ref.gram_eigenvalues("tv", N)[:, : N // 2 + 1]
    return FastConvDict(N, M, d.shape[0], lam, rho, beta, Pinv, bhat, theta, rho_n)


def convdict_step(C: FastConvDict, z, t, u):
    """Alg. 2 iteration (same order as oracle.admm.convdict_step), z/t/u [L, M, N, N]."""
    Z = np.moveaxis(rfft2(z), (0, 1), (2, 3))                   # [N, H, L, M]
    p = np.einsum("abl,ablm->abm", C.theta, Z)
    X = np.matmul(C.Pinv, (C.bhat + p)[..., None])[..., 0]     # [N, H, M]
    x = irfft2(np.moveaxis(X, 2, 0), C.N)
    G = np.moveaxis(rfft2(t - u), (0, 1), (2, 3))               # [N, H, L, M]
    c = C.theta.conj()[..., None] * X[:, :, None, :] + C.rho * G
    th = C.theta[..., None]
    dot = np.sum(th * c, axis=2, keepdims=True)                 # theta^T c
    nrm = np.sum(np.abs(C.theta) ** 2, axis=2)[..., None, None]
    rn = C.rho_n[..., None, None]
    v = (c - th.conj() * dot / (rn + nrm)) / rn
    z_new = irfft2(np.moveaxis(v, (2, 3), (0, 1)), C.N)
    t_new = ref.soft(z_new + u, C.lam / C.rho)
    return x, z_new, t_new, u + z_new - t_new


def run_convdict_adaptive(h, y, d, lam, rho, beta, iters: int, check_every: int, tau: float = 2.0,
                          mu_bal: float = 10.0, mu: float = 0.0):
    """Alg. 2 from zero state with the penalty of Eq. paramS adapted after every check_every-th
    iteration (r = ||z - t||, s = rho ||t - t_prev||; readings R17, R18: u rescaled by
    rho/rho').  The x-update factor (I + beta Lambda^H Lambda) does not depend on rho; the z-update
    diagonal and the shrinkage threshold follow the current rho.  Returns (x, z, t, u, rhos)."""
    C = convdict_setup(h, y, d, lam, rho, beta, mu)
    z = np.zeros((C.L, C.M, C.N, C.N))
    t = np.zeros_like(z)
    u = np.zeros_like(z)
    rhos = []
    x = None
    for it in range(iters):
        x, z_new, t_new, u_new = convdict_step(C, z, t, u)
        if (it + 1) % check_every == 0:
            r = float(np.linalg.norm(z_new - t_new))
            s = C.rho * float(np.linalg.norm(t_new - t))
            rho_new = ref.adapt_rho(C.rho, r, s, tau, mu_bal)
            if rho_new != C.rho:
                u_new = u_new * (C.rho / rho_new)
                C = convdict_setup(h, y, d, lam, rho_new, beta, mu)
        z, t, u = z_new, t_new, u_new
        rhos.append(C.rho)
    return x, z, t, u, rhos


def dict_update(x, z, g, e, sigma: float, P: int):
    """Same filter-ADMM step as oracle.admm.dict_update on the half spectrum (batched solves)."""
    N = x.shape[-1]
    Zh = np.moveaxis(rfft2(z), (0, 1), (2, 3))                  # [N, H, L, S]
    Xh = np.moveaxis(rfft2(x), 0, 2)                            # [N, H, S]
    GE = np.moveaxis(rfft2(g - e), 0, 2)                        # [N, H, L]
    L = Zh.shape[2]
    A = sigma * np.eye(L) + np.einsum("abls,abks->ablk", Zh.conj(), Zh)
    rhs = np.einsum("abls,abs->abl", Zh.conj(), Xh) + sigma * GE
    dh = np.linalg.solve(A, rhs[..., None])[..., 0]
    d = irfft2(np.moveaxis(dh, 2, 0), N)
    g_new = ref.project_filters(d + e, P)
    return d, g_new, e + d - g_new


def run_convdict_learn(h, y, d0, lam, rho, beta, sigma: float, iters: int, check_every: int = 0,
                       tau: float = 2.0, mu: float = 10.0):
    """Same schedule as oracle.admm.run_convdict_learn (with the same optional adaptation of sigma).
    Returns (x, z, t, u, filters [L, P, P]) plus the sigmas when adapting."""
    P = d0.shape[-1]
    C = convdict_setup(h, y, d0, lam, rho, beta)
    N = C.N
    g = ref.embed_filters(d0, N)
    e = np.zeros_like(g)
    z = np.zeros((C.L, C.M, N, N))
    t = np.zeros_like(z)
    u = np.zeros_like(z)
    x = None
    sigmas = []
    for it in range(iters):
        C.theta = np.moveaxis(rfft2(g), 0, 2)
        x, z, t, u = convdict_step(C, z, t, u)
        g_prev = g
        d, g, e = dict_update(x, z, g, e, sigma, P)
        if check_every > 0 and (it + 1) % check_every == 0:
            r = float(np.linalg.norm(d - g))
            s_ = sigma * float(np.linalg.norm(g - g_prev))
            sigma_new = ref.adapt_rho(sigma, r, s_, tau, mu)
            if sigma_new != sigma:
                e = e * (sigma / sigma_new)
                sigma = sigma_new
        sigmas.append(sigma)
    if check_every > 0:
        return x, z, t, u, ref.crop_filters(g, P), sigmas
    return x, z, t, u, ref.crop_filters(g, P)


@dataclass
class FastConvDict3D:
    N: int
    M: int
    L: int
    lam: float
    rho: float
    beta: float
    Pinv: np.ndarray    # [N, H, M, M]
    bhat: np.ndarray    # [N, H, M]
    theta3: np.ndarray  # [L, S(kappa), N, H]


def convdict3d_setup(h, y, d3, lam, rho, beta) -> FastConvDict3D:
    """Same setup as oracle.admm.convdict3d_setup on the half spectrum (3D DFT = rfft2 of every
    slice, then the full FFT along the channel axis)."""
    K, M, N, _ = h.shape
    Lam = np.moveaxis(rfft2(h), (0, 1), (2, 3))
    Pinv = np.linalg.inv(np.eye(M) + beta * np.einsum("abki,abkj->abij", Lam.conj(), Lam))
    Y = np.moveaxis(rfft2(y), 0, 2)
    bhat = beta * np.einsum("abkm,abk->abm", Lam.conj(), Y)
    theta3 = sfft.fft(rfft2(ref.embed_filters3d(d3, N, M)), axis=1)
    return FastConvDict3D(N, M, d3.shape[0], lam, rho, beta, Pinv, bhat, theta3)


def convdict3d_step(C: FastConvDict3D, z, t, u):
    """Same steps as oracle.admm.convdict3d_step, z/t/u [L, S, N, N]."""
    Zh = sfft.fft(rfft2(z), axis=1)                              # [L, S, N, H]
    q = np.einsum("lkab,lkab->kab", C.theta3, Zh)
    p = np.moveaxis(sfft.ifft(q, axis=0), 0, 2)                   # [N, H, S]
    X = np.matmul(C.Pinv, (C.bhat + p)[..., None])[..., 0]       # [N, H, S]
    x = irfft2(np.moveaxis(X, 2, 0), C.N)
    X3 = sfft.fft(np.moveaxis(X, 2, 0), axis=0)                  # [S, N, H]
    c = C.theta3.conj() * X3[None] + C.rho * sfft.fft(rfft2(t - u), axis=1)
    dot = np.sum(C.theta3 * c, axis=0, keepdims=True)
    nrm = np.sum(np.abs(C.theta3) ** 2, axis=0, keepdims=True)
    v = (c - C.theta3.conj() * dot / (C.rho + nrm)) / C.rho
    z_new = irfft2(sfft.ifft(v, axis=1), C.N)
    t_new = ref.soft(z_new + u, C.lam / C.rho)
    return x, z_new, t_new, u + z_new - t_new


def run_convdict3d(C: FastConvDict3D, iters: int):
    z = np.zeros((C.L, C.M, C.N, C.N))
    t = np.zeros_like(z)
    u = np.zeros_like(z)
    x = None
    for _ in range(iters):
        x, z, t, u = convdict3d_step(C, z, t, u)
    return x, z, t, u


def run_convdict(C: FastConvDict, iters: int):
    z = np.zeros((C.L, C.M, C.N, C.N))
    t = np.zeros_like(z)
    u = np.zeros_like(z)
    x = None
    for _ in range(iters):
        x, z, t, u = convdict_step(C, z, t, u)
    return x, z, t, u

"""Plain FP64 CPU oracle for the ADMM reconstruction of Dogan & Oktem,
"Efficient Algorithms for Convolutional Inverse Problems in Multidimensional
Imaging" (arXiv 2006.08303).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this module.  It shares no code with the CUDA
library (no kernels, tables, constants or helpers); it uses NumPy alone.

Everything is float64 / complex128 and written for readability, not speed:
  * the 2D DFT is the explicit separable DFT matrix product (entries
    exp(-2 pi i ((j k) mod N) / N)), unnormalised forward, 1/N^2 inverse;
  * the forward operator H is a spatial circular convolution;
  * per-frequency matrices are formed and inverted with numpy.linalg.

Notation follows the paper: K measurements, S (here M) unknown channels,
N x N images, Lambda = DFT of the PSFs (Section IV-A, "Image update"),
Psi = rho g(w) I + beta Lambda^H Lambda, t auxiliary, u scaled dual.

Readings where the paper is silent or garbled (each listed in the design notes):
  R1 anisotropic TV: T = [D_h; D_v] circular forward differences; the
     x-update uses the general closed form with T^H T (Eq. solx_Trans) whose
     DFT eigenvalues g(w) come from the circulant kernel of D^T D.
  R2 at bins where g(w) = 0 (the DC bin of TV) Psi is singular when all PSFs
     have unit sum; the oracle takes the min-norm pseudo-inverse (eigenvalues
     below 1e-10 * max eigenvalue dropped), which is what a least-squares
     solve of the dense system returns.
  R3 Psi_{i,j} = rho delta_{ij} I + beta sum_k Lambda_{k,i}^H Lambda_{k,j}
     (the printed block formula drops rho and swaps indices).
  R4 Lambda is the unnormalised DFT of h, so H_{k,s} = F^H diag(Lambda) F.
  R5 t^0 = u^0 = 0 (and z^0 = 0 for the synthesis prior).
  R9 synthesis objective uses 1/2 ||D z - x||^2 and rho/2 ||z - t + u||^2.
  R10 Sherman-Morrison per bin with theta~_n = conj(theta_n):
      v = (c - conj(theta) (theta^T c) / (rho + ||theta||^2)) / rho.
  R11 residuals as in Eq. paramS: r = ||Tx - t||, s = rho ||t - t_prev||;
      relative forms r / max(||Tx||, ||t||) and s / ||rho u||.
"""
from __future__ import annotations

import functools
import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


# ---------------------------------------------------------------------------
# DFT (Section IV-A: F_2D diagonalises each BCCB block H_{k,s})
# ---------------------------------------------------------------------------
def dft_matrix(N: int, sign: int = -1) -> np.ndarray:
    """Explicit N x N DFT matrix, entry (j,k) = exp(sign 2 pi i ((j k) mod N) / N)."""
    jk = np.outer(np.arange(N), np.arange(N)) % N
    ang = 2.0 * math.pi * jk / N
    return np.cos(ang) + 1j * sign * np.sin(ang)


def dft2(x: np.ndarray) -> np.ndarray:
    """Unnormalised 2D DFT over the last two axes, X = F x F^T (F symmetric)."""
    N = x.shape[-1]
    assert x.shape[-2] == N
    F = dft_matrix(N, -1)
    return F @ x @ F


def idft2(X: np.ndarray) -> np.ndarray:
    """Inverse of dft2 (1/N^2 normalisation); returns complex."""
    N = X.shape[-1]
    G = dft_matrix(N, +1)
    return (G @ X @ G) / (N * N)


# ---------------------------------------------------------------------------
# Forward model, Section II (Eq. forward model): y_k = sum_s x_s (*) h_{k,s}
# ---------------------------------------------------------------------------
def circconv2(x: np.ndarray, h: np.ndarray) -> np.ndarray:
    """Spatial circular convolution y[n] = sum_j x[j] h[(n - j) mod N] over the
    last two axes (x and h broadcast over leading axes)."""
    N = x.shape[-1]
    y = np.zeros(np.broadcast_shapes(x.shape, h.shape), dtype=np.result_type(x, h))
    for a in range(N):
        for b in range(N):
            y = y + h[..., a:a + 1, b:b + 1] * np.roll(x, shift=(a, b), axis=(-2, -1))
    return y


def circcorr2(y: np.ndarray, h: np.ndarray) -> np.ndarray:
    """Adjoint of circconv2 in x: x[j] = sum_n y[n] h[(n - j) mod N]."""
    N = y.shape[-1]
    x = np.zeros(np.broadcast_shapes(y.shape, h.shape), dtype=np.result_type(y, h))
    for a in range(N):
        for b in range(N):
            x = x + h[..., a:a + 1, b:b + 1] * np.roll(y, shift=(-a, -b), axis=(-2, -1))
    return x


def forward_H(x: np.ndarray, h: np.ndarray) -> np.ndarray:
    """Stacked forward operator (Eq. forwardModel): x [M,N,N] -> y [K,N,N]."""
    K, M = h.shape[:2]
    return np.stack([sum(circconv2(x[m], h[k, m]) for m in range(M)) for k in range(K)])


def adjoint_H(y: np.ndarray, h: np.ndarray) -> np.ndarray:
    """H^T y: [K,N,N] -> [M,N,N]."""
    K, M = h.shape[:2]
    return np.stack([sum(circcorr2(y[k], h[k, m]) for k in range(K)) for m in range(M)])


# ---------------------------------------------------------------------------
# Analysis operators T (Eq. analysis) and their adjoints
# ---------------------------------------------------------------------------
def tv_forward(x: np.ndarray) -> np.ndarray:
    """Anisotropic TV (reading R1): [..., N, N] -> [..., 2, N, N];
    component 0 = x[r, c+1] - x[r, c], component 1 = x[r+1, c] - x[r, c] (circular)."""
    dh = np.roll(x, -1, axis=-1) - x
    dv = np.roll(x, -1, axis=-2) - x
    return np.stack([dh, dv], axis=-3)


def tv_adjoint(w: np.ndarray) -> np.ndarray:
    """D^T: [..., 2, N, N] -> [..., N, N]; D_h^T a = a[r, c-1] - a[r, c], likewise along rows."""
    ah, av = w[..., 0, :, :], w[..., 1, :, :]
    return (np.roll(ah, 1, axis=-1) - ah) + (np.roll(av, 1, axis=-2) - av)


def dct8_matrix() -> np.ndarray:
    """Orthonormal 8-point DCT-II, C[k, n] = a_k cos(pi (2n+1) k / 16),
    a_0 = sqrt(1/8), a_k = sqrt(2/8)."""
    k = np.arange(8)[:, None]
    n = np.arange(8)[None, :]
    C = np.cos(math.pi * (2 * n + 1) * k / 16.0)
    C[0, :] *= math.sqrt(1.0 / 8.0)
    C[1:, :] *= math.sqrt(2.0 / 8.0)
    return C


def _blocks(x: np.ndarray) -> np.ndarray:
    N = x.shape[-1]
    lead = x.shape[:-2]
    return x.reshape(*lead, N // 8, 8, N // 8, 8)


def _unblocks(b: np.ndarray) -> np.ndarray:
    lead = b.shape[:-4]
    N = b.shape[-4] * 8
    return b.reshape(*lead, N, N)


def dct8_forward(x: np.ndarray) -> np.ndarray:
    """Blockwise orthonormal 8x8 DCT-II, blocks aligned at (0,0): [..., N, N] -> [..., 1, N, N]."""
    C = dct8_matrix()
    b = _blocks(x)
    w = np.einsum("ka,...iajb,lb->...ikjl", C, b, C)
    return _unblocks(w)[..., None, :, :]


def dct8_adjoint(w: np.ndarray) -> np.ndarray:
    """Inverse (= adjoint) of dct8_forward: [..., 1, N, N] -> [..., N, N]."""
    C = dct8_matrix()
    b = _blocks(w[..., 0, :, :])
    x = np.einsum("ka,...ikjl,lb->...iajb", C, b, C)
    return _unblocks(x)


def l1_forward(x: np.ndarray) -> np.ndarray:
    """T = I (plain l1 prior)."""
    return x[..., None, :, :].copy()


def l1_adjoint(w: np.ndarray) -> np.ndarray:
    return w[..., 0, :, :].copy()


# ---------------------------------------------------------------------------
# Kronecker prior T = (2D Symmlet-8 wavelet) (x) (1D DCT along the channels) (Section V,
# the analysis prior of the spectral experiments; readings R24-R26)
# ---------------------------------------------------------------------------
def symlet_lowpass(p: int) -> np.ndarray:
    """Orthonormal lowpass filter (2p taps, sum sqrt(2)) with p vanishing moments and the most
    nearly linear phase (Daubechies' least-asymmetric construction, reading R24):
      |m0(w)|^2 = cos^{2p}(w/2) P(sin^2(w/2)),  P(y) = sum_{k<p} C(p-1+k, k) y^k,
    each root y of P gives the root pair z, 1/z of z^2 - 2(1 - 2y) z + 1; one of each pair (one
    conjugate pair of pairs for complex y) is kept, every choice is formed, and the one whose
    remaining factor Q(e^{iw}) has the smallest least-squares deviation of its unwrapped phase
    from a straight line on [0, pi] wins; of the two mirror-image winners the one with the
    smaller energy centroid sum_n n h_n^2 is returned."""
    coeffs = [math.comb(p - 1 + k, k) for k in range(p)]
    ys = list(np.roots(coeffs[::-1])) if p > 1 else []
    groups = []                       # each: the inside-circle z roots of one real y / conjugate pair
    taken = [False] * len(ys)
    for i, y in enumerate(ys):
        if taken[i]:
            continue
        taken[i] = True
        w = 1.0 - 2.0 * y
        z = w + np.sqrt(w * w - 1.0 + 0j)
        z_in = z if abs(z) < 1.0 else 1.0 / z
        if abs(y.imag) <= 1e-9 * max(1.0, abs(y)):
            groups.append([complex(z_in.real, 0.0)])
        else:
            j = min((k for k in range(len(ys)) if not taken[k]), key=lambda k: abs(ys[k] - np.conj(y)))
            taken[j] = True
            groups.append([z_in, np.conj(z_in)])
    omega = math.pi * np.arange(513) / 512.0
    best = None
    for pick in range(1 << len(groups)):
        roots = []
        for b, g in enumerate(groups):
            roots += g if not (pick >> b) & 1 else [1.0 / z for z in g]
        q = np.array([1.0 + 0j])
        for r in roots:
            q = np.convolve(q, [1.0, -r])
        h = q
        for _ in range(p):
            h = np.convolve(h, [1.0, 1.0])
        h = h.real * (math.sqrt(2.0) / h.real.sum())
        Q = np.ones(omega.shape, dtype=complex)
        for r in roots:
            Q *= 1.0 - r * np.exp(-1j * omega)
        phase = np.unwrap(np.angle(Q))
        A = np.stack([np.ones_like(omega), omega], axis=1)
        fit = A @ np.linalg.lstsq(A, phase, rcond=None)[0]
        dev = float(np.sum((phase - fit) ** 2))
        centroid = float(np.sum(np.arange(h.size) * h * h))
        key = (round(dev, 6), centroid)
        if best is None or key < best[0]:
            best = (key, h)
    return best[1]


@functools.lru_cache(maxsize=None)
def _sym8_cached() -> tuple:
    return tuple(symlet_lowpass(8))


def _sym8() -> np.ndarray:
    return np.array(_sym8_cached())


def wavelet_levels(N: int) -> int:
    """Decomposition depth: down to a 16 x 16 coarse band (reading R25)."""
    return int(round(math.log2(N))) - 4


def dwt_matrix(n: int, h: np.ndarray) -> np.ndarray:
    """One level of the periodic orthonormal DWT on length n: rows i < n/2 are the lowpass
    taps h[(j - 2i) mod n], rows n/2 + i the highpass taps g[k] = (-1)^k h[L-1-k]."""
    L = h.size
    g = np.array([(-1) ** k * h[L - 1 - k] for k in range(L)])
    A = np.zeros((n, n))
    for i in range(n // 2):
        for k in range(L):
            A[i, (2 * i + k) % n] += h[k]
            A[n // 2 + i, (2 * i + k) % n] += g[k]
    return A


def dct_matrix(n: int) -> np.ndarray:
    """Orthonormal DCT-II, C[k, m] = a_k cos(pi (2m+1) k / (2n)), a_0 = sqrt(1/n), a_k = sqrt(2/n)."""
    k = np.arange(n)[:, None]
    m = np.arange(n)[None, :]
    C = np.cos(math.pi * (2 * m + 1) * k / (2.0 * n))
    C[0, :] *= math.sqrt(1.0 / n)
    C[1:, :] *= math.sqrt(2.0 / n)
    return C


def wdct_forward(x: np.ndarray) -> np.ndarray:
    """T x for T = W (x) C: the J-level periodic 2D Symmlet-8 transform of every channel (Mallat
    layout: level by level rows then columns of the current coarse band), then the DCT-II along
    the channel axis.  x [M, N, N] -> [M, 1, N, N]."""
    M, N, _ = x.shape
    h = _sym8()
    w = x.astype(float).copy()
    n = N
    for _ in range(wavelet_levels(N)):
        A = dwt_matrix(n, h)
        w[:, :n, :n] = w[:, :n, :n] @ A.T     # rows
        w[:, :n, :n] = A @ w[:, :n, :n]       # columns
        n //= 2
    return np.einsum("km,mij->kij", dct_matrix(M), w)[:, None, :, :]


def wdct_adjoint(c: np.ndarray) -> np.ndarray:
    """T^T (= T^-1, T orthonormal): inverse DCT along channels, then the inverse levels from the
    coarsest.  [M, 1, N, N] -> [M, N, N]."""
    M, N = c.shape[0], c.shape[-1]
    h = _sym8()
    w = np.einsum("km,kij->mij", dct_matrix(M), c[:, 0])
    J = wavelet_levels(N)
    for lev in reversed(range(J)):
        n = N >> lev
        A = dwt_matrix(n, h)
        w[:, :n, :n] = A.T @ w[:, :n, :n]     # columns
        w[:, :n, :n] = w[:, :n, :n] @ A       # rows
    return w


PRIORS = {
    "tv": (tv_forward, tv_adjoint),
    "tv_iso": (tv_forward, tv_adjoint),   # isotropic TV: same T, coupled shrinkage (reading R20)
    "dct8": (dct8_forward, dct8_adjoint),
    "l1": (l1_forward, l1_adjoint),
    "wdct": (wdct_forward, wdct_adjoint),   # Symmlet-8 (x) channel DCT (readings R24-R26)
}


def ncomp_of(prior: str) -> int:
    return 2 if prior in ("tv", "tv_iso") else 1


def gram_eigenvalues(prior: str, N: int) -> np.ndarray:
    """g(w): DFT eigenvalues of the circulant T^T T.  Computed as the DFT of
    the kernel T^T T delta (Eq. solx_Trans with BCCB T^T T).  For an
    orthonormal T (DCT, identity) T^T T = I and g = 1 (Eq. solx_Trans_DFT)."""
    if prior in ("dct8", "l1", "wdct"):
        return np.ones((N, N))
    fwd, adj = PRIORS[prior]
    delta = np.zeros((N, N))
    delta[0, 0] = 1.0
    kern = adj(fwd(delta))
    g = dft2(kern)
    return g.real


def group_soft(v: np.ndarray, tau: float) -> np.ndarray:
    """Proximal map of tau ||.||_2 on the two-component axis (-3) of v = [..., 2, N, N]:
    v max(0, 1 - tau / ||v||), the t-update of isotropic TV (reading R20)."""
    n = np.sqrt(np.sum(v * v, axis=-3, keepdims=True))
    f = np.where(n > tau, 1.0 - tau / np.where(n > 0, n, 1.0), 0.0)
    return v * f


def shrink(prior: str, v: np.ndarray, tau: float) -> np.ndarray:
    """t-update of Eq. solt_trans for the prior: coupled for isotropic TV, elementwise otherwise."""
    return group_soft(v, tau) if prior == "tv_iso" else soft(v, tau)


def soft(w: np.ndarray, tau: float) -> np.ndarray:
    """Soft-thresholding (Eq. solt_trans): sign(w) max(|w| - tau, 0), with
    sign(w) = 1 for w > 0 and -1 otherwise."""
    s = np.where(w > 0, 1.0, -1.0)
    return s * np.maximum(np.abs(w) - tau, 0.0)


# ---------------------------------------------------------------------------
# Per-frequency algebra (Section IV-A, Eqs. solx_Trans_DFT and recinv)
# ---------------------------------------------------------------------------
def psf_spectra(h: np.ndarray) -> np.ndarray:
    """Lambda[k, m] = unnormalised DFT of h_{k,m} (reading R4)."""
    return dft2(h)


def per_bin_lambda(Lam: np.ndarray) -> np.ndarray:
    """[K, M, N, N] -> [N, N, K, M]: the K x M matrix Lambda(w) at each bin."""
    return np.transpose(Lam, (2, 3, 0, 1))


def form_psi(Lam: np.ndarray, g: np.ndarray, rho: float, beta: float) -> np.ndarray:
    """Psi(w) = rho g(w) I + beta Lambda(w)^H Lambda(w)  -> [N, N, M, M] (reading R3)."""
    Lb = per_bin_lambda(Lam)
    M = Lb.shape[-1]
    LhL = np.einsum("abki,abkj->abij", Lb.conj(), Lb)
    return rho * g[..., None, None] * np.eye(M) + beta * LhL


def pinv_hermitian(A: np.ndarray, rel_cut: float = 1e-10) -> np.ndarray:
    """Min-norm pseudo-inverse of a Hermitian PSD matrix (reading R2)."""
    ev, V = np.linalg.eigh(A)
    cut = rel_cut * max(ev.max(), 0.0)
    inv = np.where(ev > cut, 1.0 / np.where(ev > cut, ev, 1.0), 0.0)
    return (V * inv) @ V.conj().T


def invert_psi(Psi: np.ndarray, g: np.ndarray, gz: float = 1e-12) -> np.ndarray:
    """Psi^{-1} at every bin; pseudo-inverse where g(w) = 0 (reading R2)."""
    out = np.linalg.inv(np.where((g <= gz * g.max())[..., None, None],
                                 np.eye(Psi.shape[-1]), Psi))
    sing = np.argwhere(g <= gz * g.max())
    for a, b in sing:
        out[a, b] = pinv_hermitian(Psi[a, b])
    return out


def recursive_block_inverse(P: np.ndarray) -> np.ndarray:
    """Inverse of one S x S matrix by the 2 x 2 block recursion of Eq. recinv:
    with S_c = P22 - P21 P11^{-1} P12 and B = -S_c^{-1},
    inv = [[P11^{-1} - P11^{-1} P12 B P21 P11^{-1}, P11^{-1} P12 B],
           [B P21 P11^{-1}, -B]]."""
    S = P.shape[0]
    if S == 1:
        return np.array([[1.0 / P[0, 0]]])
    h = S // 2
    P11, P12, P21, P22 = P[:h, :h], P[:h, h:], P[h:, :h], P[h:, h:]
    P11i = recursive_block_inverse(P11)
    B = -recursive_block_inverse(P22 - P21 @ P11i @ P12)
    A = P11i - P11i @ P12 @ B @ P21 @ P11i
    top = np.concatenate([A, P11i @ P12 @ B], axis=1)
    bot = np.concatenate([B @ P21 @ P11i, -B], axis=1)
    return np.concatenate([top, bot], axis=0)


def rhs_bhat(Lam: np.ndarray, y: np.ndarray, beta: float) -> np.ndarray:
    """b(w) = beta Lambda(w)^H (F y)(w)  -> [M, N, N] (Alg. 1, setup)."""
    Y = dft2(y)
    return beta * np.einsum("kmab,kab->mab", Lam.conj(), Y)


def apply_per_bin(Pinv: np.ndarray, v: np.ndarray) -> np.ndarray:
    """x(w) = Pinv(w) v(w); Pinv [N,N,M,M], v [M,N,N] -> [M,N,N]."""
    return np.einsum("abij,jab->iab", Pinv, v)


# ---------------------------------------------------------------------------
# Algorithm 1 (analysis prior)
# ---------------------------------------------------------------------------
@dataclass
class AnalysisSetup:
    N: int
    M: int
    prior: str
    lam: float
    rho: float
    beta: float
    Lam: np.ndarray     # [K, M, N, N]
    g: np.ndarray       # [N, N]
    Pinv: np.ndarray    # [N, N, M, M]
    bhat: np.ndarray    # [M, N, N]


def analysis_setup(h: np.ndarray, y: np.ndarray, prior: str, lam: float, rho: float,
                   beta: float) -> AnalysisSetup:
    """Alg. 1 setup: Psi^{-1} = (rho T^H T + beta Lambda^H Lambda)^{-1} per bin and
    beta Lambda^H F y."""
    K, M, N, _ = h.shape
    Lam = psf_spectra(h)
    g = gram_eigenvalues(prior, N)
    Psi = form_psi(Lam, g, rho, beta)
    Pinv = invert_psi(Psi, g)
    return AnalysisSetup(N, M, prior, lam, rho, beta, Lam, g, Pinv, rhs_bhat(Lam, y, beta))


def x_update(S: AnalysisSetup, t: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Eq. solx_Trans_DFT: x = F^H Psi^{-1} (beta Lambda^H F y + rho F T^H (t - u))."""
    _, adj = PRIORS[S.prior]
    q = adj(t - u)
    xhat = apply_per_bin(S.Pinv, S.bhat + S.rho * dft2(q))
    return idft2(xhat).real


def t_u_update(S: AnalysisSetup, x: np.ndarray, u: np.ndarray):
    """Eq. solt_trans and Eq. subu_trans: t = soft(Tx + u, lambda/rho); u += Tx - t."""
    fwd, _ = PRIORS[S.prior]
    w = fwd(x)
    t = shrink(S.prior, w + u, S.lam / S.rho)
    return t, u + w - t, w


@dataclass
class IterRecord:
    x: np.ndarray
    t: np.ndarray
    u: np.ndarray
    r: float            # ||Tx - t||
    s: float            # rho ||t - t_prev||
    r_rel: float
    s_rel: float


def analysis_step(S: AnalysisSetup, t: np.ndarray, u: np.ndarray):
    """One iteration of Alg. 1 (x, then t, then u).  Returns (x, t_new, u_new, w=Tx)."""
    x = x_update(S, t, u)
    t_new, u_new, w = t_u_update(S, x, u)
    return x, t_new, u_new, w


def run_analysis(S: AnalysisSetup, iters: int, t0=None, u0=None, keep_history: bool = False):
    """Alg. 1 for a fixed number of iterations from t^0 = u^0 = 0 (reading R5)."""
    ncomp = ncomp_of(S.prior)
    t = np.zeros((S.M, ncomp, S.N, S.N)) if t0 is None else t0.copy()
    u = np.zeros_like(t) if u0 is None else u0.copy()
    hist: List[IterRecord] = []
    x = None
    for _ in range(iters):
        x, t_new, u_new, w = analysis_step(S, t, u)
        r = float(np.linalg.norm(w - t_new))
        s = S.rho * float(np.linalg.norm(t_new - t))
        den_r = max(float(np.linalg.norm(w)), float(np.linalg.norm(t_new)), 1e-300)
        den_s = max(S.rho * float(np.linalg.norm(u_new)), 1e-300)
        if keep_history:
            hist.append(IterRecord(x, t_new, u_new, r, s, r / den_r, s / den_s))
        t, u = t_new, u_new
    return x, t, u, hist


def adapt_rho(rho: float, r: float, s: float, tau: float = 2.0, mu: float = 10.0) -> float:
    """Eq. paramS: tau rho if ||r|| > mu ||s||, rho / tau if ||s|| > mu ||r||, else rho
    (r the primal residual ||Tx - t||, s the dual residual rho ||t - t_prev||, reading R11)."""
    if r > mu * s:
        return rho * tau
    if s > mu * r:
        return rho / tau
    return rho


def run_analysis_adaptive(h: np.ndarray, y: np.ndarray, prior: str, lam: float, rho: float, beta: float,
                          iters: int, check_every: int, tau: float = 2.0, mu: float = 10.0):
    """Alg. 1 from t = u = 0 with the penalty adapted by Eq. paramS after every check_every-th
    iteration (reading R17).  When rho changes the scaled dual is rescaled, u <- u rho/rho', so
    that the unscaled multiplier rho u is unchanged (reading R18), and Psi^{-1} and the data term
    are formed again for rho'.  Returns (x, t, u, [rho after each iteration])."""
    S = analysis_setup(h, y, prior, lam, rho, beta)
    ncomp = ncomp_of(prior)
    t = np.zeros((S.M, ncomp, S.N, S.N))
    u = np.zeros_like(t)
    rhos = []
    x = None
    for it in range(iters):
        x, t_new, u_new, w = analysis_step(S, t, u)
        if (it + 1) % check_every == 0:
            r = float(np.linalg.norm(w - t_new))
            s = S.rho * float(np.linalg.norm(t_new - t))
            rho_new = adapt_rho(S.rho, r, s, tau, mu)
            if rho_new != S.rho:
                u_new = u_new * (S.rho / rho_new)
                S = analysis_setup(h, y, prior, lam, rho_new, beta)
        t, u = t_new, u_new
        rhos.append(S.rho)
    return x, t, u, rhos


def objective(x: np.ndarray, h: np.ndarray, y: np.ndarray, prior: str, lam: float, beta: float) -> float:
    """Eq. rls with the analysis prior: beta/2 ||y - Hx||^2 + lambda ||Tx||_1 (H spatial)."""
    fwd, _ = PRIORS[prior]
    res = y - forward_H(x, h)
    w = fwd(x)
    reg = np.sum(np.sqrt(np.sum(w * w, axis=-3))) if prior == "tv_iso" else np.sum(np.abs(w))
    return 0.5 * beta * float(np.sum(res * res)) + lam * float(reg)


# ---------------------------------------------------------------------------
# Algorithm 2 (synthesis prior, 2D convolutional dictionary per slice)
# ---------------------------------------------------------------------------
@dataclass
class ConvDictSetup:
    N: int
    M: int
    L: int
    lam: float
    rho: float
    beta: float
    Lam: np.ndarray     # [K, M, N, N]
    theta: np.ndarray   # [L, N, N]  DFT of the embedded filters
    Pinv: np.ndarray    # [N, N, M, M] (I + beta Lambda^H Lambda)^{-1}
    bhat: np.ndarray    # [M, N, N]
    mu: float = 0.0     # Tikhonov weight on the code gradients (Eq. DL_PriorHP_conv)
    rho_n: np.ndarray = None  # [N, N] diagonal of the z-update per bin: rho + mu (|r1^|^2 + |r2^|^2)


def embed_filters(d: np.ndarray, N: int) -> np.ndarray:
    """P x P filter (centre P//2) placed on the N x N torus, centre at (0,0)."""
    L, P, _ = d.shape
    c = P // 2
    out = np.zeros((L, N, N))
    for l in range(L):
        for i in range(P):
            for j in range(P):
                out[l, (i - c) % N, (j - c) % N] = d[l, i, j]
    return out


def convdict_setup(h: np.ndarray, y: np.ndarray, d: np.ndarray, lam: float, rho: float,
                   beta: float, mu: float = 0.0) -> ConvDictSetup:
    """Alg. 2 setup with t = 1 (P = I for the convolutional dictionary, Eq. solx_synt).

    mu > 0 adds the gradient (Tikhonov) penalty mu/2 sum_m sum_i ||r_i * z_m||^2 on the codes
    (Eq. DL_PriorHP_conv, 2D: r_1, r_2 the circular differences along the two axes).  Its normal
    equation gains mu sum_i R_i^H R_i (the note after Eq. solz), diagonalised by the DFT with the
    eigenvalues of D^T D of the TV operator, so per bin the z-update matrix is
    (rho + mu g(w)) I + conj(theta) theta^T: still diagonal plus rank one."""
    K, M, N, _ = h.shape
    Lam = psf_spectra(h)
    Psi = form_psi(Lam, np.ones((N, N)), 1.0, beta)
    Pinv = np.linalg.inv(Psi)
    theta = dft2(embed_filters(d, N))
    rho_n = rho + mu * gram_eigenvalues("tv", N)
    return ConvDictSetup(N, M, d.shape[0], lam, rho, beta, Lam, theta, Pinv, rhs_bhat(Lam, y, beta), mu, rho_n)


def sherman_morrison(theta_n: np.ndarray, c_n: np.ndarray, rho: float) -> np.ndarray:
    """Eq. solz_DFT_SM at one bin (reading R10): solve (rho I + conj(theta) theta^T) v = c.
    With the gradient penalty, rho is the bin's diagonal rho + mu g(w)."""
    a = theta_n.conj()
    return (c_n - a * (theta_n @ c_n) / (rho + np.vdot(theta_n, theta_n).real)) / rho


def convdict_step(C: ConvDictSetup, z: np.ndarray, t: np.ndarray, u: np.ndarray):
    """One iteration of Alg. 2: x (Eq. solx_synt_DFT), z (Eqs. solz_DFT,
    solz_DFT_SM), t (Eq. softADMM), u (Eq. subu_dic).  z, t, u: [L, M, N, N]."""
    Z = dft2(z)                                            # F z per (l, m)
    p = np.einsum("lab,lmab->mab", C.theta, Z)             # F D z per channel
    xhat = apply_per_bin(C.Pinv, C.bhat + p)
    x = idft2(xhat).real
    c = C.theta.conj()[:, None] * dft2(x)[None] + C.rho * dft2(t - u)
    v = np.empty_like(c)
    for a in range(C.N):
        for b in range(C.N):
            th = C.theta[:, a, b]
            for m in range(C.M):
                v[:, m, a, b] = sherman_morrison(th, c[:, m, a, b], C.rho_n[a, b])
    z_new = idft2(v).real
    t_new = soft(z_new + u, C.lam / C.rho)
    u_new = u + z_new - t_new
    return x, z_new, t_new, u_new


# ---------------------------------------------------------------------------
# 3D convolutional dictionary (Section IV-B, the 3D case of Alg. 2; readings R27-R28): L filters
# d_l of Q x P x P taps (channel, row, column), one 3D code map z_l of S x N x N per filter,
# x_s = sum_l (d_l (*)_3 z_l)_s with circular convolution along all three axes
# ---------------------------------------------------------------------------
def dft1_matrix(S: int, sign: int = -1) -> np.ndarray:
    """S-point DFT matrix, entries exp(sign 2 pi i ((j k) mod S) / S)."""
    j = np.arange(S)
    return np.exp(sign * 2j * math.pi * ((j[:, None] * j[None, :]) % S) / S)


def dft3(v: np.ndarray) -> np.ndarray:
    """Unnormalised 3D DFT over the last three axes [..., S, N, N]: the 2D DFT of every slice,
    then the 1D DFT along the channel axis (F_3D = F_1D (x) F_2D)."""
    V = dft2(v)
    return np.einsum("ks,...sab->...kab", dft1_matrix(v.shape[-3]), V)


def idft3(V: np.ndarray) -> np.ndarray:
    S = V.shape[-3]
    W = np.einsum("sk,...kab->...sab", dft1_matrix(S, +1), V) / S
    return idft2(W)


def embed_filters3d(d: np.ndarray, N: int, S: int) -> np.ndarray:
    """Q x P x P filters (centre (Q//2, P//2, P//2)) placed on the S x N x N torus with the centre
    at (0, 0, 0) (reading R27)."""
    L, Q, P, _ = d.shape
    out = np.zeros((L, S, N, N))
    for l in range(L):
        for q in range(Q):
            for i in range(P):
                for j in range(P):
                    out[l, (q - Q // 2) % S, (i - P // 2) % N, (j - P // 2) % N] += d[l, q, i, j]
    return out


@dataclass
class ConvDict3DSetup:
    N: int
    M: int          # image channels S
    L: int
    lam: float
    rho: float
    beta: float
    Pinv: np.ndarray    # [N, N, M, M] (I + beta Lambda^H Lambda)^{-1}
    bhat: np.ndarray    # [M, N, N]
    theta3: np.ndarray  # [L, M, N, N] 3D DFT of the embedded filters (kappa, w1, w2)


def convdict3d_setup(h: np.ndarray, y: np.ndarray, d3: np.ndarray, lam: float, rho: float,
                     beta: float) -> ConvDict3DSetup:
    """Alg. 2 setup for 3D filters: the x-update factor is the 2D one (t = 1, Eq. solx_synt_DFT);
    Theta_l is the 3D DFT of the embedded filter."""
    K, M, N, _ = h.shape
    if d3.shape[1] > M:
        raise ValueError("filter depth Q must not exceed the channel count")
    Lam = psf_spectra(h)
    Pinv = np.linalg.inv(form_psi(Lam, np.ones((N, N)), 1.0, beta))
    theta3 = dft3(embed_filters3d(d3, N, M))
    return ConvDict3DSetup(N, M, d3.shape[0], lam, rho, beta, Pinv, rhs_bhat(Lam, y, beta), theta3)


def convdict3d_step(C: ConvDict3DSetup, z: np.ndarray, t: np.ndarray, u: np.ndarray):
    """One iteration of Alg. 2 with 3D filters, z, t, u [L, S, N, N]:
    x: the last term of Eq. solx_synt_DFT is F~ D~ z = (F_1D^H (x) I) sum_l Theta_l F_3D z_l, i.e.
       the 3D spectra multiplied and summed over l, then a 1D inverse DFT along the channel axis;
    z: the normal equation Eq. solz, (rho I + D~^H D~) z = D~^H x + rho (t - u), is diagonal plus
       rank one in every 3D bin (Sherman-Morrison, Eq. solz_DFT_SM with reading R10), with
       D~^H x <-> conj(Theta_l) F_3D x;
    t, u: Eqs. softADMM and subu_dic."""
    S = C.M
    Zh = dft3(z)                                                    # [L, S(kappa), N, N]
    q = np.einsum("lkab,lkab->kab", C.theta3, Zh)                   # F_3D of D~ z
    p = np.einsum("sk,kab->sab", dft1_matrix(S, +1), q) / S         # 2D spectra of (D~ z)_s
    xhat = apply_per_bin(C.Pinv, C.bhat + p)
    x = idft2(xhat).real
    X3 = np.einsum("ks,sab->kab", dft1_matrix(S), xhat)             # F_3D x
    c = C.theta3.conj() * X3[None] + C.rho * dft3(t - u)
    v = np.empty_like(c)
    for k in range(S):
        for a in range(C.N):
            for b in range(C.N):
                v[:, k, a, b] = sherman_morrison(C.theta3[:, k, a, b], c[:, k, a, b], C.rho)
    z_new = idft3(v).real
    t_new = soft(z_new + u, C.lam / C.rho)
    u_new = u + z_new - t_new
    return x, z_new, t_new, u_new


def run_convdict3d(C: ConvDict3DSetup, iters: int):
    z = np.zeros((C.L, C.M, C.N, C.N))
    t = np.zeros_like(z)
    u = np.zeros_like(z)
    x = None
    for _ in range(iters):
        x, z, t, u = convdict3d_step(C, z, t, u)
    return x, z, t, u


def run_convdict(C: ConvDictSetup, iters: int, keep_history: bool = False):
    """Alg. 2 from z^0 = t^0 = u^0 = 0 (reading R5)."""
    z = np.zeros((C.L, C.M, C.N, C.N))
    t = np.zeros_like(z)
    u = np.zeros_like(z)
    hist = []
    x = None
    for _ in range(iters):
        x, z, t_new, u = convdict_step(C, z, t, u)
        if keep_history:
            hist.append((x, z, t_new, u))
        t = t_new
    return x, z, t, u, hist


# ---------------------------------------------------------------------------
# Online convolutional dictionary update (Section IV-B "Convolutional dictionary update",
# Eqs. set, Constrained2, d_admm, g_admm, h_admm, sold_3D; 2D filters shared by the slices)
# ---------------------------------------------------------------------------
def crop_filters(v: np.ndarray, P: int) -> np.ndarray:
    """Q^T: the P x P support (centre at P//2, placed at the origin of the torus) of [L, N, N] maps."""
    N = v.shape[-1]
    idx = (np.arange(P) - P // 2) % N
    return v[:, idx][:, :, idx]


def project_filters(v: np.ndarray, P: int) -> np.ndarray:
    """Solution of Eq. g_admm: Q Q^T v / ||Q^T v|| per filter (support constraint and unit norm)."""
    L, N, _ = v.shape
    c = crop_filters(v, P)
    n = np.sqrt(np.sum(c * c, axis=(1, 2)))
    return embed_filters(c / n[:, None, None], N)


def dict_update(x: np.ndarray, z: np.ndarray, g: np.ndarray, e: np.ndarray, sigma: float, P: int):
    """One step of the filter ADMM (Eqs. d_admm, g_admm, h_admm): d solves the normal equation of
    Eq. sold_3D summed over the slices, per frequency
        (sigma I + sum_s conj(zhat_s) zhat_s^T) dhat = sum_s conj(zhat_s) xhat_s + sigma F(g - e),
    then g = projection of d + e onto the constraint set (Eq. set) and e <- e + d - g (readings
    R21-R23).  x [S, N, N], z [L, S, N, N], g, e [L, N, N]."""
    L, S, N, _ = z.shape
    Zh = dft2(z)
    Xh = dft2(x)
    GE = dft2(g - e)
    dh = np.empty((L, N, N), dtype=complex)
    for a in range(N):
        for b in range(N):
            zs = Zh[:, :, a, b]                                   # [L, S]
            A = sigma * np.eye(L) + zs.conj() @ zs.T
            rhs = zs.conj() @ Xh[:, a, b] + sigma * GE[:, a, b]
            dh[:, a, b] = np.linalg.solve(A, rhs)
    d = idft2(dh).real
    g_new = project_filters(d + e, P)
    return d, g_new, e + d - g_new


def run_convdict_learn(h: np.ndarray, y: np.ndarray, d0: np.ndarray, lam: float, rho: float, beta: float,
                       sigma: float, iters: int, check_every: int = 0, tau: float = 2.0, mu: float = 10.0):
    """Alg. 2 with the online dictionary update after every iteration (reading R21): the x-, z-,
    t- and u-updates use the current filters g, then one filter-ADMM step updates (d, g, e) from
    the new x and z.  From z = t = u = 0, g = the given unit-norm filters, e = 0.

    check_every > 0 adapts sigma like rho (Section V applies the Eq. paramS rule to sigma too,
    reading R29): after every check_every-th iteration, with r = ||d - g|| and
    s = sigma ||g - g_prev||, sigma' = adapt_rho(sigma, r, s, tau, mu), and on a change the scaled
    dual is rescaled, e <- e sigma / sigma', so that the multiplier sigma e is kept.
    Returns (x, z, t, u, filters [L, P, P]), plus the sigma after each iteration when adapting."""
    P = d0.shape[-1]
    C = convdict_setup(h, y, d0, lam, rho, beta)
    g = embed_filters(d0, C.N)
    e = np.zeros_like(g)
    z = np.zeros((C.L, C.M, C.N, C.N))
    t = np.zeros_like(z)
    u = np.zeros_like(z)
    x = None
    sigmas = []
    for it in range(iters):
        C.theta = dft2(g)
        x, z, t_new, u = convdict_step(C, z, t, u)
        t = t_new
        g_prev = g
        d, g, e = dict_update(x, z, g, e, sigma, P)
        if check_every > 0 and (it + 1) % check_every == 0:
            r = float(np.linalg.norm(d - g))
            s_ = sigma * float(np.linalg.norm(g - g_prev))
            sigma_new = adapt_rho(sigma, r, s_, tau, mu)
            if sigma_new != sigma:
                e = e * (sigma / sigma_new)
                sigma = sigma_new
        sigmas.append(sigma)
    if check_every > 0:
        return x, z, t, u, crop_filters(g, P), sigmas
    return x, z, t, u, crop_filters(g, P)


def convdict_objective(x, z, d, h, y, lam, beta) -> float:
    """beta/2 ||y - Hx||^2 + 1/2 ||sum_l d_l (*) z_l - x||^2 + lambda ||z||_1 (reading R9)."""
    N = x.shape[-1]
    de = embed_filters(d, N)
    Dz = np.stack([sum(circconv2(z[l, m], de[l]) for l in range(z.shape[0])) for m in range(x.shape[0])])
    r1 = y - forward_H(x, h)
    r2 = Dz - x
    return 0.5 * beta * float(np.sum(r1 * r1)) + 0.5 * float(np.sum(r2 * r2)) + lam * float(np.sum(np.abs(z)))

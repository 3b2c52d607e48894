"""Seeded synthetic inputs for the superimposed-convolution imaging model.

This module only *draws* data: images, point-spread functions, dictionary
filters, sparse codes, noise and request streams.  It holds none of the
reconstruction method's arithmetic (no ADMM step, no factor, no transform of
the prior).  Both the CUDA path and the FP64 oracle consume what it returns.

The forward model used to synthesise measurements is the paper's Section II
model, y_k = sum_s x_s (*) h_{k,s} + w_k with circular 2D convolution and the
PSF origin at index (0, 0).  The convolution here is done with numpy's FFT as
a library primitive purely to make test data; the oracle has its own spatial
convolution and never calls this module.

Every generator takes an explicit ``numpy.random.Generator`` or seed; nothing
reads global random state.  Seeds default to 20060830 + workload index.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

BASE_SEED = 20060830


# --------------------------------------------------------------------------
# point-spread functions (origin at (0,0), circular wrap, unit sum)
# --------------------------------------------------------------------------
def _wrapped_coords(N: int):
    d = np.arange(N)
    d = np.minimum(d, N - d).astype(np.float64)  # wrapped distance to 0
    # signed wrapped offsets, used where direction matters
    return d


def gaussian_psf(N: int, sigma: float) -> np.ndarray:
    """Isotropic Gaussian defocus PSF of width ``sigma`` px centred at (0,0),
    wrapped on the N x N torus and normalised to unit sum."""
    d = _wrapped_coords(N)
    r2 = d[:, None] ** 2 + d[None, :] ** 2
    h = np.exp(-0.5 * r2 / (sigma * sigma))
    return h / h.sum()


def _fft_circconv(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Circular convolution through numpy's FFT (data synthesis only)."""
    s = a.shape[-2:]
    return np.fft.irfft2(np.fft.rfft2(a) * np.fft.rfft2(b), s=s)


def disk_gaussian_psf(N: int, radius: float, sigma0: float = 1.0) -> np.ndarray:
    """Disk of the given radius (pixels whose wrapped distance to (0,0) is at
    most ``radius``; radius 0 is a delta) convolved with a Gaussian of width
    ``sigma0``, normalised to unit sum."""
    d = _wrapped_coords(N)
    r = np.sqrt(d[:, None] ** 2 + d[None, :] ** 2)
    disk = (r <= radius + 1e-12).astype(np.float64)
    disk /= disk.sum()
    h = _fft_circconv(disk, gaussian_psf(N, sigma0))
    h = np.maximum(h, 0.0)
    return h / h.sum()


def gaussian_psf_bank(N: int, K: int, M: int) -> np.ndarray:
    """h[k, m] Gaussian with sigma_{k,m} = 0.5 + 1.5 |k - m| px."""
    h = np.empty((K, M, N, N), dtype=np.float64)
    for k in range(K):
        for m in range(M):
            h[k, m] = gaussian_psf(N, 0.5 + 1.5 * abs(k - m))
    return h


def disk_gaussian_psf_bank(N: int, K: int, M: int, rmax: float = 12.0) -> np.ndarray:
    """h[k, m] = disk(r_{k,m}) (*) Gaussian(1 px), r_{k,m} = rmax |k-m| / (max(K,M)-1)."""
    h = np.empty((K, M, N, N), dtype=np.float64)
    denom = max(max(K, M) - 1, 1)
    cache = {}
    for k in range(K):
        for m in range(M):
            r = rmax * abs(k - m) / denom
            if r not in cache:
                cache[r] = disk_gaussian_psf(N, r)
            h[k, m] = cache[r]
    return h


# --------------------------------------------------------------------------
# images
# --------------------------------------------------------------------------
def rectangles_image(rng: np.random.Generator, N: int, M: int, n_rect: int = 8) -> np.ndarray:
    """Nonnegative image: per channel, ``n_rect`` additive axis-aligned
    rectangles, side lengths uniform in [4, N/4], positions uniform (wrapped),
    amplitudes U[0, 1]."""
    x = np.zeros((M, N, N), dtype=np.float64)
    lo, hi = 4, max(4, N // 4)
    for m in range(M):
        for _ in range(n_rect):
            h_ = int(rng.integers(lo, hi + 1))
            w_ = int(rng.integers(lo, hi + 1))
            r0 = int(rng.integers(0, N))
            c0 = int(rng.integers(0, N))
            a = float(rng.uniform(0.0, 1.0))
            rows = (r0 + np.arange(h_)) % N
            cols = (c0 + np.arange(w_)) % N
            x[m][np.ix_(rows, cols)] += a
    return x


def spectral_image(rng: np.random.Generator, N: int, M: int, n_cells: int = 16) -> np.ndarray:
    """Piecewise-constant spatial masks (Voronoi cells of ``n_cells`` random
    sites) times smooth spectra: each cell's spectrum along the channel axis
    is a sum of 3 Gaussians with amplitude U[0.2,1], centre U[0,M-1] and
    width U[1, M/2]."""
    sites = rng.uniform(0, N, size=(n_cells, 2))
    ii, jj = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    best = np.full((N, N), np.inf)
    label = np.zeros((N, N), dtype=np.int64)
    for c in range(n_cells):
        di = np.abs(ii - sites[c, 0]); di = np.minimum(di, N - di)
        dj = np.abs(jj - sites[c, 1]); dj = np.minimum(dj, N - dj)
        d2 = di * di + dj * dj
        upd = d2 < best
        best[upd] = d2[upd]
        label[upd] = c
    chan = np.arange(M, dtype=np.float64)
    spectra = np.zeros((n_cells, M))
    for c in range(n_cells):
        for _ in range(3):
            a = rng.uniform(0.2, 1.0)
            mu = rng.uniform(0.0, max(M - 1, 0))
            wd = rng.uniform(1.0, max(M / 2.0, 1.0))
            spectra[c] += a * np.exp(-0.5 * ((chan - mu) / wd) ** 2)
    return np.ascontiguousarray(spectra[label].transpose(2, 0, 1))


# --------------------------------------------------------------------------
# convolutional dictionary data
# --------------------------------------------------------------------------
def gabor_filters(rng: np.random.Generator, L: int = 32, P: int = 11) -> np.ndarray:
    """L zero-mean, unit-L2 Gabor filters of size P x P (centre at P//2):
    orientation U[0, pi), envelope width U[1.5, 3.5] px, wavelength 2.5 sigma,
    phase U[0, 2 pi)."""
    c = P // 2
    v, u = np.meshgrid(np.arange(P) - c, np.arange(P) - c, indexing="ij")
    d = np.empty((L, P, P), dtype=np.float64)
    for l in range(L):
        th = rng.uniform(0.0, math.pi)
        sg = rng.uniform(1.5, 3.5)
        lam = 2.5 * sg
        ph = rng.uniform(0.0, 2.0 * math.pi)
        env = np.exp(-(u * u + v * v) / (2.0 * sg * sg))
        car = np.cos(2.0 * math.pi * (u * math.cos(th) + v * math.sin(th)) / lam + ph)
        f = env * car
        f -= f.mean()
        f /= np.linalg.norm(f)
        d[l] = f
    return d


def embed_filters(d: np.ndarray, N: int) -> np.ndarray:
    """Place P x P filters (centre at P//2) on the N x N torus with their
    centre at index (0, 0)."""
    L, P, _ = d.shape
    c = P // 2
    out = np.zeros((L, N, N), dtype=np.float64)
    idx = (np.arange(P) - c) % N
    for l in range(L):
        out[l][np.ix_(idx, idx)] = d[l]
    return out


def bernoulli_gaussian_codes(rng: np.random.Generator, L: int, M: int, N: int, p: float = 0.01) -> np.ndarray:
    """z[l, m] with Bernoulli(p) support and N(0,1) values."""
    mask = rng.random((L, M, N, N)) < p
    return np.where(mask, rng.standard_normal((L, M, N, N)), 0.0)


def convdict_image(d_embedded: np.ndarray, z: np.ndarray) -> np.ndarray:
    """x_m = sum_l d_l (*) z_{l,m} (data synthesis)."""
    L, M = z.shape[:2]
    Dh = np.fft.rfft2(d_embedded)  # [L, N, N/2+1]
    Zh = np.fft.rfft2(z)           # [L, M, N, N/2+1]
    Xh = np.einsum("lab,lmab->mab", Dh, Zh)
    return np.fft.irfft2(Xh, s=z.shape[-2:])


# --------------------------------------------------------------------------
# measurements
# --------------------------------------------------------------------------
def measure(rng: np.random.Generator, x: np.ndarray, h: np.ndarray, snr_db: Optional[float]):
    """y_k = sum_m h_{k,m} (*) x_m + w_k with one noise level for all k:
    sigma^2 = mean((Hx)^2) / 10^(SNR/10).  Returns (y, sigma)."""
    K, M = h.shape[:2]
    Hh = np.fft.rfft2(h)
    Xh = np.fft.rfft2(x)
    clean = np.fft.irfft2(np.einsum("kmab,mab->kab", Hh, Xh), s=x.shape[-2:])
    if snr_db is None:
        return clean, 0.0
    sigma = math.sqrt(float(np.mean(clean * clean)) / 10.0 ** (snr_db / 10.0))
    return clean + sigma * rng.standard_normal(clean.shape), sigma


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Problem:
    """One reconstruction instance: inputs plus ADMM parameters."""
    name: str
    N: int
    K: int
    M: int
    prior: str            # "tv" | "dct8" | "l1" | "convdict"
    lam: float
    rho: float
    beta: float
    iters: int
    h: np.ndarray         # [K, M, N, N] float64
    y: np.ndarray         # [K, N, N] float64
    x_true: np.ndarray    # [M, N, N] float64
    filters: Optional[np.ndarray] = None  # [L, P, P] (convdict only)
    dtype: str = "f32"

    @property
    def voxels(self) -> int:
        return self.N * self.N * self.M


def tiny_tv(seed: int = BASE_SEED + 0, N: int = 64, M: int = 3, iters: int = 50, dtype: str = "f64") -> Problem:
    """M=K=3, 64x64, Gaussian defocus PSFs sigma = 0.5 + 1.5|k-m|, 8 random
    rectangles per channel, 30 dB, anisotropic TV, lambda=1e-2, rho=1,
    beta=1, 50 iterations."""
    rng = np.random.default_rng(seed)
    x = rectangles_image(rng, N, M)
    h = gaussian_psf_bank(N, M, M)
    y, _ = measure(rng, x, h, 30.0)
    return Problem("tiny_tv_64x64x3", N, M, M, "tv", 1e-2, 1.0, 1.0, iters, h, y, x, dtype=dtype)


def spectral_dct(seed: int = BASE_SEED + 1, N: int = 512, M: int = 10, iters: int = 200,
                 lam: float = 1e-3, rho: float = 1e-2, dtype: str = "f32") -> Problem:
    """M=K=10, 512x512, disk-plus-Gaussian defocus PSFs (radius up to 12 px),
    smooth spectra x piecewise-constant masks, 8x8 block-DCT l1 prior,
    30 dB, lambda=1e-3, rho=1e-2, beta=1, 200 iterations."""
    rng = np.random.default_rng(seed)
    x = spectral_image(rng, N, M)
    h = disk_gaussian_psf_bank(N, M, M)
    y, _ = measure(rng, x, h, 30.0)
    return Problem(f"spectral_dct_{N}x{N}x{M}", N, M, M, "dct8", lam, rho, 1.0, iters, h, y, x, dtype=dtype)


def convdict_problem(seed: int = BASE_SEED + 2, N: int = 256, M: int = 5, L: int = 32, P: int = 11,
                     iters: int = 300, dtype: str = "f32") -> Problem:
    """M=K=5, 256x256, 32 Gabor 11x11 filters, 1% Bernoulli-Gaussian codes,
    Gaussian PSFs as in the tiny instance, 25 dB, lambda=0.15, beta=4, rho=8."""
    rng = np.random.default_rng(seed)
    d = gabor_filters(rng, L, P)
    z = bernoulli_gaussian_codes(rng, L, M, N, 0.01)
    x = convdict_image(embed_filters(d, N), z)
    h = gaussian_psf_bank(N, M, M)
    y, _ = measure(rng, x, h, 25.0)
    return Problem(f"convdict_{N}x{N}x{M}_L{L}", N, M, M, "convdict", 0.15, 8.0, 4.0, iters, h, y, x,
                   filters=d, dtype=dtype)


def channel_profile_filters(rng: np.random.Generator, d2: np.ndarray, Q: int) -> np.ndarray:
    """3D filters [L][Q][P][P]: each 2D filter times a Gaussian profile along the channels (centre
    Q//2, width U[0.7, 2] channels), scaled to unit L2 (data synthesis for the 3D dictionary)."""
    L = d2.shape[0]
    q = np.arange(Q) - Q // 2
    out = np.empty((L,) + (Q,) + d2.shape[1:], dtype=np.float64)
    for l in range(L):
        w = np.exp(-(q * q) / (2.0 * rng.uniform(0.7, 2.0) ** 2))
        out[l] = w[:, None, None] * d2[l][None]
        out[l] /= np.linalg.norm(out[l])
    return out


def convdict3d_image(d3: np.ndarray, z: np.ndarray) -> np.ndarray:
    """x = sum_l d3_l (*) z_l with circular 3D convolution over (channel, row, column), filters
    [L][Q][P][P] centred at (Q//2, P//2, P//2), codes [L][M][N][N] (data synthesis)."""
    L, Q, P, _ = d3.shape
    M, N = z.shape[1], z.shape[-1]
    emb = np.zeros((L, M, N, N))
    iq, ip = (np.arange(Q) - Q // 2) % M, (np.arange(P) - P // 2) % N
    for l in range(L):
        emb[l][np.ix_(iq, ip, ip)] = d3[l]
    Xh = np.einsum("lkab,lkab->kab", np.fft.fftn(emb, axes=(1, 2, 3)), np.fft.fftn(z, axes=(1, 2, 3)))
    return np.fft.ifftn(Xh, axes=(0, 1, 2)).real


def convdict3d_problem(seed: int = BASE_SEED + 5, N: int = 256, M: int = 16, L: int = 6, Q: int = 5, P: int = 11,
                       iters: int = 30, dtype: str = "f32") -> Problem:
    """3D convolutional dictionary (Section V's spectral experiment in shape: filters of Q taps
    along the channels): Gabor P x P filters times a Gaussian channel profile, 1%
    Bernoulli-Gaussian 3D codes, Gaussian defocus PSFs as in the tiny instance, 25 dB,
    lambda=0.15, beta=4, rho=8."""
    rng = np.random.default_rng(seed)
    d3 = channel_profile_filters(rng, gabor_filters(rng, L, P), Q)
    z = bernoulli_gaussian_codes(rng, L, M, N, 0.01)
    x = convdict3d_image(d3, z)
    h = gaussian_psf_bank(N, M, M)
    y, _ = measure(rng, x, h, 25.0)
    return Problem(f"convdict3d_{N}x{N}x{M}_L{L}_Q{Q}", N, M, M, "convdict", 0.15, 8.0, 4.0, iters, h, y, x,
                   filters=d3, dtype=dtype)


def mixed_batch(seed: int = BASE_SEED + 3, n_inst: int = 64, sizes: Sequence[int] = (128, 256, 512, 1024),
                Ms: Sequence[int] = (3, 5, 10), iters: int = 100) -> List[Problem]:
    """Uneven batch: N uniform over ``sizes``, M=K uniform over ``Ms``; M=3
    instances draw rectangles + Gaussian PSFs, the others spectral images +
    disk-plus-Gaussian PSFs; anisotropic TV, lambda=1e-2, rho=1, beta=1, 30 dB."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_inst):
        N = int(rng.choice(list(sizes)))
        M = int(rng.choice(list(Ms)))
        sub = np.random.default_rng(int(rng.integers(0, 2**63 - 1)))
        if M == 3:
            x = rectangles_image(sub, N, M)
            h = gaussian_psf_bank(N, M, M)
        else:
            x = spectral_image(sub, N, M)
            h = disk_gaussian_psf_bank(N, M, M)
        y, _ = measure(sub, x, h, 30.0)
        out.append(Problem(f"batch{i}_{N}x{N}x{M}", N, M, M, "tv", 1e-2, 1.0, 1.0, iters, h, y, x))
    return out


@dataclasses.dataclass
class Request:
    arrival_s: float
    N: int
    M: int
    prior: str
    psf_id: int
    seed: int


def request_stream(seed: int = BASE_SEED + 4, n: int = 2000, rate_hz: float = 200.0,
                   sizes: Sequence[int] = (256, 512, 1024, 2048), Ms: Sequence[int] = (3, 5, 10),
                   priors: Sequence[str] = ("tv", "dct8"), psf_pool: int = 4) -> List[Request]:
    """Poisson arrivals (exponential gaps, mean 1/rate) of reconstructions with
    N, M and prior drawn uniformly; PSF sets come from a small pool per (N, M)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(n):
        t += float(rng.exponential(1.0 / rate_hz))
        out.append(Request(t, int(rng.choice(list(sizes))), int(rng.choice(list(Ms))),
                           str(rng.choice(list(priors))), int(rng.integers(0, psf_pool)),
                           int(rng.integers(0, 2**31 - 1))))
    return out


def request_problem(req: Request, iters: int = 300) -> Problem:
    """Materialise one served request (rectangles/Gaussian PSFs for M=3,
    spectral/disk PSFs otherwise; lambda=1e-2, rho=1 for TV; lambda=1e-3,
    rho=1e-2 for DCT)."""
    rng = np.random.default_rng(req.seed)
    N, M = req.N, req.M
    if M == 3:
        x = rectangles_image(rng, N, M)
        h = gaussian_psf_bank(N, M, M)
    else:
        x = spectral_image(rng, N, M)
        h = disk_gaussian_psf_bank(N, M, M)
    y, _ = measure(rng, x, h, 30.0)
    if req.prior == "tv":
        lam, rho = 1e-2, 1.0
    else:
        lam, rho = 1e-3, 1e-2
    return Problem(f"req_{N}x{N}x{M}_{req.prior}", N, M, M, req.prior, lam, rho, 1.0, iters, h, y, x)


def random_state(rng: np.random.Generator, prior: str, M: int, N: int, scale: float = 0.1):
    """Random ADMM auxiliary/dual pair (t, u) in the prior's transform domain
    (TV: 2 components per channel, DCT/l1: 1), for step-level parity tests."""
    ncomp = 2 if prior in ("tv", "tv_iso") else 1
    t = scale * rng.standard_normal((M, ncomp, N, N))
    u = scale * rng.standard_normal((M, ncomp, N, N))
    return t, u

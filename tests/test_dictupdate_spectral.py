"""The frequency-domain form of the filter-ADMM projection and dual update (Section IV-B, Eqs. g_admm
and h_admm), which the GPU filter update computes, against the oracle's spatial filter step (CPU).

The GPU keeps the scaled dual e only as its spectrum and the filters g only on their P x P support:
  w = F(d + e);  Y(a, k2) = sum_k1 w(k1, k2) exp(+2 pi i k1 a / N)            (support rows a)
  v(a, b) = N^-2 sum_k2 c_k2 Re[Y(a, k2) exp(+2 pi i k2 b / N)]                (c = 1 at k2 = 0, N/2)
  g = v / ||v||;  G(a, k2) = sum_b g(a, b) exp(-2 pi i k2 b / N)
  g-hat(k1, k2) = sum_a exp(-2 pi i k1 a / N) G(a, k2);  e-hat <- w - g-hat
with a, b the support offsets -P//2 .. P - 1 - P//2.  Written out here in NumPy from those formulas
(not from the library), it must reproduce the oracle's spatial step: v = Q^T (d + e), g, F g and
F e_new on the half spectrum."""
import numpy as np
import pytest

from oracle import admm as ref
from oracle import fast
from paper_2006_08303_gb300 import inputs


@pytest.mark.parametrize("N,P", [(32, 5), (32, 4), (64, 7)])
def test_support_partial_dfts_reproduce_the_spatial_projection(N, P):
    rng = np.random.default_rng(7 + N + P)
    L, M = 3, 2
    d0 = inputs.gabor_filters(rng, L, P)
    z = inputs.bernoulli_gaussian_codes(rng, L, M, N, 0.05)
    x = inputs.convdict_image(inputs.embed_filters(d0, N), z) + 0.01 * rng.standard_normal((M, N, N))
    g = ref.embed_filters(d0 + 0.1 * rng.standard_normal(d0.shape), N)
    e = 0.05 * rng.standard_normal((L, N, N))
    sigma = 3.0
    d, g_new, e_new = fast.dict_update(x, z, g, e, sigma, P)

    H = N // 2 + 1
    off = np.arange(P) - P // 2                                # support offsets
    k1 = np.arange(N)[:, None]
    k2 = np.arange(H)[None, :]
    w = np.fft.rfft2(d + e)                                    # [L, N, H]
    Y = np.einsum("lkh,ak->lah", w, np.exp(2j * np.pi * np.outer(off, np.arange(N)) / N))
    c = np.where((k2[0] == 0) | (k2[0] == N // 2), 1.0, 2.0)
    Eb = np.exp(2j * np.pi * np.outer(np.arange(H), off) / N)  # [H, P]: exp(+2 pi i k2 b / N)
    v = np.einsum("lah,h,hb->lab", Y, c, Eb).real / (N * N)    # [L, P, P]
    assert np.allclose(v, ref.crop_filters(d + e, P), atol=1e-12)

    gs = v / np.sqrt(np.sum(v * v, axis=(1, 2)))[:, None, None]
    assert np.allclose(gs, ref.crop_filters(g_new, P), atol=1e-12)
    G = np.einsum("lab,hb->lah", gs, np.conj(Eb))              # sum_b g(a, b) exp(-2 pi i k2 b / N)
    gh = np.einsum("ak,lah->lkh", np.exp(-2j * np.pi * np.outer(off, np.arange(N)) / N), G)
    assert np.allclose(gh, np.fft.rfft2(g_new), atol=1e-10)
    eh = w - gh
    assert np.allclose(eh, np.fft.rfft2(e_new), atol=1e-10)
    # the spectrum the next filter solve reads, F(g - e) = 2 g-hat - w
    assert np.allclose(2 * gh - w, np.fft.rfft2(g_new - e_new), atol=1e-10)
    # the primal residual of the sigma rule by Parseval on the half spectrum
    r2 = np.sum(c[None, None, :] * np.abs(np.fft.rfft2(d) - gh) ** 2) / (N * N)
    assert np.isclose(r2, np.sum((d - g_new) ** 2), rtol=1e-10)

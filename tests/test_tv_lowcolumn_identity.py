"""The identity behind the TV low-column correction of the x-update (CPU).

For a = (a_h, a_v) and the circular forward differences of reading R1, the transform of the
adjoint is F D^T a = conj(d_h) F a_h + conj(d_v) F a_v with d_h(k2) = exp(2 pi i k2 / N) - 1 along
the row frequency and d_v(k1) = exp(2 pi i k1 / N) - 1 along the column frequency.  For the two
lowest row frequencies the GPU forms the row DFTs of a_h and a_v by direct sums with table twiddles
(sum_c a[r, c] and sum_c a[r, c] exp(-2 pi i c / N)) and takes Q from the right-hand side, whose
rounding Psi^{-1} does not amplify near DC.  Checked here on random fields against the oracle's D^T
and NumPy's FFT, together with the direct sums."""
import numpy as np
import pytest

from oracle import admm as ref


@pytest.mark.parametrize("N", [16, 64])
def test_transform_of_the_tv_adjoint_is_the_weighted_sum_of_component_transforms(N):
    rng = np.random.default_rng(N)
    a = rng.standard_normal((2, N, N))
    lhs = np.fft.fft2(ref.tv_adjoint(a))
    k = np.arange(N)
    dh = np.exp(2j * np.pi * k / N) - 1.0            # along the last axis (row frequency k2)
    dv = np.exp(2j * np.pi * k / N) - 1.0            # along the first axis (column frequency k1)
    rhs = np.conj(dh)[None, :] * np.fft.fft2(a[0]) + np.conj(dv)[:, None] * np.fft.fft2(a[1])
    assert np.allclose(lhs, rhs, atol=1e-10 * np.abs(lhs).max())
    # and D is the adjoint of D^T (the same operators as the x-update's g = |d_h|^2 + |d_v|^2)
    x = rng.standard_normal((N, N))
    assert np.isclose(np.sum(ref.tv_forward(x) * a), np.sum(x * ref.tv_adjoint(a)))


@pytest.mark.parametrize("N", [32, 2048])
def test_low_row_frequencies_by_direct_sums(N):
    rng = np.random.default_rng(N + 1)
    rows = rng.standard_normal((4, N))
    c = np.arange(N)
    tw = np.exp(-2j * np.pi * c / N)                 # the table twiddle exp(-2 pi i c / N)
    s0 = rows.sum(axis=1)
    s1 = rows @ tw
    spec = np.fft.rfft(rows, axis=1)
    assert np.allclose(s0, spec[:, 0].real, atol=1e-9 * np.sqrt(N))
    assert np.allclose(s1, spec[:, 1], atol=1e-9 * np.sqrt(N))

"""Out-of-bounds writes into caller memory (a stand-in for compute-sanitizer, which this pool does
not offer): every entry point that writes a caller buffer gets a view into the middle of a larger
allocation filled with a guard value; after the call, the guard words before and after the view
must be untouched and the view itself must be overwritten.  GPU only."""
import numpy as np
import pytest

from paper_2006_08303_gb300 import inputs

pytestmark = pytest.mark.gpu

GUARD = 4096          # guard elements on each side
CANARY = 1234.5678


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    return torch


def guarded(torch, shape, dtype, fill=CANARY):
    n = int(np.prod(shape))
    buf = torch.full((n + 2 * GUARD,), fill, dtype=dtype, device="cuda")
    return buf, buf[GUARD:GUARD + n].view(*shape)


def check(torch, buf, n):
    torch.cuda.synchronize()
    h = buf.cpu().numpy()
    assert np.all(h[:GUARD] == CANARY), "write before the caller's buffer"
    assert np.all(h[GUARD + n:] == CANARY), "write after the caller's buffer"
    assert np.count_nonzero(h[GUARD:GUARD + n] == CANARY) < n, "buffer not written"


def analysis_plan(torch, prior, N, K, M, dtype="f32"):
    from paper_2006_08303_gb300 import api
    rng = np.random.default_rng(N + M)
    x = inputs.rectangles_image(rng, N, M, n_rect=4)
    h = inputs.gaussian_psf_bank(N, K, M)
    y, _ = inputs.measure(rng, x, h, 30.0)
    td = torch.float32 if dtype == "f32" else torch.float64
    P = api.Plan(N, K, M, dtype)
    P.set_prior(prior, 1e-2, 1.0, 1.0)
    P.set_psfs(torch.as_tensor(h, dtype=td).cuda())
    P.set_measurements(torch.as_tensor(y, dtype=td).cuda())
    P.iterate(3)
    return P, td


@pytest.mark.parametrize("prior,N,K,M,dtype", [("tv", 64, 3, 3, "f32"), ("dct8", 128, 2, 5, "f32"),
                                                ("tv_iso", 256, 2, 2, "f64"), ("l1", 2048, 1, 1, "f32")])
def test_reads_back_stay_inside_caller_buffers(torch, prior, N, K, M, dtype):
    P, td = analysis_plan(torch, prior, N, K, M, dtype)
    buf, view = guarded(torch, (M, N, N), td)
    P.get_x(view)
    check(torch, buf, M * N * N)
    shape = P.state_shape
    buf, view = guarded(torch, shape, td)
    P.get_u(view)
    check(torch, buf, int(np.prod(shape)))
    nbytes = P.state_size()
    buf, view = guarded(torch, (nbytes,), torch.uint8, fill=0xA5)
    P.state_export(view)
    torch.cuda.synchronize()
    h = buf.cpu().numpy()
    assert np.all(h[:GUARD] == 0xA5) and np.all(h[GUARD + nbytes:] == 0xA5)
    P.close()


def test_dictionary_reads_stay_inside_caller_buffers(torch):
    from paper_2006_08303_gb300 import api
    rng = np.random.default_rng(7)
    N, K, M, L, Pf = 64, 2, 2, 3, 5
    d = inputs.gabor_filters(rng, L, Pf)
    z = inputs.bernoulli_gaussian_codes(rng, L, M, N, 0.02)
    x = inputs.convdict_image(inputs.embed_filters(d, N), z)
    h = inputs.gaussian_psf_bank(N, K, M)
    y, _ = inputs.measure(rng, x, h, 25.0)
    f = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32).cuda()
    P = api.Plan(N, K, M, "f32")
    P.set_prior("convdict", 0.15, 8.0, 4.0)
    P.set_dictionary(f(d))
    P.set_psfs(f(h))
    P.set_measurements(f(y))
    P.iterate(4)
    buf, view = guarded(torch, (M, L, N, N), torch.float32)
    P.get_coefficients(view)
    check(torch, buf, M * L * N * N)
    buf, view = guarded(torch, (M, N, N), torch.float32)
    P.get_x(view)
    check(torch, buf, M * N * N)
    P.close()

"""The setup precision of complex64 plans where the per-frequency factor is worst conditioned.

Psi = rho g I + beta Lambda^H Lambda (Section IV-A) has condition number of order
1 + beta ||Lambda||^2 / rho for the DCT prior (g = 1) and of order K M / (rho (2 pi / N)^2) near
DC for TV.  complex64 plans form Lambda, Psi^{-1} and the data term in double-float (about 44
bits) and round them once; these tests run that path against the FP64 oracle where the factor is
least forgiving: the 512 x 512 x 10 spectral DCT instance across rho in {1, 1e-1, 1e-2, 1e-3}
(reading R7's sweep) and TV at 2048 x 2048 x 3.  Tolerances as everywhere: 1e-5 per step, 1e-4
on the free-running x.  The FP64 plan's error is computed beside each case and must stay at
FP64 level, so that a miss would point at the double-float setup, not at the model."""
import numpy as np
import pytest

from oracle import fast
from paper_2006_08303_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    return torch


def gpu_run(torch, pr, rho, iters, dtype, t0=None, u0=None):
    from paper_2006_08303_gb300 import api
    tdt = torch.float32 if dtype == "f32" else torch.float64
    f = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=tdt).cuda()
    P = api.Plan(pr.N, pr.K, pr.M, dtype)
    P.set_prior(pr.prior, pr.lam, rho, pr.beta)
    P.set_psfs(f(pr.h))
    P.set_measurements(f(pr.y))
    if t0 is not None:
        P.state_import(f(t0), f(u0))
    P.iterate(iters)
    x = P.get_x().double().cpu().numpy()
    P.close()
    return x


@pytest.mark.parametrize("rho", [1.0, 1e-1, 1e-2, 1e-3])
def test_dct_rho_sweep_512x512x10(torch, rho):
    pr = inputs.spectral_dct(iters=40)
    S = fast.analysis_setup(pr.h, pr.y, pr.prior, pr.lam, rho, pr.beta)
    t = np.zeros((pr.M, 1, pr.N, pr.N))
    u = np.zeros_like(t)
    step_err = []
    x_or = None
    for l in range(pr.iters):
        x_or, t1, u1, _ = fast.analysis_step(S, t, u)
        if l in (0, 20):
            xg = gpu_run(torch, pr, rho, 1, "f32", t, u)
            step_err.append(rel(xg, x_or))
        t, u = t1, u1
    final32 = rel(gpu_run(torch, pr, rho, pr.iters, "f32"), x_or)
    final64 = rel(gpu_run(torch, pr, rho, pr.iters, "f64"), x_or)
    print(f"rho={rho:g}: step {max(step_err):.2e}, final complex64 {final32:.2e}, final FP64 plan {final64:.2e}")
    assert max(step_err) <= 1e-5, step_err
    assert final32 <= 1e-4, final32
    assert final64 <= 1e-10, final64


def test_tv_2048x2048x3(torch):
    pr = inputs.tiny_tv(N=2048, M=3, iters=20, dtype="f32")
    S = fast.analysis_setup(pr.h, pr.y, pr.prior, pr.lam, pr.rho, pr.beta)
    t = np.zeros((pr.M, 2, pr.N, pr.N))
    u = np.zeros_like(t)
    step_err = None
    x_or = None
    for l in range(pr.iters):
        x_or, t1, u1, _ = fast.analysis_step(S, t, u)
        if l == 10:
            step_err = rel(gpu_run(torch, pr, pr.rho, 1, "f32", t, u), x_or)
        t, u = t1, u1
    final32 = rel(gpu_run(torch, pr, pr.rho, pr.iters, "f32"), x_or)
    final64 = rel(gpu_run(torch, pr, pr.rho, pr.iters, "f64"), x_or)
    print(f"TV 2048x2048x3: step {step_err:.2e}, final complex64 {final32:.2e}, final FP64 plan {final64:.2e}")
    assert step_err <= 1e-5, step_err
    assert final32 <= 1e-4, final32
    assert final64 <= 1e-10, final64

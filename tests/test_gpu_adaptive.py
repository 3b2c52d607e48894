"""Adaptive penalty (Section IV-C, Eq. paramS) on the GPU vs the FP64 oracle.  GPU only.

The oracle adapts rho after every check_every-th iteration, rescales the scaled dual and forms
the factor again (readings R17, R18); the library does the same at its residual checks.  The
runs start from a badly chosen rho so that rho changes several times; the final rho must be
the oracle's and the final x within the final-x tolerance."""
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


def run_gpu(torch, P, rho0, iters, dtype, check_every=10, adapt=True):
    from paper_2006_08303_gb300 import api
    td = torch.float32 if dtype == "f32" else torch.float64
    f = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=td).cuda()
    K, M, N = P.h.shape[0], P.h.shape[1], P.h.shape[-1]
    plan = api.Plan(N, K, M, dtype, check_every=check_every)
    plan.set_prior(P.prior, P.lam, rho0, P.beta)
    if adapt:
        plan.set_rho_adaptation(2.0, 10.0)
    plan.set_psfs(f(P.h))
    plan.set_measurements(f(P.y))
    plan.iterate(iters)
    x = plan.get_x().double().cpu().numpy()
    rho = plan.rho
    plan.close()
    return x, rho


@pytest.mark.parametrize("dtype,tol", [("f32", 1e-4), ("f64", 1e-9)])
def test_adaptive_tv_tiny(torch, dtype, tol):
    P = inputs.tiny_tv(dtype="f64")
    rho0, iters = 64.0, 80
    x_ref, _, _, rhos, _ = fast.run_analysis_adaptive(P.h, P.y, P.prior, P.lam, rho0, P.beta, iters, 10)
    assert len(set(rhos)) > 2
    x, rho = run_gpu(torch, P, rho0, iters, dtype)
    assert rho == rhos[-1], (rho, rhos[-1])
    assert rel(x, x_ref) <= tol, rel(x, x_ref)


def test_adaptive_dct_moves_rho_up(torch):
    P = inputs.spectral_dct(N=128, M=3, iters=60)
    rho0 = 1e-4
    x_ref, _, _, rhos, _ = fast.run_analysis_adaptive(P.h, P.y, P.prior, P.lam, rho0, P.beta, 60, 10)
    assert rhos[-1] > rho0
    x, rho = run_gpu(torch, P, rho0, 60, "f32")
    assert rho == rhos[-1], (rho, rhos[-1])
    assert rel(x, x_ref) <= 1e-4, rel(x, x_ref)


def test_adaptation_must_precede_measurements(torch):
    from paper_2006_08303_gb300 import api
    P = inputs.tiny_tv(dtype="f64")
    f = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32).cuda()
    K, M, N = P.h.shape[0], P.h.shape[1], P.h.shape[-1]
    plan = api.Plan(N, K, M, "f32")
    plan.set_prior(P.prior, P.lam, P.rho, P.beta)
    plan.set_psfs(f(P.h))
    plan.set_measurements(f(P.y))
    with pytest.raises(Exception):
        plan.set_rho_adaptation(2.0, 10.0)
    plan.set_rho_adaptation(0.0, 0.0)  # turning it off is always allowed
    plan.close()

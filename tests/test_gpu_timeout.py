"""The bounded device wait and its error path (CIP_ERR_TIMEOUT), exercised without a GPU fault.

The prior pass stages the u rows of its tile in shared memory with one bulk copy completed on an
mbarrier, and waits for it with a bounded wait.  cip_set_test_fault(plan, 1) makes that barrier
one that can never complete (two arrivals expected, one given, no copy issued) and caps the wait
at 64 polls, so the wait gives up with nothing in flight.  The kernel then reads u from global
memory, so the iterate is unchanged, and flags the plan: cip_get_residuals and the residual checks
of cip_iterate report CIP_ERR_TIMEOUT until the next state reset.
"""
import numpy as np
import pytest

from paper_2006_08303_gb300 import inputs

CIP_ERR_TIMEOUT = 6


def _plan(api, torch, P, **kw):
    f = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32).cuda()
    plan = api.Plan(P.N, P.K, P.M, "f32", **kw)
    plan.set_prior(P.prior, P.lam, P.rho, P.beta)
    plan.set_psfs(f(P.h))
    plan.set_measurements(f(P.y))
    return plan


@pytest.mark.gpu
def test_timeout_is_reported_and_the_context_stays_usable():
    import torch
    from paper_2006_08303_gb300 import api
    P = inputs.spectral_dct(N=64, M=3, iters=3)
    ref = _plan(api, torch, P)
    ref.iterate(3)
    x_ok = ref.get_x().cpu().numpy()
    ref.residuals()  # no fault: the residuals are available
    ref.close()

    bad = _plan(api, torch, P)
    bad.set_test_fault(1)
    bad.iterate(3)
    torch.cuda.synchronize()
    with pytest.raises(api.CipError) as ei:
        bad.residuals()
    assert ei.value.status == CIP_ERR_TIMEOUT
    # the kernel gave up the wait and read u from global memory: the iterate is the same
    assert np.array_equal(bad.get_x().cpu().numpy(), x_ok)
    # with a tolerance the residual check of cip_iterate reports the timeout itself
    bad.reset_state()
    with pytest.raises(api.CipError) as ei:
        bad.iterate(20, tol=1e-12)
    assert ei.value.status == CIP_ERR_TIMEOUT
    # switched off and reset, the same plan runs cleanly again
    bad.set_test_fault(0)
    bad.reset_state()
    bad.iterate(3)
    bad.residuals()
    assert np.array_equal(bad.get_x().cpu().numpy(), x_ok)
    bad.close()

    # and so does a new plan on the same device
    fresh = _plan(api, torch, P)
    fresh.iterate(3)
    fresh.residuals()
    assert np.array_equal(fresh.get_x().cpu().numpy(), x_ok)
    fresh.close()


def test_test_fault_rejects_unknown_kinds():
    """Host-side argument check (no GPU work): only kinds 0 and 1 exist."""
    from paper_2006_08303_gb300 import _lib
    import ctypes
    L = _lib.load()
    assert L.cip_set_test_fault(None, 1) == 1  # CIP_ERR_INVALID_ARG for a null plan

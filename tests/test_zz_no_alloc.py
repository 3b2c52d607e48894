"""cip_shrink_dual_noalloc -- the entry point for callers that cannot allocate
device memory (inside a stream capture, a fixed framework arena, a real-time
loop) -- gives the same u-update and residuals as the plan's own prior pass in
cip_iterate, on two calls in a row.  Its scratch is a static device array, so
the second call also checks that state left by the first call does not leak
into the result.  GPU only; collected last on purpose."""
import numpy as np
import pytest

from oracle import fast
from paper_2006_08303_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("prior", ["tv", "dct8"])
def test_noalloc_matches_iterate_on_two_calls(prior):
    import torch
    from paper_2006_08303_gb300 import api

    if prior == "tv":
        Pr = inputs.tiny_tv(N=128, M=3)
    else:
        Pr = inputs.spectral_dct(N=128, M=4)
    nc = 2 if prior == "tv" else 1
    f = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32).cuda()
    # an ADMM state a few iterations in, from the oracle
    S = fast.analysis_setup(Pr.h, Pr.y, Pr.prior, Pr.lam, Pr.rho, Pr.beta)
    t = np.zeros((Pr.M, nc, Pr.N, Pr.N))
    u = np.zeros_like(t)
    for _ in range(3):
        _, t, u, _ = fast.analysis_step(S, t, u)

    plan = api.Plan(Pr.N, Pr.K, Pr.M, "f32")
    plan.set_prior(Pr.prior, Pr.lam, Pr.rho, Pr.beta)
    plan.set_psfs(f(Pr.h))
    plan.set_measurements(f(Pr.y))
    plan.state_import(f(t), f(u))

    u_prev, t_prev = f(u), f(t)
    u_out = torch.empty_like(u_prev)
    t_out = torch.empty_like(t_prev)
    for call in range(2):
        plan.iterate(1)
        x = plan.get_x()
        u_ref = plan.get_u().cpu().numpy()
        r_ref, s_ref = plan.residuals()
        resid = np.zeros(2, dtype=np.float64)
        api.shrink_dual_noalloc(prior, Pr.lam, Pr.rho, x, u_prev, t_prev, u_out, resid, t_out=t_out)
        torch.cuda.synchronize()
        ug = u_out.cpu().numpy()
        assert rel(ug, u_ref) <= 1e-5, (call, rel(ug, u_ref))
        assert abs(resid[0] - r_ref) <= 1e-5 * r_ref, (call, resid[0], r_ref)
        assert abs(resid[1] - s_ref) <= 1e-5 * s_ref, (call, resid[1], s_ref)
        # device-pointer output for the residuals as well
        resid_dev = torch.zeros(2, dtype=torch.float64, device="cuda")
        api.shrink_dual_noalloc(prior, Pr.lam, Pr.rho, x, u_prev, t_prev, torch.empty_like(u_prev), resid_dev)
        assert np.allclose(resid_dev.cpu().numpy(), resid, rtol=0, atol=0)
        u_prev, t_prev = u_out.clone(), t_out.clone()
    plan.close()

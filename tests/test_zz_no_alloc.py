"""cip_shrink_dual_noalloc -- the entry point for callers that cannot allocate device memory (code
recording a stream capture that must not gain allocation nodes, a framework's fixed memory arena,
a real-time loop) -- checked three ways, each on two calls in a row (its scratch is a static device
array, so the second call also shows that the first call's leftovers do not leak into the result):

  * against the FP64 oracle's t/u update and residuals on the same inputs,
  * against the plan's own prior pass inside cip_iterate,
  * recorded into a CUDA graph by a stream capture and replayed, against the uncaptured call,
    with the device's free memory and torch's allocation count unchanged across the calls.

GPU only; collected last on purpose."""
import numpy as np
import pytest

from oracle import admm as ref
from oracle import fast
from paper_2006_08303_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _problem(prior):
    if prior == "tv":
        return inputs.tiny_tv(N=128, M=3)
    Pr = inputs.spectral_dct(N=128, M=4)
    Pr.prior = prior
    return Pr


def _oracle_state(Pr, iters=3):
    """An ADMM state a few iterations in, from the oracle."""
    nc = ref.ncomp_of(Pr.prior)
    S = fast.analysis_setup(Pr.h, Pr.y, Pr.prior, Pr.lam, Pr.rho, Pr.beta)
    t = np.zeros((Pr.M, nc, Pr.N, Pr.N))
    u = np.zeros_like(t)
    for _ in range(iters):
        _, t, u, _ = fast.analysis_step(S, t, u)
    return S, t, u


def _oracle_tu(prior, lam, rho, x, u, t_prev):
    """t/u update and relative residuals of Eqs. solt_trans, subu_trans and paramS (reading R11),
    in FP64 from the same inputs the GPU call gets."""
    fwd, _ = ref.PRIORS[prior]
    w = fwd(x)
    t = ref.shrink(prior, w + u, lam / rho)
    un = u + w - t
    r = np.linalg.norm(w - t) / max(np.linalg.norm(w), np.linalg.norm(t))
    s = rho * np.linalg.norm(t - t_prev) / (rho * np.linalg.norm(un))
    return w, t, un, r, s


@pytest.mark.parametrize("prior", ["tv", "dct8", "l1"])
def test_noalloc_matches_oracle_and_iterate_on_two_calls(prior):
    import torch
    from paper_2006_08303_gb300 import api

    Pr = _problem(prior)
    f = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32).cuda()
    S, t, u = _oracle_state(Pr)

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
        ug, tg = u_out.cpu().numpy(), t_out.cpu().numpy()
        # the FP64 oracle on the same (float32) inputs; u at the scale of Tx it is computed at (R15)
        w_or, t_or, u_or, r_or, s_or = _oracle_tu(prior, Pr.lam, Pr.rho, x.double().cpu().numpy(),
                                                  u_prev.double().cpu().numpy(), t_prev.double().cpu().numpy())
        scale = max(np.linalg.norm(u_or), np.linalg.norm(w_or))
        assert np.linalg.norm(ug - u_or) <= 1e-5 * scale, (call, np.linalg.norm(ug - u_or) / scale)
        assert np.linalg.norm(tg - t_or) <= 1e-5 * scale, (call, np.linalg.norm(tg - t_or) / scale)
        assert abs(resid[0] - r_or) <= 1e-5 * r_or + 1e-7, (call, resid[0], r_or)
        assert abs(resid[1] - s_or) <= 1e-5 * s_or + 1e-6, (call, resid[1], s_or)
        # and the plan's own prior pass in cip_iterate
        assert rel(ug, u_ref) <= 1e-5, (call, rel(ug, u_ref))
        assert abs(resid[0] - r_ref) <= 1e-5 * r_ref, (call, resid[0], r_ref)
        assert abs(resid[1] - s_ref) <= 1e-5 * s_ref, (call, resid[1], s_ref)
        # device-pointer output for the residuals as well
        resid_dev = torch.zeros(2, dtype=torch.float64, device="cuda")
        api.shrink_dual_noalloc(prior, Pr.lam, Pr.rho, x, u_prev, t_prev, torch.empty_like(u_prev), resid_dev)
        assert np.allclose(resid_dev.cpu().numpy(), resid, rtol=0, atol=0)
        u_prev, t_prev = u_out.clone(), t_out.clone()
    plan.close()


@pytest.mark.parametrize("prior", ["tv", "dct8"])
def test_noalloc_under_stream_capture_allocates_nothing(prior):
    import torch
    from paper_2006_08303_gb300 import api

    Pr = _problem(prior)
    f = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32).cuda()
    S, t, u = _oracle_state(Pr)
    x = f(fast.x_update(S, t, u))
    u_in, t_prev = f(u), f(t)
    u_a, t_a = torch.empty_like(u_in), torch.empty_like(t_prev)
    u_b, t_b = torch.empty_like(u_in), torch.empty_like(t_prev)
    r_a = torch.zeros(2, dtype=torch.float64, device="cuda")
    r_b = torch.zeros(2, dtype=torch.float64, device="cuda")
    host = np.zeros(2, dtype=np.float64)

    # first call on this device outside any capture (it looks up the scratch array's address)
    api.shrink_dual_noalloc(prior, Pr.lam, Pr.rho, x, u_in, t_prev, u_a, r_a, t_out=t_a)
    torch.cuda.synchronize()

    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side, capture_error_mode="thread_local"):
            api.shrink_dual_noalloc(prior, Pr.lam, Pr.rho, x, u_in, t_prev, u_b, r_b, t_out=t_b, stream=side)
            # a host output cannot be captured: refused with CIP_ERR_INVALID_ARG, capture intact
            with pytest.raises(api.CipError) as ei:
                api.shrink_dual_noalloc(prior, Pr.lam, Pr.rho, x, u_in, t_prev, u_b, host, t_out=t_b, stream=side)
            assert ei.value.status == 1
    torch.cuda.current_stream().wait_stream(side)
    for _ in range(2):  # two replays in a row
        u_b.zero_()
        r_b.zero_()
        torch.cuda.synchronize()
        free_r0, _ = torch.cuda.mem_get_info()
        g.replay()
        torch.cuda.synchronize()
        free_r1, _ = torch.cuda.mem_get_info()
        assert free_r1 == free_r0, (free_r0, free_r1)
        assert torch.equal(u_b, u_a) and torch.equal(t_b, t_a)
        assert torch.equal(r_b, r_a)
    # and two more plain calls: nothing allocated by the library at any point (measured around the
    # library calls alone, with no torch operation in between)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(2):
        api.shrink_dual_noalloc(prior, Pr.lam, Pr.rho, x, u_in, t_prev, u_b, r_b, t_out=t_b)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() == alloc0
    assert free1 == free0, (free0, free1)
    assert torch.equal(u_b, u_a) and torch.equal(r_b, r_a)
    del g

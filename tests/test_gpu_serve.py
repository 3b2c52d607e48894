"""Request server (continuous batching, admission by device-memory budget).  GPU only.

Each served result must equal the same reconstruction run alone through the plan API
(same kernels, same check points), whatever else shares the device."""
import time

import numpy as np
import pytest

from paper_2006_08303_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    return torch


def make_req(seed, N, M, prior, K=None):
    rng = np.random.default_rng(seed)
    x = inputs.rectangles_image(rng, N, M, n_rect=5)
    h = inputs.gaussian_psf_bank(N, M if K is None else K, M)
    y, _ = inputs.measure(rng, x, h, 30.0)
    lam, rho = (1e-2, 1.0) if prior != "dct8" else (1e-3, 0.1)
    return h.astype(np.float32), y.astype(np.float32), prior, lam, rho


def alone(torch, h, y, prior, lam, rho, tol, max_iter):
    from paper_2006_08303_gb300 import api
    K, M, N = h.shape[0], h.shape[1], h.shape[-1]
    P = api.Plan(N, K, M, "f32", check_every=10)
    P.set_prior(prior, lam, rho, 1.0)
    P.set_psfs(h)
    P.set_measurements(y)
    n = P.iterate(max_iter, tol)
    x = np.empty((M, N, N), np.float32)
    P.get_x(x)
    P.close()
    return x, n


MIX = [(64, 3, "tv"), (128, 2, "dct8"), (256, 3, "tv"), (64, 5, "l1"), (128, 3, "tv"), (256, 2, "dct8"),
       (64, 2, "tv"), (128, 5, "l1")]


def test_served_results_equal_alone(torch):
    from paper_2006_08303_gb300 import api
    S = api.Server(hbm_budget=8 << 30, max_active=3, check_every=10)
    reqs = [make_req(i, *c) for i, c in enumerate(MIX)]
    ids = []
    for i, (h, y, prior, lam, rho) in enumerate(reqs):
        ids.append(S.submit(h, y, prior, lam, rho, tol=1e-3, max_iter=200))
        if i == 3:
            time.sleep(0.05)  # later requests arrive while the first ones run
    results = [S.wait(rid) for rid, _ in ids]
    S.close()
    # continuous batching: requests were in flight on the device at the same time (one admitted
    # while another was still running), not served one after another
    overlaps = sum(1 for a in results for b in results
                   if a is not b and a["t_admit"] < b["t_done"] and b["t_admit"] < a["t_done"])
    assert overlaps > 0, [(r["t_admit"], r["t_done"]) for r in results]
    for (rid, x_out), res, (h, y, prior, lam, rho) in zip(ids, results, reqs):
        assert res["state"] == "done", res
        assert res["t_submit"] <= res["t_admit"] <= res["t_done"]
        x_alone, n_alone = alone(torch, h, y, prior, lam, rho, 1e-3, 200)
        assert res["iterations"] == n_alone
        assert np.array_equal(x_out, x_alone)


def test_budget_limits_admission_and_all_finish(torch):
    from paper_2006_08303_gb300 import api
    one = api.plan_bytes(256, 3, 3, "f32", "tv")
    S = api.Server(hbm_budget=int(1.5 * one), max_active=8)
    ids = [S.submit(*make_req(10 + i, 256, 3, "tv"), max_iter=40)[0] for i in range(5)]
    peak = 0
    while True:
        st = S.stats()
        peak = max(peak, st["running"])
        assert st["bytes_in_use"] <= int(1.5 * one)
        if all(S.poll(r)["state"] in ("done", "failed") for r in ids):
            break
        time.sleep(0.002)
    assert peak <= 1
    assert all(S.poll(r)["state"] == "done" for r in ids)
    S.close()


def test_cancel_and_failure_do_not_disturb_others(torch):
    from paper_2006_08303_gb300 import api
    S = api.Server(hbm_budget=8 << 30, max_active=1)
    a = S.submit(*make_req(1, 128, 3, "tv"), max_iter=100)[0]
    h, y, prior, lam, rho = make_req(2, 128, 3, "tv")
    bad = S.submit(h, y, prior, -1.0, rho, max_iter=50)[0]        # invalid lambda: fails at setup
    c = S.submit(*make_req(3, 128, 3, "tv"), max_iter=100)[0]
    S.cancel(c)                                                   # cancelled while queued
    d = S.submit(*make_req(4, 64, 2, "dct8"), max_iter=30)[0]
    ra, rb, rc, rd = S.wait(a), S.wait(bad), S.wait(c), S.wait(d)
    assert ra["state"] == "done" and rd["state"] == "done"
    assert rb["state"] == "failed" and rb["status"] != 0
    assert rc["state"] == "cancelled"
    S.close()


def test_factor_cache_shared_between_requests(torch):
    from paper_2006_08303_gb300 import api
    S = api.Server(hbm_budget=8 << 30, max_active=4)
    base = make_req(5, 128, 3, "tv")
    rng = np.random.default_rng(9)
    outs = []
    for i in range(3):
        h, y, prior, lam, rho = base
        y2 = (y + 0.01 * rng.standard_normal(y.shape)).astype(np.float32)
        rid, x = S.submit(h, y2, prior, lam, rho, max_iter=60, psf_key=77)
        outs.append((rid, x, y2))
    for rid, x, y2 in outs:
        assert S.wait(rid)["state"] == "done"
    st = S.stats()
    assert st["cache_hits"] >= 2 and st["cache_misses"] == 1
    h, _, prior, lam, rho = base
    for rid, x, y2 in outs:
        x_alone, _ = alone(torch, h, y2, prior, lam, rho, 0.0, 60)
        assert np.array_equal(x, x_alone)
    S.close()


def test_oversize_request_is_rejected(torch):
    from paper_2006_08303_gb300 import api
    S = api.Server(hbm_budget=1 << 20, max_active=2)
    with pytest.raises(api.CipError):
        S.submit(*make_req(6, 256, 3, "tv"))
    S.close()


def test_served_k_differs_from_m(torch):
    """Requests with K != M (one frame of three channels, four frames of two channels, four
    frames of one image: multiframe deconvolution) are served alongside K = M ones, each result
    equal to the plan run alone, and isotropic TV is served like the other analysis priors."""
    from paper_2006_08303_gb300 import api
    S = api.Server(hbm_budget=8 << 30, max_active=3, check_every=10)
    cases = [(128, 3, "tv", 1), (64, 2, "dct8", 4), (128, 1, "tv_iso", 4), (64, 3, "tv", 3)]
    reqs = [make_req(40 + i, N, M, prior, K) for i, (N, M, prior, K) in enumerate(cases)]
    ids = [S.submit(h, y, prior, lam, rho, tol=1e-3, max_iter=150) for (h, y, prior, lam, rho) in reqs]
    results = [S.wait(rid) for rid, _ in ids]
    S.close()
    # continuous batching: requests were in flight on the device at the same time (one admitted
    # while another was still running), not served one after another
    overlaps = sum(1 for a in results for b in results
                   if a is not b and a["t_admit"] < b["t_done"] and b["t_admit"] < a["t_done"])
    assert overlaps > 0, [(r["t_admit"], r["t_done"]) for r in results]
    for (rid, x_out), res, (h, y, prior, lam, rho) in zip(ids, results, reqs):
        assert res["state"] == "done", res
        x_alone, n_alone = alone(torch, h, y, prior, lam, rho, 1e-3, 150)
        assert res["iterations"] == n_alone
        assert np.array_equal(x_out, x_alone)


def test_served_wavelet_prior_and_adaptive_penalty(torch):
    """The Kronecker wavelet (x) DCT prior and the adaptive penalty of Eq. paramS are served like
    the other requests: each result equals the same reconstruction through the plan API (the
    adaptive one with cip_set_rho_adaptation, whose rho changes at the same checks), also when
    it shares the device with other requests."""
    from paper_2006_08303_gb300 import api
    S = api.Server(hbm_budget=8 << 30, max_active=4, check_every=10)
    wd = make_req(51, 128, 3, "tv")
    wd = (wd[0], wd[1], "wdct", 1e-2, 0.5)
    ad = make_req(52, 128, 3, "tv")
    ad = (ad[0], ad[1], "tv", 1e-2, 16.0)  # rho far from its adapted value: it changes several times
    other = make_req(53, 256, 3, "dct8")
    ids = [S.submit(*wd, tol=1e-4, max_iter=150),
           S.submit(*ad, tol=1e-4, max_iter=300, rho_tau=2.0, rho_mu=10.0, psf_key=7),
           S.submit(*other, tol=1e-3, max_iter=100)]
    res = [S.wait(rid) for rid, _ in ids]
    S.close()
    assert all(r["state"] == "done" for r in res), res
    x_w, n_w = alone(torch, *wd, 1e-4, 150)
    assert res[0]["iterations"] == n_w and np.array_equal(ids[0][1], x_w)
    P = api.Plan(128, 3, 3, "f32", check_every=10)
    P.set_prior("tv", 1e-2, 16.0, 1.0)
    P.set_rho_adaptation(2.0, 10.0)
    P.set_psfs(ad[0])
    P.set_measurements(ad[1])
    n_a = P.iterate(300, 1e-4)
    assert P.rho != 16.0  # the penalty did adapt
    x_a = np.empty((3, 128, 128), np.float32)
    P.get_x(x_a)
    P.close()
    assert res[1]["iterations"] == n_a and np.array_equal(ids[1][1], x_a)
    with pytest.raises(api.CipError):
        S2 = api.Server(hbm_budget=1 << 30)
        try:
            S2.submit(*ad, rho_tau=0.5, rho_mu=10.0)
        finally:
            S2.close()

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

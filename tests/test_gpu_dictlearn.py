"""Online convolutional dictionary update (Section IV-B, Eqs. d_admm, g_admm, h_admm, sold_3D)
of the CUDA library vs the FP64 oracle.  GPU only.

Alg. 2 with one filter-ADMM step after every z-update (reading R21) runs free from
z = t = u = 0, g = d0, e = 0 on both sides; x, the coefficient maps z and the learnt filters
are compared at relative L2 <= 1e-5 after one iteration and <= 1e-4 after the stated run
(complex64 path), 1e-9 on the FP64 path."""
import numpy as np
import pytest

from oracle import fast
from paper_2006_08303_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def gl(a):
    """oracle layout [L][M][N][N] -> library layout [M][L][N][N]"""
    return np.ascontiguousarray(np.transpose(a, (1, 0, 2, 3)))


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    return torch


def problem(seed=31, N=64, K=2, M=3, L=4, Pf=5):
    rng = np.random.default_rng(seed)
    d = inputs.gabor_filters(rng, L, Pf)
    z = inputs.bernoulli_gaussian_codes(rng, L, M, N, 0.02)
    x = inputs.convdict_image(inputs.embed_filters(d, N), z)
    h = inputs.gaussian_psf_bank(N, K, M)
    y, _ = inputs.measure(rng, x, h, 25.0)
    # start the learning from perturbed filters so that the update has work to do
    d0 = d + 0.3 * rng.standard_normal(d.shape) * np.abs(d).max()
    return h, y, d0


def learning_plan(torch, h, y, d, lam, rho, beta, sigma, dtype="f32", check_every=0):
    from paper_2006_08303_gb300 import api
    K, M, N, _ = h.shape
    f = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32 if dtype == "f32" else torch.float64).cuda()
    P = api.Plan(N, K, M, dtype, check_every=check_every)
    P.set_prior("convdict", lam, rho, beta)
    P.set_dictionary(f(d))
    P.set_dictionary_learning(sigma)
    P.set_psfs(f(h))
    P.set_measurements(f(y))
    return P, f


LAM, RHO, BETA = 0.15, 8.0, 4.0


@pytest.mark.parametrize("dtype,iters,tol", [("f32", 1, 1e-5), ("f32", 2, 1e-5), ("f32", 25, 1e-4),
                                             ("f64", 1, 1e-10), ("f64", 25, 1e-9)])
@pytest.mark.parametrize("sigma", [2.0, 10.0])
def test_learning_parity_small(torch, dtype, iters, tol, sigma):
    h, y, d0 = problem()
    x_or, z_or, _, u_or, f_or = fast.run_convdict_learn(h, y, d0, LAM, RHO, BETA, sigma, iters)
    P, _ = learning_plan(torch, h, y, d0, LAM, RHO, BETA, sigma, dtype)
    P.iterate(iters)
    xg = P.get_x().double().cpu().numpy()
    zg = P.get_coefficients().double().cpu().numpy()
    fg = P.get_dictionary().double().cpu().numpy()
    P.close()
    assert rel(fg, f_or) <= tol, rel(fg, f_or)
    assert rel(xg, x_or) <= tol, rel(xg, x_or)
    assert rel(zg, gl(z_or)) <= tol, rel(zg, gl(z_or))
    # the learnt filters lie in the constraint set of Eq. Constrained2 (unit norm)
    assert np.allclose(np.linalg.norm(fg.reshape(fg.shape[0], -1), axis=1), 1.0, atol=1e-5)


@pytest.mark.parametrize("N,K,M,L,Pf,dtype,tol", [(128, 3, 5, 7, 7, "f32", 1e-4), (64, 2, 8, 3, 3, "f32", 1e-4),
                                                  (64, 2, 8, 3, 3, "f64", 1e-9), (64, 1, 1, 5, 4, "f32", 1e-4)])
def test_learning_parity_channel_counts(torch, N, K, M, L, Pf, dtype, tol):
    """Channel counts 1, 5 and 8 (each its own register-resident M x M solve), odd and even
    filter sizes, 12 iterations."""
    h, y, d0 = problem(seed=8, N=N, K=K, M=M, L=L, Pf=Pf)
    sigma, iters = 5.0, 12
    x_or, z_or, _, _, f_or = fast.run_convdict_learn(h, y, d0, LAM, RHO, BETA, sigma, iters)
    P, _ = learning_plan(torch, h, y, d0, LAM, RHO, BETA, sigma, dtype)
    P.iterate(iters)
    xg = P.get_x().double().cpu().numpy()
    fg = P.get_dictionary().double().cpu().numpy()
    P.close()
    assert rel(fg, f_or) <= tol, rel(fg, f_or)
    assert rel(xg, x_or) <= tol, rel(xg, x_or)


def test_learning_full_size(torch):
    """The benchmark's dictionary workload: N = 256, M = K = 5, L = 32 Gabor filters of 11 x 11
    (every lane of the per-bin warp a filter), sigma = 10, 5 iterations."""
    pr = inputs.convdict_problem()
    sigma, iters = 10.0, 5
    x_or, _, _, _, f_or = fast.run_convdict_learn(pr.h, pr.y, pr.filters, pr.lam, pr.rho, pr.beta, sigma, iters)
    P, _ = learning_plan(torch, pr.h, pr.y, pr.filters, pr.lam, pr.rho, pr.beta, sigma)
    P.iterate(iters)
    xg = P.get_x().double().cpu().numpy()
    fg = P.get_dictionary().double().cpu().numpy()
    P.close()
    assert rel(fg, f_or) <= 1e-4, rel(fg, f_or)
    assert rel(xg, x_or) <= 1e-4, rel(xg, x_or)


def test_learning_split_calls_and_checkpoint(torch):
    """Iterations split over calls give the same iterates; the exported state carries the
    filters and their dual, so a restore replays bit for bit."""
    h, y, d0 = problem(seed=4)
    P, _ = learning_plan(torch, h, y, d0, LAM, RHO, BETA, 3.0)
    P.iterate(3)
    P.iterate(4)
    ck = P.state_export()
    P.iterate(5)
    xa = P.get_x().cpu().numpy()
    fa = P.get_dictionary().cpu().numpy()
    P.state_restore(ck)
    P.iterate(5)
    xb = P.get_x().cpu().numpy()
    fb = P.get_dictionary().cpu().numpy()
    P.close()
    assert np.array_equal(xa, xb) and np.array_equal(fa, fb)
    x_or, _, _, _, f_or = fast.run_convdict_learn(h, y, d0, LAM, RHO, BETA, 3.0, 12)
    assert rel(fa, f_or) <= 1e-4 and rel(xa, x_or) <= 1e-4


def test_learning_off_and_rejections(torch):
    from paper_2006_08303_gb300 import api
    h, y, d0 = problem(seed=6)
    P, f = learning_plan(torch, h, y, d0, LAM, RHO, BETA, 2.0)
    P.iterate(3)
    P.set_dictionary_learning(0.0)
    with pytest.raises(api.CipError):
        P.get_dictionary()
    with pytest.raises(api.CipError):
        P.set_dictionary_learning(-1.0)
    P.close()
    # off from the start: plain Alg. 2
    Q, _ = learning_plan(torch, h, y, d0, LAM, RHO, BETA, 0.0)
    Q.iterate(5)
    x_plain = Q.get_x().double().cpu().numpy()
    Q.close()
    C = fast.convdict_setup(h, y, d0, LAM, RHO, BETA)
    x_or = fast.run_convdict(C, 5)[0]
    assert rel(x_plain, x_or) <= 1e-5
    # analysis plans and M > 8 channels are rejected
    A = api.Plan(64, 1, 1, "f32")
    A.set_prior("tv", 0.1, 1.0, 1.0)
    with pytest.raises(api.CipError):
        A.set_dictionary_learning(1.0)
    A.close()
    B = api.Plan(64, 1, 9, "f32")
    B.set_prior("convdict", LAM, RHO, BETA)
    B.set_dictionary(f(d0))
    with pytest.raises(api.CipError):
        B.set_dictionary_learning(1.0)
    B.close()


@pytest.mark.parametrize("sigma0,dtype,tol", [(0.05, "f32", 1e-4), (500.0, "f32", 1e-4), (500.0, "f64", 1e-9)])
def test_sigma_adaptation_matches_oracle(torch, sigma0, dtype, tol):
    """Adaptation of sigma by the rule of Eq. paramS (reading R29), checked every 5 filter steps:
    the sigma trajectory equals the oracle's (run_convdict_learn with check_every), rising from
    0.05 or falling from 500 several times in 30 iterations; x, z and the filters agree; a
    checkpoint carries the adapted sigma and replays bit for bit."""
    h, y, d0 = problem()
    iters, ce = 30, 5
    x_or, z_or, _, _, f_or, sig_or = fast.run_convdict_learn(h, y, d0, LAM, RHO, BETA, sigma0, iters, check_every=ce)
    assert len(set(sig_or)) >= 4  # the schedule changes sigma several times
    P, _ = learning_plan(torch, h, y, d0, LAM, RHO, BETA, sigma0, dtype, check_every=ce)
    P.set_sigma_adaptation(2.0, 10.0)
    sig, ck, ck_sigma = [], None, None
    for it in range(iters):
        P.iterate(1)
        sig.append(P.sigma)
        if it == 11:
            ck, ck_sigma = P.state_export(), P.sigma
    assert sig == sig_or, (sig, sig_or)
    xg = P.get_x().double().cpu().numpy()
    zg = P.get_coefficients().double().cpu().numpy()
    fg = P.get_dictionary().double().cpu().numpy()
    assert rel(fg, f_or) <= tol, rel(fg, f_or)
    assert rel(xg, x_or) <= tol, rel(xg, x_or)
    assert rel(zg, gl(z_or)) <= tol, rel(zg, gl(z_or))
    xa, fa = P.get_x().cpu().numpy(), P.get_dictionary().cpu().numpy()
    P.set_dictionary_learning(sigma0 * 3)  # a different sigma, replaced by the checkpoint's
    P.state_restore(ck)
    assert P.sigma == ck_sigma
    for _ in range(iters - 12):
        P.iterate(1)
    assert P.sigma == sig_or[-1]
    assert np.array_equal(P.get_x().cpu().numpy(), xa) and np.array_equal(P.get_dictionary().cpu().numpy(), fa)
    with pytest.raises(Exception):
        P.set_sigma_adaptation(0.5, 10.0)
    P.close()


def test_filter_update_is_three_launches(torch):
    """One step of the filter ADMM adds exactly three kernel launches to an iteration (filter
    solve with the partial inverse DFT at the support rows; projection; spectra, dual and p)."""
    h, y, d0 = problem(seed=12)
    counts = []
    for sigma in (0.0, 4.0):
        P, _ = learning_plan(torch, h, y, d0, LAM, RHO, BETA, sigma)
        P.iterate(2)
        n0 = P.launches()
        P.iterate(6)
        counts.append(P.launches() - n0)
        P.close()
    assert counts[1] - counts[0] == 3 * 6, counts

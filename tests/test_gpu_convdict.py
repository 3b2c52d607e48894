"""Convolutional-dictionary path (Alg. 2) of the CUDA library vs the FP64 oracle.  GPU only.

One GPU iteration from the oracle's (z^l, t^l, u^l) is compared with the oracle's iteration
l+1 (x: Eq. solx_synt_DFT; z: Eqs. solz_DFT, solz_DFT_SM; u: Eqs. softADMM, subu_dic) at relative
L2 <= 1e-5, and the free-running x after the stated iterations at <= 1e-4."""
import numpy as np
import pytest

from oracle import admm, fast
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


def plan_for(torch, h, y, d, lam, rho, beta, dtype="f32"):
    from paper_2006_08303_gb300 import api
    K, M, N, _ = h.shape
    f = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32 if dtype == "f32" else torch.float64).cuda()
    P = api.Plan(N, K, M, dtype)
    P.set_prior("convdict", lam, rho, beta)
    P.set_dictionary(f(d))
    P.set_psfs(f(h))
    P.set_measurements(f(y))
    return P, f


def small_problem(seed=21, N=64, K=2, M=3, L=4, Pf=5):
    rng = np.random.default_rng(seed)
    d = inputs.gabor_filters(rng, L, Pf)
    z = inputs.bernoulli_gaussian_codes(rng, L, M, N, 0.02)
    x = inputs.convdict_image(inputs.embed_filters(d, N), z)
    h = inputs.gaussian_psf_bank(N, K, M)
    y, _ = inputs.measure(rng, x, h, 25.0)
    return h, y, d


@pytest.mark.parametrize("dtype,tol", [("f32", 1e-5), ("f64", 1e-10)])
def test_convdict_step_parity_small(torch, dtype, tol):
    h, y, d = small_problem()
    lam, rho, beta = 0.15, 8.0, 4.0
    S = fast.convdict_setup(h, y, d, lam, rho, beta)
    P, f = plan_for(torch, h, y, d, lam, rho, beta, dtype)
    L, M, N = d.shape[0], h.shape[1], h.shape[-1]
    z = np.zeros((L, M, N, N)); t = np.zeros_like(z); u = np.zeros_like(z)
    for l in range(6):
        x1, z1, t1, u1 = fast.convdict_step(S, z, t, u)
        if l in (0, 1, 5):
            P.state_import_coefficients(f(gl(z)), f(gl(t)), f(gl(u)))
            P.iterate(1)
            xg = P.get_x().double().cpu().numpy()
            zg = P.get_coefficients().double().cpu().numpy()
            ug = P.get_u().double().cpu().numpy()
            assert rel(xg, x1) <= tol, (l, rel(xg, x1))
            assert rel(zg, gl(z1)) <= tol, (l, rel(zg, gl(z1)))
            scale = max(np.linalg.norm(u1), np.linalg.norm(z1))
            assert np.linalg.norm(ug - gl(u1)) / scale <= tol
        z, t, u = z1, t1, u1
    P.close()


def test_convdict_small_matches_naive_oracle(torch):
    """Free-running 12 iterations from z = t = u = 0 against the naive-DFT oracle (N = 64, FP64 path)."""
    rng = np.random.default_rng(5)
    N, K, M, L, Pf = 64, 2, 2, 3, 3
    d = rng.standard_normal((L, Pf, Pf))
    d /= np.linalg.norm(d.reshape(L, -1), axis=1)[:, None, None]
    h = inputs.gaussian_psf_bank(N, K, M)
    y = rng.standard_normal((K, N, N))
    C = admm.convdict_setup(h, y, d, 0.1, 0.9, 1.7)
    x_or, z_or, t_or, u_or, _ = admm.run_convdict(C, 12)
    P, f = plan_for(torch, h, y, d, 0.1, 0.9, 1.7, "f64")
    P.iterate(12)
    assert rel(P.get_x().double().cpu().numpy(), x_or) <= 1e-10
    assert rel(P.get_coefficients().double().cpu().numpy(), gl(z_or)) <= 1e-10
    P.close()


@pytest.fixture(scope="module")
def cd_full():
    """The 256 x 256 x 5 workload with 32 Gabor 11 x 11 filters (25 dB, lambda=0.15, beta=4, rho=8)."""
    Pr = inputs.convdict_problem()
    S = fast.convdict_setup(Pr.h, Pr.y, Pr.filters, Pr.lam, Pr.rho, Pr.beta)
    return Pr, S


def test_convdict_full_size_steps(torch, cd_full):
    Pr, S = cd_full
    P, f = plan_for(torch, Pr.h, Pr.y, Pr.filters, Pr.lam, Pr.rho, Pr.beta)
    L, M, N = Pr.filters.shape[0], Pr.M, Pr.N
    z = np.zeros((L, M, N, N)); t = np.zeros_like(z); u = np.zeros_like(z)
    for l in range(11):
        x1, z1, t1, u1 = fast.convdict_step(S, z, t, u)
        if l in (0, 10):
            P.state_import_coefficients(f(gl(z)), f(gl(t)), f(gl(u)))
            P.iterate(1)
            assert rel(P.get_x().double().cpu().numpy(), x1) <= 1e-5
            assert rel(P.get_coefficients().double().cpu().numpy(), gl(z1)) <= 1e-5
        z, t, u = z1, t1, u1
    P.close()


def test_convdict_full_size_final_x(torch, cd_full):
    """300 free-running iterations of the 256 x 256 x 5, L = 32 workload: x within 1e-4 of the oracle's."""
    Pr, S = cd_full
    x_or, z_or, t_or, u_or = fast.run_convdict(S, Pr.iters)
    P, f = plan_for(torch, Pr.h, Pr.y, Pr.filters, Pr.lam, Pr.rho, Pr.beta)
    assert P.iterate(Pr.iters) == Pr.iters
    xg = P.get_x().double().cpu().numpy()
    r, s = P.residuals()
    P.close()
    assert rel(xg, x_or) <= 1e-4, rel(xg, x_or)
    assert np.isfinite(r) and np.isfinite(s)


def test_convdict_checkpoint_resume(torch):
    h, y, d = small_problem(seed=3)
    P, f = plan_for(torch, h, y, d, 0.15, 8.0, 4.0)
    P.iterate(4)
    ck = P.state_export()
    P.iterate(5)
    xa = P.get_x().cpu().numpy()
    P.state_restore(ck)
    P.iterate(5)
    xb = P.get_x().cpu().numpy()
    P.close()
    assert np.array_equal(xa, xb)


@pytest.mark.parametrize("mu", [0.01, 0.5])
def test_convdict_gradient_penalty_step_parity(torch, mu):
    """Gradient (Tikhonov) penalty on the codes (Eq. DL_PriorHP_conv): one GPU iteration from the
    oracle's state vs the oracle's, with mu = 0.01 (the paper's Tikhonov setting) and a larger
    mu that changes the z-update visibly; per-step tolerance 1e-5 (complex64 path)."""
    h, y, d = small_problem(seed=23)
    lam, rho, beta = 0.15, 8.0, 4.0
    S = fast.convdict_setup(h, y, d, lam, rho, beta, mu)
    S0 = fast.convdict_setup(h, y, d, lam, rho, beta, 0.0)
    P, f = plan_for(torch, h, y, d, lam, rho, beta)
    P.set_code_gradient_weight(mu)
    L, M, N = d.shape[0], h.shape[1], h.shape[-1]
    z = np.zeros((L, M, N, N)); t = np.zeros_like(z); u = np.zeros_like(z)
    for l in range(5):
        x1, z1, t1, u1 = fast.convdict_step(S, z, t, u)
        if l in (1, 4):
            P.state_import_coefficients(f(gl(z)), f(gl(t)), f(gl(u)))
            P.iterate(1)
            zg = P.get_coefficients().double().cpu().numpy()
            xg = P.get_x().double().cpu().numpy()
            assert rel(xg, x1) <= 1e-5, (l, rel(xg, x1))
            assert rel(zg, gl(z1)) <= 1e-5, (l, rel(zg, gl(z1)))
            _, z0, _, _ = fast.convdict_step(S0, z, t, u)
            assert rel(z0, z1) > 100 * max(rel(zg, gl(z1)), 1e-9)  # the penalty is really applied
        z, t, u = z1, t1, u1
    P.close()


def test_convdict_gradient_penalty_final(torch):
    """Free-running 40 iterations with mu = 0.1 from zero state: final x within 1e-4 of the oracle."""
    h, y, d = small_problem(seed=24)
    lam, rho, beta, mu = 0.15, 8.0, 4.0, 0.1
    S = fast.convdict_setup(h, y, d, lam, rho, beta, mu)
    x_ref, _, _, _ = fast.run_convdict(S, 40)
    P, f = plan_for(torch, h, y, d, lam, rho, beta)
    P.set_code_gradient_weight(mu)
    P.iterate(40)
    xg = P.get_x().double().cpu().numpy()
    assert rel(xg, x_ref) <= 1e-4, rel(xg, x_ref)
    P.close()


def test_gradient_weight_rejected_outside_dictionary(torch):
    from paper_2006_08303_gb300 import api
    P = api.Plan(64, 2, 2, "f32")
    P.set_prior("tv", 0.01, 1.0, 1.0)
    with pytest.raises(Exception):
        P.set_code_gradient_weight(0.1)
    P.close()


def test_convdict_adaptive_penalty(torch):
    """Adaptive penalty (Eq. paramS) on Alg. 2 from rho = 64: the rho trajectory is the oracle's
    (five halvings in 60 iterations, checks every 10) and the final x within 1e-4."""
    from paper_2006_08303_gb300 import api
    rng = np.random.default_rng(25)
    d = inputs.gabor_filters(rng, 4, 5)
    z = inputs.bernoulli_gaussian_codes(rng, 4, 3, 64, 0.02)
    x = inputs.convdict_image(inputs.embed_filters(d, 64), z)
    h = inputs.gaussian_psf_bank(64, 2, 3)
    y, _ = inputs.measure(rng, x, h, 25.0)
    lam, rho, beta = 0.15, 64.0, 4.0
    x_ref, _, _, _, rhos = fast.run_convdict_adaptive(h, y, d, lam, rho, beta, 60, 10)
    assert rhos[-1] == 2.0
    f = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32).cuda()
    P = api.Plan(64, 2, 3, "f32", check_every=10)
    P.set_prior("convdict", lam, rho, beta)
    P.set_rho_adaptation(2.0, 10.0)
    P.set_dictionary(f(d))
    P.set_psfs(f(h))
    P.set_measurements(f(y))
    P.iterate(60)
    assert P.rho == rhos[-1], (P.rho, rhos[-1])
    xg = P.get_x().double().cpu().numpy()
    assert rel(xg, x_ref) <= 1e-4, rel(xg, x_ref)
    P.close()

"""Pins for the FP64 oracle against mathematics and library routines, not
against itself.  Each test names the paper passage it pins; a plausible
mistake in the oracle (dropped term, wrong sign or index, transposed operand,
missing conjugate) fails at least one of them.  CPU only."""
import math

import numpy as np
import pytest
import scipy.fft as sfft

from oracle import admm
from oracle import fast
from paper_2006_08303_gb300 import inputs

RNG = np.random.default_rng(1234)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def random_psfs(rng, K, M, N):
    """Asymmetric, non-unit-sum PSFs so that Lambda is complex and K x M is not square-symmetric."""
    return rng.uniform(0.0, 1.0, size=(K, M, N, N)) * (rng.random((K, M, N, N)) < 0.4)


def dense_operator(apply, in_shape):
    """Columns = apply(unit vector)."""
    n = int(np.prod(in_shape))
    cols = []
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        cols.append(np.asarray(apply(e.reshape(in_shape))).ravel())
    return np.stack(cols, axis=1)


# ----------------------------------------------------------------- DFT & conv
@pytest.mark.parametrize("N", [4, 8, 16])
def test_dft_matches_library(N):
    """Section IV-A: F_2D is the 2D DFT; pinned to numpy.fft (textbook DFT)."""
    x = RNG.standard_normal((2, N, N)) + 1j * RNG.standard_normal((2, N, N))
    assert np.abs(admm.dft2(x) - np.fft.fft2(x)).max() < 1e-12 * N * N
    assert np.abs(admm.idft2(np.fft.fft2(x)) - x).max() < 1e-12


def test_parseval():
    x = RNG.standard_normal((8, 8))
    assert abs(np.sum(np.abs(admm.dft2(x)) ** 2) / 64 - np.sum(x * x)) < 1e-12


def test_circular_convolution_shift_and_theorem():
    """Eq. forward model: circular convolution with origin at (0,0).
    A delta at (1,2) shifts h by (1,2); the DFT of a convolution is the product (Section IV-A, BCCB)."""
    N = 8
    h = RNG.standard_normal((N, N))
    d = np.zeros((N, N)); d[1, 2] = 1.0
    y = admm.circconv2(d, h)
    assert np.array_equal(y, np.roll(h, (1, 2), axis=(0, 1)))
    x = RNG.standard_normal((N, N))
    y = admm.circconv2(x, h)
    assert np.abs(admm.dft2(y) - admm.dft2(x) * admm.dft2(h)).max() < 1e-10
    # brute-force definition at one output pixel
    n1, n2 = 3, 6
    direct = sum(x[j1, j2] * h[(n1 - j1) % N, (n2 - j2) % N] for j1 in range(N) for j2 in range(N))
    assert abs(y[n1, n2] - direct) < 1e-12


def test_forward_adjoint_pair():
    """H^T is the adjoint of H (needed by Eq. solx_Trans)."""
    K, M, N = 3, 2, 8
    h = random_psfs(RNG, K, M, N)
    x = RNG.standard_normal((M, N, N))
    y = RNG.standard_normal((K, N, N))
    lhs = np.sum(admm.forward_H(x, h) * y)
    rhs = np.sum(x * admm.adjoint_H(y, h))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


# ----------------------------------------------------------------- priors
def test_tv_explicit_values():
    """Anisotropic TV with circular forward differences (reading R1), hand example."""
    x = np.array([[0., 1., 3., 6.], [1., 1., 1., 1.], [2., 0., 2., 0.], [5., 4., 3., 2.]])
    w = admm.tv_forward(x)
    assert np.array_equal(w[0, 0], [1., 2., 3., -6.])          # x[0,c+1]-x[0,c], wraps 0-6
    assert np.array_equal(w[1][:, 0], [1., 1., 3., -5.])       # x[r+1,0]-x[r,0], wraps 0-5


@pytest.mark.parametrize("prior", ["tv", "dct8", "l1"])
def test_prior_adjoint(prior):
    """<Tx, w> = <x, T^T w> for every analysis operator."""
    fwd, adj = admm.PRIORS[prior]
    N = 16
    x = RNG.standard_normal((2, N, N))
    w = RNG.standard_normal(fwd(x).shape)
    assert abs(np.sum(fwd(x) * w) - np.sum(x * adj(w))) < 1e-11


def test_dct8_is_library_orthonormal_dct():
    """Block DCT (reading R12) equals scipy's orthonormal DCT-II on each aligned 8x8 block."""
    N = 16
    x = RNG.standard_normal((N, N))
    w = admm.dct8_forward(x)[0]
    for bi in range(0, N, 8):
        for bj in range(0, N, 8):
            ref = sfft.dctn(x[bi:bi + 8, bj:bj + 8], type=2, norm="ortho")
            assert np.abs(w[bi:bi + 8, bj:bj + 8] - ref).max() < 1e-13
    C = admm.dct8_matrix()
    assert np.abs(C @ C.T - np.eye(8)).max() < 1e-14
    assert np.abs(admm.dct8_adjoint(admm.dct8_forward(x)) - x).max() < 1e-13


@pytest.mark.parametrize("N", [8, 16])
def test_tv_gram_eigenvalues_closed_form(N):
    """g(w) for D^T D equals 4 sin^2(pi k1/N) + 4 sin^2(pi k2/N) (textbook Laplacian spectrum)."""
    g = admm.gram_eigenvalues("tv", N)
    k = np.arange(N)
    cf = 4 * np.sin(np.pi * k / N)[:, None] ** 2 + 4 * np.sin(np.pi * k / N)[None, :] ** 2
    assert np.abs(g - cf).max() < 1e-12


def test_soft_threshold_is_prox():
    """Eq. solt_trans: soft(v, lam/rho) = argmin_t lam|t| + rho/2 (t - v)^2, by grid search."""
    lam, rho = 0.3, 1.7
    grid = np.linspace(-3, 3, 600001)
    for v in [-2.1, -0.17, 0.0, 0.05, 0.176, 0.9, 2.4]:
        f = lam * np.abs(grid) + 0.5 * rho * (grid - v) ** 2
        tb = grid[np.argmin(f)]
        assert abs(admm.soft(np.array(v), lam / rho) - tb) < 2e-5
    assert admm.soft(np.array(-1.0), 0.5) == -0.5 and admm.soft(np.array(0.2), 0.5) == 0.0


# ----------------------------------------------------------------- per-bin algebra
@pytest.mark.parametrize("S", [1, 2, 3, 5, 10])
def test_recursive_block_inverse(S):
    """Eq. recinv (2x2 block recursion) agrees with a library inverse and inverts Psi."""
    A = RNG.standard_normal((S + 2, S)) + 1j * RNG.standard_normal((S + 2, S))
    P = 0.3 * np.eye(S) + A.conj().T @ A
    Ri = admm.recursive_block_inverse(P)
    assert np.abs(Ri - np.linalg.inv(P)).max() < 1e-12 * np.abs(Ri).max()
    assert np.abs(P @ Ri - np.eye(S)).max() < 1e-12


def test_psi_block_formula_reading():
    """Reading R3: Psi_{ij}(w) = rho delta_ij + beta sum_k conj(Lam_{k,i}) Lam_{k,j}; checked entrywise."""
    K, M, N = 3, 2, 4
    h = random_psfs(RNG, K, M, N)
    Lam = admm.psf_spectra(h)
    g = np.ones((N, N)) * 0.7
    Psi = admm.form_psi(Lam, g, 2.0, 3.0)
    a, b = 1, 2
    for i in range(M):
        for j in range(M):
            e = 2.0 * 0.7 * (i == j) + 3.0 * sum(np.conj(Lam[k, i, a, b]) * Lam[k, j, a, b] for k in range(K))
            assert abs(Psi[a, b, i, j] - e) < 1e-12


# ----------------------------------------------------------------- x-update vs dense LS
@pytest.mark.parametrize("prior,K,M,unit_sum", [("tv", 2, 2, True), ("tv", 3, 2, False),
                                                 ("dct8", 2, 3, False), ("l1", 3, 2, False),
                                                 ("tv", 1, 1, True)])
def test_x_update_equals_dense_least_squares(prior, K, M, unit_sum):
    """Eq. iter_ADMM1 solved densely: x = argmin beta/2||y-Hx||^2 + rho/2||Tx - t + u||^2,
    i.e. lstsq on [sqrt(beta) H; sqrt(rho) T] x = [sqrt(beta) y; sqrt(rho)(t-u)] (min-norm where singular,
    which pins reading R2).  The oracle's frequency-domain Eq. solx_Trans_DFT must match it."""
    N = 8
    rng = np.random.default_rng(7 + K + 10 * M)
    if unit_sum:
        h = inputs.gaussian_psf_bank(N, K, M)
        h = h * (1 + 0.2 * rng.random((K, M, N, N)))
        h /= h.sum(axis=(-2, -1), keepdims=True)
    else:
        h = random_psfs(rng, K, M, N)
    x_true = rng.standard_normal((M, N, N))
    y = admm.forward_H(x_true, h) + 0.1 * rng.standard_normal((K, N, N))
    beta, rho, lam = 1.3, 0.7, 0.05
    fwd, _ = admm.PRIORS[prior]
    ncomp = 2 if prior == "tv" else 1
    t = rng.standard_normal((M, ncomp, N, N))
    u = rng.standard_normal((M, ncomp, N, N))
    H = dense_operator(lambda v: admm.forward_H(v, h), (M, N, N))
    T = dense_operator(fwd, (M, N, N))
    A = np.concatenate([math.sqrt(beta) * H, math.sqrt(rho) * T])
    b = np.concatenate([math.sqrt(beta) * y.ravel(), math.sqrt(rho) * (t - u).ravel()])
    x_ls = np.linalg.lstsq(A, b, rcond=1e-11)[0].reshape(M, N, N)
    S = admm.analysis_setup(h, y, prior, lam, rho, beta)
    x_or = admm.x_update(S, t, u)
    assert rel(x_or, x_ls) < 1e-9


def test_normal_equation_residual_tiny_workload():
    """At 64x64x3 (tiny TV instance): (beta H^T H + rho T^T T) x = beta H^T y + rho T^T (t - u)
    with H applied by spatial convolution, to 1e-12 relative."""
    P = inputs.tiny_tv()
    S = admm.analysis_setup(P.h, P.y, P.prior, P.lam, P.rho, P.beta)
    rng = np.random.default_rng(3)
    t, u = inputs.random_state(rng, "tv", P.M, P.N)
    x = fast.x_update(fast.analysis_setup(P.h, P.y, P.prior, P.lam, P.rho, P.beta), t, u)
    assert rel(x, admm.x_update(S, t, u)) < 1e-11
    lhs = P.beta * admm.adjoint_H(admm.forward_H(x, P.h), P.h) + P.rho * admm.tv_adjoint(admm.tv_forward(x))
    rhs = P.beta * admm.adjoint_H(P.y, P.h) + P.rho * admm.tv_adjoint(t - u)
    # the DC null space (per-channel constants summing to zero) is invisible to both sides
    assert rel(lhs, rhs) < 1e-11


# ----------------------------------------------------------------- whole loop
def test_closed_form_l1_identity():
    """h = delta, K = M = 1, T = I: the problem min beta/2||y-x||^2 + lam||x||_1 has x* = soft(y, lam/beta)."""
    N = 8
    h = np.zeros((1, 1, N, N)); h[0, 0, 0, 0] = 1.0
    y = RNG.standard_normal((1, N, N))
    lam, beta, rho = 0.4, 1.0, 1.0
    S = admm.analysis_setup(h, y, "l1", lam, rho, beta)
    x, t, u, _ = admm.run_analysis(S, 400)
    assert np.abs(x - admm.soft(y, lam / beta)).max() < 1e-10


def test_closed_form_dct_identity():
    """h = delta, T = orthonormal block DCT: x* = T^T soft(T y, lam/beta)."""
    N = 16
    h = np.zeros((1, 1, N, N)); h[0, 0, 0, 0] = 1.0
    y = RNG.standard_normal((1, N, N))
    lam, beta, rho = 0.3, 2.0, 1.5
    S = admm.analysis_setup(h, y, "dct8", lam, rho, beta)
    x, _, _, _ = admm.run_analysis(S, 600)
    xs = admm.dct8_adjoint(admm.soft(admm.dct8_forward(y), lam / beta))
    assert np.abs(x - xs).max() < 1e-9


@pytest.fixture(scope="module")
def tv16():
    rng = np.random.default_rng(99)
    N, M = 16, 2
    x0 = inputs.rectangles_image(rng, N, M, n_rect=3)
    h = inputs.gaussian_psf_bank(N, 3, M)
    y, _ = inputs.measure(rng, x0, h, 30.0)
    lam, rho, beta = 1e-2, 0.5, 1.0
    S = admm.analysis_setup(h, y, "tv", lam, rho, beta)
    x, t, u, hist = admm.run_analysis(S, 3000, keep_history=True)
    return dict(h=h, y=y, lam=lam, rho=rho, beta=beta, S=S, x=x, t=t, u=u, hist=hist)


def test_dual_invariant_every_iteration(tv16):
    """From Eqs. solt_trans and subu_trans: u^{l+1} = clip(Tx + u^l, +-lam/rho), so |u| <= lam/rho and
    u = sign(t) lam/rho wherever t != 0 (the scaled dual is a subgradient of lam||t||_1 / rho)."""
    tau = tv16["lam"] / tv16["rho"]
    for rec in tv16["hist"][:60]:
        assert np.abs(rec.u).max() <= tau * (1 + 1e-12)
        nz = rec.t != 0
        assert np.abs(rec.u[nz] - np.sign(rec.t[nz]) * tau).max() < 1e-12


def test_kkt_at_convergence(tv16):
    """KKT certificate of Eq. rls with the TV prior: stationarity beta H^T(Hx - y) + rho T^T u = 0,
    feasibility Tx = t."""
    h, y, x, t, u = tv16["h"], tv16["y"], tv16["x"], tv16["t"], tv16["u"]
    g = tv16["beta"] * admm.adjoint_H(admm.forward_H(x, h) - y, h) + tv16["rho"] * admm.tv_adjoint(u)
    assert np.linalg.norm(g) / np.linalg.norm(tv16["beta"] * admm.adjoint_H(y, h)) < 1e-6
    w = admm.tv_forward(x)
    assert np.linalg.norm(w - t) <= 1e-6 * np.linalg.norm(w)


def test_he_yuan_monotone(tv16):
    """Two-block ADMM with fixed rho (He & Yuan 2015): rho(||t^{l+1}-t^l||^2 + ||u^{l+1}-u^l||^2)
    is non-increasing."""
    h = tv16["hist"]
    q = [np.sum((b.t - a.t) ** 2) + np.sum((b.u - a.u) ** 2) for a, b in zip(h[:-1], h[1:])]
    q = np.array(q[:800])
    assert np.all(q[1:] <= q[:-1] * (1 + 1e-9) + 1e-28)


def test_objective_decreases(tv16):
    S, rec = tv16["S"], tv16["hist"]
    f = lambda x: admm.objective(x, tv16["h"], tv16["y"], "tv", tv16["lam"], tv16["beta"])
    assert f(rec[-1].x) < f(rec[0].x)
    tail = np.array([f(r.x) for r in rec[-400::50]])
    assert np.all(np.abs(np.diff(tail)) <= 1e-9 * abs(tail[-1]) + 1e-12) or np.all(np.diff(tail) <= 1e-12)


# ----------------------------------------------------------------- synthesis (Alg. 2)
def test_sherman_morrison_dense():
    """Eq. solz_DFT_SM with reading R10 solves (rho I + conj(theta) theta^T) v = c."""
    L = 32
    th = RNG.standard_normal(L) + 1j * RNG.standard_normal(L)
    c = RNG.standard_normal(L) + 1j * RNG.standard_normal(L)
    rho = 0.8
    A = rho * np.eye(L) + np.outer(th.conj(), th)
    v = admm.sherman_morrison(th, c, rho)
    assert np.abs(A @ v - c).max() < 1e-12


@pytest.fixture(scope="module")
def cd8():
    rng = np.random.default_rng(5)
    N, K, M, L, P = 8, 2, 2, 3, 3
    d = rng.standard_normal((L, P, P))
    d /= np.linalg.norm(d.reshape(L, -1), axis=1)[:, None, None]
    h = random_psfs(rng, K, M, N)
    x0 = rng.standard_normal((M, N, N))
    y = admm.forward_H(x0, h)
    C = admm.convdict_setup(h, y, d, 0.1, 0.9, 1.7)
    z = rng.standard_normal((L, M, N, N))
    t = rng.standard_normal((L, M, N, N))
    u = rng.standard_normal((L, M, N, N))
    return dict(rng=rng, N=N, K=K, M=M, L=L, d=d, h=h, y=y, C=C, z=z, t=t, u=u)


@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_convdict_x_and_z_update_dense(cd8, mu):
    """Eq. iterd_ADMM1 and Eq. iterd_ADMM2 solved densely (reading R9: 1/2||Dz - x||^2,
    rho/2 ||z - t + u||^2; with mu > 0 also mu/2 sum ||r_i * z_m||^2 of Eq. DL_PriorHP_conv,
    r_i the circular differences along each axis, built here as an explicit dense operator)
    match Eqs. solx_synt_DFT and solz_DFT/solz_DFT_SM of the oracle."""
    N, M, L, d, h, y = cd8["N"], cd8["M"], cd8["L"], cd8["d"], cd8["h"], cd8["y"]
    C0 = cd8["C"]
    C = admm.convdict_setup(h, y, d, C0.lam, C0.rho, C0.beta, mu)
    z, t, u = cd8["z"], cd8["t"], cd8["u"]
    de = admm.embed_filters(d, N)
    Dop = lambda zz: np.stack([sum(admm.circconv2(zz[l, m], de[l]) for l in range(L)) for m in range(M)])
    H = dense_operator(lambda v: admm.forward_H(v, h), (M, N, N))
    D = dense_operator(Dop, (L, M, N, N))

    def grad_op(zz):  # [L, M, N, N] -> both axis differences of every code map, by index shifts
        return np.stack([np.roll(zz, -1, axis=2) - zz, np.roll(zz, -1, axis=3) - zz])

    G = dense_operator(grad_op, (L, M, N, N))
    beta, rho = C.beta, C.rho
    A = np.concatenate([math.sqrt(beta) * H, np.eye(M * N * N)])
    b = np.concatenate([math.sqrt(beta) * y.ravel(), Dop(z).ravel()])
    x_ls = np.linalg.lstsq(A, b, rcond=None)[0].reshape(M, N, N)
    A2 = np.concatenate([D, math.sqrt(rho) * np.eye(L * M * N * N), math.sqrt(mu) * G])
    b2 = np.concatenate([x_ls.ravel(), math.sqrt(rho) * (t - u).ravel(), np.zeros(G.shape[0])])
    z_ls = np.linalg.lstsq(A2, b2, rcond=None)[0].reshape(L, M, N, N)
    x, z_new, t_new, u_new = admm.convdict_step(C, z, t, u)
    assert rel(x, x_ls) < 1e-10
    assert rel(z_new, z_ls) < 1e-9
    assert np.allclose(t_new, admm.soft(z_new + u, C.lam / C.rho), atol=0)
    assert np.allclose(u_new, u + z_new - t_new, atol=0)


# ----------------------------------------------------------------- fast form vs naive
@pytest.mark.parametrize("prior", ["tv", "dct8", "l1"])
def test_fast_oracle_matches_naive(prior):
    """The fast FP64 oracle (pocketfft) reproduces the naive DFT oracle to <= 1e-11."""
    rng = np.random.default_rng(11)
    N, K, M = 16, 3, 2
    h = random_psfs(rng, K, M, N) if prior != "tv" else inputs.gaussian_psf_bank(N, K, M)
    y = rng.standard_normal((K, N, N))
    S = admm.analysis_setup(h, y, prior, 0.05, 0.7, 1.2)
    F = fast.analysis_setup(h, y, prior, 0.05, 0.7, 1.2)
    xs, ts, us, _ = admm.run_analysis(S, 20)
    xf, tf, uf, _, _ = fast.run_analysis(F, 20)
    assert rel(xf, xs) < 1e-11 and rel(uf, us) < 1e-11


@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_fast_convdict_matches_naive(cd8, mu):
    C0 = cd8["C"]
    C = admm.convdict_setup(cd8["h"], cd8["y"], cd8["d"], C0.lam, C0.rho, C0.beta, mu)
    F = fast.convdict_setup(cd8["h"], cd8["y"], cd8["d"], C.lam, C.rho, C.beta, mu)
    xs, zs, ts, us, _ = admm.run_convdict(C, 6)
    xf, zf, tf, uf = fast.run_convdict(F, 6)
    assert rel(xf, xs) < 1e-11 and rel(zf, zs) < 1e-11


def test_fast_oracle_tiny_workload_residuals():
    """At 64x64x3 the fast and naive oracles agree on 50 iterations of Alg. 1 and on the residuals."""
    P = inputs.tiny_tv()
    S = admm.analysis_setup(P.h, P.y, P.prior, P.lam, P.rho, P.beta)
    F = fast.analysis_setup(P.h, P.y, P.prior, P.lam, P.rho, P.beta)
    xs, _, us, hist = admm.run_analysis(S, 50, keep_history=True)
    xf, _, uf, n, rr = fast.run_analysis(F, 50, tol=1e-30)
    assert n == 50 and rel(xf, xs) < 1e-11
    assert abs(rr[0] - hist[-1].r_rel) < 1e-9 * hist[-1].r_rel
    assert abs(rr[1] - hist[-1].s_rel) < 1e-9 * hist[-1].s_rel


# ----------------------------------------------------------------- adaptive penalty (Eq. paramS)
def test_adapt_rho_rule():
    assert admm.adapt_rho(1.0, 11.0, 1.0) == 2.0        # primal residual dominates: rho * tau
    assert admm.adapt_rho(1.0, 1.0, 11.0) == 0.5        # dual residual dominates: rho / tau
    assert admm.adapt_rho(1.0, 5.0, 1.0) == 1.0         # balanced within mu
    assert admm.adapt_rho(3.0, 1.0, 100.0, tau=3.0, mu=5.0) == 1.0


def test_adaptive_rho_reaches_the_fixed_rho_minimiser():
    """The minimiser of Eq. rls does not depend on rho: adaptive-rho ADMM, started from a badly
    chosen rho, ends at the fixed-rho solution, and it does change rho on the way."""
    P = inputs.tiny_tv(N=16, M=2, iters=1)
    S = admm.analysis_setup(P.h, P.y, P.prior, P.lam, 1.0, P.beta)
    x_fix, _, _, _ = admm.run_analysis(S, 3000)
    x_ad, _, _, rhos = admm.run_analysis_adaptive(P.h, P.y, P.prior, P.lam, 100.0, P.beta, 600, 10)
    assert len(set(rhos)) > 1
    assert rel(x_ad, x_fix) < 1e-6


def test_adaptive_rho_keeps_the_unscaled_multiplier():
    """Reading R18: at a change of rho the scaled dual is rescaled so that rho u is continuous;
    the first iteration after the change equals one fixed-rho step at the new rho from
    (t, u rho_old / rho_new)."""
    P = inputs.tiny_tv(N=16, M=2, iters=1)
    x10, t10, u10, rhos = admm.run_analysis_adaptive(P.h, P.y, P.prior, P.lam, 100.0, P.beta, 10, 10)
    assert rhos[-1] != 100.0
    x11, t11, u11, _ = admm.run_analysis_adaptive(P.h, P.y, P.prior, P.lam, 100.0, P.beta, 11, 10)
    S_new = admm.analysis_setup(P.h, P.y, P.prior, P.lam, rhos[-1], P.beta)
    x_step, t_step, u_step, _ = admm.analysis_step(S_new, t10, u10)
    assert rel(x11, x_step) < 1e-12 and rel(u11, u_step) < 1e-12
    _, _, u_pre, _ = admm.run_analysis(admm.analysis_setup(P.h, P.y, P.prior, P.lam, 100.0, P.beta), 10)
    assert rel(rhos[-1] * u10, 100.0 * u_pre) < 1e-12


def test_fast_adaptive_matches_naive():
    P = inputs.tiny_tv(N=16, M=2, iters=1)
    xn, tn, un, rn = admm.run_analysis_adaptive(P.h, P.y, P.prior, P.lam, 100.0, P.beta, 60, 10)
    xf, tf, uf, rf, _ = fast.run_analysis_adaptive(P.h, P.y, P.prior, P.lam, 100.0, P.beta, 60, 10)
    assert rn == rf
    assert rel(xf, xn) < 1e-10 and rel(uf, un) < 1e-10


# ----------------------------------------------------------------- isotropic TV (reading R20)
def test_group_soft_is_the_prox():
    """t = v max(0, 1 - tau/||v||) minimises 1/2||t - v||^2 + tau ||t||_2 per pixel: checked by the
    optimality conditions (t - v + tau t/||t|| = 0 where t != 0, ||v|| <= tau where t = 0) and
    against every point of a fine polar grid around v."""
    rng = np.random.default_rng(3)
    v = rng.standard_normal((5, 2, 7, 7))
    tau = 0.9
    t = admm.group_soft(v, tau)
    n_t = np.sqrt(np.sum(t * t, axis=1, keepdims=True))
    n_v = np.sqrt(np.sum(v * v, axis=1))
    nz = n_t[:, 0] > 0
    g = (t - v + tau * t / np.where(n_t > 0, n_t, 1.0))
    assert np.abs(np.moveaxis(g, 1, -1)[nz]).max() < 1e-12
    assert np.all(n_v[~nz] <= tau + 1e-12) and np.all(n_v[nz] > tau)
    f = lambda tt, vv: 0.5 * np.sum((tt - vv) ** 2) + tau * np.sqrt(np.sum(tt * tt))
    vv = v[0, :, 0, 0]
    best = f(t[0, :, 0, 0], vv)
    rr, th = np.meshgrid(np.linspace(0, 3, 301), np.linspace(0, 2 * np.pi, 361))
    grid = np.stack([rr * np.cos(th), rr * np.sin(th)], -1).reshape(-1, 2)
    assert best <= min(f(p, vv) for p in grid) + 1e-9


@pytest.fixture(scope="module")
def tviso16():
    rng = np.random.default_rng(98)
    N, M = 16, 2
    x0 = inputs.rectangles_image(rng, N, M, n_rect=3)
    h = inputs.gaussian_psf_bank(N, 3, M)
    y, _ = inputs.measure(rng, x0, h, 30.0)
    lam, rho, beta = 1e-2, 0.5, 1.0
    S = admm.analysis_setup(h, y, "tv_iso", lam, rho, beta)
    x, t, u, hist = admm.run_analysis(S, 3000, keep_history=True)
    return dict(h=h, y=y, lam=lam, rho=rho, beta=beta, S=S, x=x, t=t, u=u, hist=hist)


def test_isotropic_dual_in_ball_every_iteration(tviso16):
    """Isotropic counterpart of the dual invariant: ||u|| <= lam/rho per pixel, and u = t/||t|| lam/rho
    wherever t != 0."""
    tau = tviso16["lam"] / tviso16["rho"]
    for rec in tviso16["hist"][:60]:
        nu = np.sqrt(np.sum(rec.u ** 2, axis=1))
        assert nu.max() <= tau * (1 + 1e-12)
        nt = np.sqrt(np.sum(rec.t ** 2, axis=1, keepdims=True))
        nz = nt[:, 0] > 0
        d = np.moveaxis(rec.u - tau * rec.t / np.where(nt > 0, nt, 1.0), 1, -1)[nz]
        assert np.abs(d).max() < 1e-12


def test_isotropic_kkt_and_objective(tviso16):
    """Stationarity beta H^T(Hx - y) + rho D^T u = 0 and feasibility Dx = t at convergence; the
    isotropic objective is below the anisotropic solution's value of it (the latter minimises
    a different problem) and below the first iterate's."""
    d = tviso16
    g = d["beta"] * admm.adjoint_H(admm.forward_H(d["x"], d["h"]) - d["y"], d["h"]) + d["rho"] * admm.tv_adjoint(d["u"])
    assert np.linalg.norm(g) / np.linalg.norm(d["beta"] * admm.adjoint_H(d["y"], d["h"])) < 1e-6
    w = admm.tv_forward(d["x"])
    assert np.linalg.norm(w - d["t"]) <= 1e-6 * np.linalg.norm(w)
    f = lambda x: admm.objective(x, d["h"], d["y"], "tv_iso", d["lam"], d["beta"])
    S_an = admm.analysis_setup(d["h"], d["y"], "tv", d["lam"], d["rho"], d["beta"])
    x_an, _, _, _ = admm.run_analysis(S_an, 3000)
    assert f(d["x"]) < f(x_an)
    assert f(d["x"]) < f(d["hist"][0].x)


def test_fast_oracle_matches_naive_tv_iso():
    rng = np.random.default_rng(12)
    N, K, M = 16, 3, 2
    h = inputs.gaussian_psf_bank(N, K, M)
    y = rng.standard_normal((K, N, N))
    S = admm.analysis_setup(h, y, "tv_iso", 0.05, 0.7, 1.2)
    F = fast.analysis_setup(h, y, "tv_iso", 0.05, 0.7, 1.2)
    xs, ts, us, _ = admm.run_analysis(S, 20)
    xf, tf, uf, _, _ = fast.run_analysis(F, 20)
    assert rel(xf, xs) < 1e-11 and rel(uf, us) < 1e-11


def test_convdict_adaptive_keeps_the_unscaled_multiplier(cd8):
    """Adaptive penalty on Alg. 2 (readings R17, R18): the iteration after a change equals one
    fixed-rho step at the new rho from (z, t, u rho_old/rho_new)."""
    C0 = cd8["C"]
    args = (cd8["h"], cd8["y"], cd8["d"], C0.lam, 50.0, C0.beta)
    x5, z5, t5, u5, rhos = fast.run_convdict_adaptive(*args, 5, 5)
    assert rhos[-1] != 50.0
    x6, z6, t6, u6, _ = fast.run_convdict_adaptive(*args, 6, 5)
    C_new = fast.convdict_setup(cd8["h"], cd8["y"], cd8["d"], C0.lam, rhos[-1], C0.beta)
    xs, zs, ts, us = fast.convdict_step(C_new, z5, t5, u5)
    assert rel(x6, xs) < 1e-12 and rel(z6, zs) < 1e-12 and rel(u6, us) < 1e-12
    _, _, _, u_fix = fast.run_convdict(fast.convdict_setup(cd8["h"], cd8["y"], cd8["d"], C0.lam, 50.0, C0.beta), 5)
    assert rel(rhos[-1] * u5, 50.0 * u_fix) < 1e-12


# ----------------------------------------------------------------- online dictionary update
def test_filter_projection_is_the_nearest_feasible_point():
    """Eq. g_admm: Q Q^T v / ||Q^T v|| has the P x P support, unit norm, and is at least as close to v
    as any other unit-norm filter on the support (checked against random ones)."""
    rng = np.random.default_rng(4)
    N, L, P = 12, 3, 5
    v = rng.standard_normal((L, N, N))
    g = admm.project_filters(v, P)
    mask = admm.embed_filters(np.ones((1, P, P)), N)[0] != 0
    assert np.all(g[:, ~mask] == 0)
    assert np.allclose(np.sqrt(np.sum(g * g, axis=(1, 2))), 1.0)
    for l in range(L):
        best = np.sum((g[l] - v[l]) ** 2)
        for _ in range(200):
            c = rng.standard_normal((P, P))
            c = admm.embed_filters((c / np.linalg.norm(c))[None], N)[0]
            assert best <= np.sum((c - v[l]) ** 2) + 1e-12


def test_filter_update_equals_dense_least_squares():
    """Eq. d_admm summed over the slices (Eq. sold_3D in 2D) solved densely: the stacked system
    [Z; sqrt(sigma) I] d = [x; sqrt(sigma)(g - e)] with Z the explicit convolution operator of the
    codes matches the oracle's per-frequency solve."""
    rng = np.random.default_rng(6)
    N, L, S, P, sigma = 6, 2, 2, 3, 1.7
    z = rng.standard_normal((L, S, N, N))
    x = rng.standard_normal((S, N, N))
    g = rng.standard_normal((L, N, N))
    e = rng.standard_normal((L, N, N))
    Zop = lambda dd: np.stack([sum(admm.circconv2(z[l, s], dd[l]) for l in range(L)) for s in range(S)])
    Zd = dense_operator(Zop, (L, N, N))
    A = np.concatenate([Zd, math.sqrt(sigma) * np.eye(L * N * N)])
    b = np.concatenate([x.ravel(), math.sqrt(sigma) * (g - e).ravel()])
    d_ls = np.linalg.lstsq(A, b, rcond=None)[0].reshape(L, N, N)
    d, g_new, e_new = admm.dict_update(x, z, g, e, sigma, P)
    assert rel(d, d_ls) < 1e-10
    assert np.allclose(e_new, e + d - g_new, atol=0)


def test_fast_learning_matches_naive(cd8):
    C = cd8["C"]
    args = (cd8["h"], cd8["y"], cd8["d"], C.lam, C.rho, C.beta, 2.0, 5)
    xn, zn, tn, un, fn = admm.run_convdict_learn(*args)
    xf, zf, tf, uf, ff = fast.run_convdict_learn(*args)
    assert rel(xf, xn) < 1e-10 and rel(ff, fn) < 1e-10
    assert rel(fn, cd8["d"] / np.linalg.norm(cd8["d"].reshape(cd8["L"], -1), axis=1)[:, None, None]) > 1e-3


# ----------------------------------------------------------------- Kronecker wavelet (x) DCT prior
def test_symlet_construction_textbook_cases():
    """Daubechies' spectral factorisation: one vanishing moment gives Haar, two give the D4
    filter (1+sqrt3, 3+sqrt3, 3-sqrt3, 1-sqrt3) / (4 sqrt2)."""
    assert np.allclose(admm.symlet_lowpass(1), [1 / math.sqrt(2)] * 2, atol=1e-15)
    s3 = math.sqrt(3.0)
    d4 = np.array([1 + s3, 3 + s3, 3 - s3, 1 - s3]) / (4 * math.sqrt(2.0))
    assert np.allclose(admm.symlet_lowpass(2), d4, atol=1e-13)


def test_sym8_orthonormal_with_eight_vanishing_moments():
    """The Symmlet-8 lowpass (Section V): 16 taps, sum sqrt 2, orthonormal to its even shifts,
    and the highpass g_k = (-1)^k h_{15-k} annihilates polynomials of degree < 8."""
    h = admm.symlet_lowpass(8)
    assert h.size == 16 and abs(h.sum() - math.sqrt(2.0)) < 1e-13
    for k in range(8):
        assert abs(np.dot(h[2 * k:], h[: 16 - 2 * k]) - (1.0 if k == 0 else 0.0)) < 1e-12
    g = np.array([(-1) ** k * h[15 - k] for k in range(16)])
    n = np.arange(16.0)
    for k in range(8):
        assert abs(np.dot(g, n ** k)) < 1e-9 * max(1.0, np.abs(n ** k).sum())


def test_sym8_is_less_asymmetric_than_the_minimum_phase_filter():
    """The least-asymmetric choice (reading R24) is not Daubechies' minimum-phase D16, and its
    energy is far more concentrated around the centre of the support."""
    h = admm.symlet_lowpass(8)
    # minimum-phase: every root of P kept inside the unit circle
    coeffs = [math.comb(7 + k, k) for k in range(8)]
    q = np.array([1.0 + 0j])
    for y in np.roots(coeffs[::-1]):
        w = 1 - 2 * y
        z = w + np.sqrt(w * w - 1 + 0j)
        q = np.convolve(q, [1.0, -(z if abs(z) < 1 else 1 / z)])
    for _ in range(8):
        q = np.convolve(q, [1.0, 1.0])
    d16 = q.real * math.sqrt(2.0) / q.real.sum()
    assert np.abs(np.abs(h) - np.abs(d16)).max() > 1e-2
    spread = lambda f: np.sum((np.arange(16) - np.sum(np.arange(16) * f * f)) ** 2 * f * f)
    assert spread(h) < 0.6 * spread(d16)


@pytest.mark.parametrize("n", [32, 64])
def test_dwt_level_is_periodic_filtering_and_orthogonal(n):
    """One level equals circular filtering with h and g followed by keeping even samples, and its
    matrix is orthogonal on any even length at least the filter length."""
    h = admm.symlet_lowpass(8)
    g = np.array([(-1) ** k * h[15 - k] for k in range(16)])
    A = admm.dwt_matrix(n, h)
    x = RNG.standard_normal(n)
    xx = np.concatenate([x, x])       # periodic extension
    lo = np.array([sum(h[k] * xx[2 * i + k] for k in range(16)) for i in range(n // 2)])
    hi = np.array([sum(g[k] * xx[2 * i + k] for k in range(16)) for i in range(n // 2)])
    assert np.allclose(A @ x, np.concatenate([lo, hi]), atol=1e-13)
    assert np.abs(A @ A.T - np.eye(n)).max() < 1e-12


def test_channel_dct_matches_library():
    for n in (1, 3, 10):
        assert np.allclose(admm.dct_matrix(n), sfft.dct(np.eye(n), axis=0, norm="ortho"), atol=1e-14)


def test_wdct_is_the_kronecker_product():
    """T = W (x) C (Section V): for x_m = a_m B, T x = (C a)_k W(B), with W(B) the 2D wavelet of
    one channel (the M = 1 transform)."""
    M, N = 4, 64
    a = RNG.standard_normal(M)
    B = RNG.standard_normal((N, N))
    x = a[:, None, None] * B[None]
    WB = admm.wdct_forward(B[None])[0, 0]
    expect = (admm.dct_matrix(M) @ a)[:, None, None] * WB[None]
    assert rel(admm.wdct_forward(x)[:, 0], expect) < 1e-13


def test_wdct_orthonormal_and_constant_image():
    """T is orthonormal (norm kept, T^T the inverse, adjoint identity); a constant image lands in
    the DC channel of the coarse 16 x 16 band with value c sqrt(M) 2^J (each level multiplies the
    constant by 2), every other coefficient zero."""
    M, N = 3, 64
    x = RNG.standard_normal((M, N, N))
    c = RNG.standard_normal((M, 1, N, N))
    Tx = admm.wdct_forward(x)
    assert abs(np.linalg.norm(Tx) - np.linalg.norm(x)) < 1e-12 * np.linalg.norm(x)
    assert np.abs(admm.wdct_adjoint(Tx) - x).max() < 1e-12
    assert abs(np.sum(Tx * c) - np.sum(x * admm.wdct_adjoint(c))) < 1e-11 * np.linalg.norm(x) * np.linalg.norm(c)
    J = admm.wavelet_levels(N)
    w = admm.wdct_forward(np.full((M, N, N), 0.7))[:, 0]
    expect = np.zeros_like(w)
    expect[0, :16, :16] = 0.7 * math.sqrt(M) * 2 ** J
    assert np.abs(w - expect).max() < 1e-10


def test_closed_form_wdct_identity():
    """h = delta per channel (K = M), T orthonormal: x* = T^T soft(T y, lam/beta)."""
    N, M = 32, 3
    h = np.zeros((M, M, N, N))
    for m in range(M):
        h[m, m, 0, 0] = 1.0
    y = RNG.standard_normal((M, N, N))
    lam, beta, rho = 0.3, 2.0, 1.5
    S = admm.analysis_setup(h, y, "wdct", lam, rho, beta)
    x, _, _, _ = admm.run_analysis(S, 400)
    xs = admm.wdct_adjoint(admm.soft(admm.wdct_forward(y), lam / beta))
    assert np.abs(x - xs).max() < 1e-9


def test_fast_wdct_matches_naive():
    rng = np.random.default_rng(17)
    N, K, M = 32, 3, 3
    h = random_psfs(rng, K, M, N)
    y = rng.standard_normal((K, N, N))
    S = admm.analysis_setup(h, y, "wdct", 0.05, 0.7, 1.0)
    F = fast.analysis_setup(h, y, "wdct", 0.05, 0.7, 1.0)
    xn = admm.run_analysis(S, 6)[0]
    xf = fast.run_analysis(F, 6)[0]
    assert rel(xf, xn) < 1e-11


# ----------------------------------------------------------------- 3D convolutional dictionary
def test_dft3_matches_library():
    v = RNG.standard_normal((2, 3, 6, 6))
    assert np.allclose(admm.dft3(v), np.fft.fftn(v, axes=(-3, -2, -1)), atol=1e-12)
    assert np.allclose(admm.idft3(admm.dft3(v)).real, v, atol=1e-12)


def conv3_brute(z, d3e):
    """Circular 3D convolution by its definition: out[s,i,j] = sum d[q,a,b] z[s-q, i-a, j-b]."""
    S, N, _ = z.shape
    out = np.zeros_like(z)
    for q in range(S):
        for a in range(N):
            for b in range(N):
                if d3e[q, a, b] != 0.0:
                    out += d3e[q, a, b] * np.roll(np.roll(np.roll(z, q, axis=0), a, axis=1), b, axis=2)
    return out


@pytest.fixture(scope="module")
def cd3():
    rng = np.random.default_rng(8)
    N, K, S, L, Q, P = 6, 2, 3, 2, 3, 3
    d3 = rng.standard_normal((L, Q, P, P))
    h = random_psfs(rng, K, S, N)
    y = rng.standard_normal((K, N, N))
    C = admm.convdict3d_setup(h, y, d3, 0.1, 0.9, 1.7)
    z, t, u = (rng.standard_normal((L, S, N, N)) for _ in range(3))
    return dict(N=N, S=S, L=L, d3=d3, h=h, y=y, C=C, z=z, t=t, u=u)


def test_convdict3d_x_and_z_update_dense(cd3):
    """The 3D case of Section IV-B solved densely with the explicit circular 3D convolution
    operator: x = argmin beta/2||y - Hx||^2 + 1/2||D~z - x||^2 and the normal equation Eq. solz
    for z match the oracle's per-bin (1D inverse DFT along the channels, Sherman-Morrison) forms."""
    N, S, L, d3, h, y, C = (cd3[k] for k in ("N", "S", "L", "d3", "h", "y", "C"))
    z, t, u = cd3["z"], cd3["t"], cd3["u"]
    de = admm.embed_filters3d(d3, N, S)
    Dop = lambda zz: sum(conv3_brute(zz[l], de[l]) for l in range(L))
    H = dense_operator(lambda v: admm.forward_H(v, h), (S, N, N))
    D = dense_operator(Dop, (L, S, N, N))
    A = np.concatenate([math.sqrt(C.beta) * H, np.eye(S * N * N)])
    b = np.concatenate([math.sqrt(C.beta) * y.ravel(), Dop(z).ravel()])
    x_ls = np.linalg.lstsq(A, b, rcond=None)[0].reshape(S, N, N)
    A2 = np.concatenate([D, math.sqrt(C.rho) * np.eye(L * S * N * N)])
    b2 = np.concatenate([x_ls.ravel(), math.sqrt(C.rho) * (t - u).ravel()])
    z_ls = np.linalg.lstsq(A2, b2, rcond=None)[0].reshape(L, S, N, N)
    x, z_new, t_new, u_new = admm.convdict3d_step(C, z, t, u)
    assert rel(x, x_ls) < 1e-10
    assert rel(z_new, z_ls) < 1e-9
    assert np.allclose(u_new, u + z_new - t_new, atol=0)


def test_convdict3d_with_one_channel_tap_is_the_2d_dictionary(cd8):
    """Q = 1: a 3D filter with a single channel tap convolves every channel with the same 2D
    filter, so Alg. 2 with 3D codes equals Alg. 2 with per-channel 2D codes."""
    C2 = cd8["C"]
    d = cd8["d"]
    C3 = admm.convdict3d_setup(cd8["h"], cd8["y"], d[:, None], C2.lam, C2.rho, C2.beta)
    z, t, u = cd8["z"], cd8["t"], cd8["u"]
    for a, b in zip(admm.convdict3d_step(C3, z, t, u), admm.convdict_step(C2, z, t, u)):
        assert rel(a, b) < 1e-11


def test_fast_convdict3d_matches_naive(cd3):
    C = cd3["C"]
    F = fast.convdict3d_setup(cd3["h"], cd3["y"], cd3["d3"], C.lam, C.rho, C.beta)
    z = np.zeros((cd3["L"], cd3["S"], cd3["N"], cd3["N"]))
    t, u = np.zeros_like(z), np.zeros_like(z)
    zn, tn, un = z, t, u
    for _ in range(4):
        xf, z, t, u = fast.convdict3d_step(F, z, t, u)
        xn, zn, tn, un = admm.convdict3d_step(C, zn, tn, un)
    assert rel(xf, xn) < 1e-11 and rel(z, zn) < 1e-11


# ----------------------------------------------------------------- adaptive sigma (filter ADMM)
def test_sigma_adaptation_never_triggered_is_the_fixed_run(cd8):
    C = cd8["C"]
    args = (cd8["h"], cd8["y"], cd8["d"], C.lam, C.rho, C.beta, 2.0, 6)
    fixed = admm.run_convdict_learn(*args)
    adapt = admm.run_convdict_learn(*args, check_every=2, tau=2.0, mu=1e30)
    assert all(s == 2.0 for s in adapt[5])
    for a, b in zip(fixed, adapt[:5]):
        assert np.array_equal(a, b)


def test_sigma_adaptation_keeps_the_unscaled_multiplier(cd8):
    """Reading R29: at a change of sigma the multiplier sigma e is kept.  An independent loop in
    unscaled form (multiplier m; the filter step fed e = m / sigma, then m = sigma e') under the
    same sigma schedule gives the oracle's iterates."""
    C0 = cd8["C"]
    h, y, d = cd8["h"], cd8["y"], cd8["d"]
    iters, ce = 8, 2
    x_a, z_a, t_a, u_a, f_a, sig = admm.run_convdict_learn(h, y, d, C0.lam, C0.rho, C0.beta, 2.0, iters,
                                                           check_every=ce, tau=2.0, mu=1.01)
    assert len(set(sig)) > 1  # the schedule really changes sigma
    P = d.shape[-1]
    C = admm.convdict_setup(h, y, d, C0.lam, C0.rho, C0.beta)
    g = admm.embed_filters(d, C.N)
    m = np.zeros_like(g)
    z = np.zeros((C.L, C.M, C.N, C.N)); t = np.zeros_like(z); u = np.zeros_like(z)
    sigma = 2.0
    for it in range(iters):
        C.theta = admm.dft2(g)
        x, z, t, u = admm.convdict_step(C, z, t, u)
        _, g, e_new = admm.dict_update(x, z, g, m / sigma, sigma, P)
        m = sigma * e_new
        sigma = sig[it]       # the schedule; m is left as it is
    assert rel(admm.crop_filters(g, P), f_a) < 1e-12 and rel(x, x_a) < 1e-12


def test_fast_sigma_adaptation_matches_naive(cd8):
    C = cd8["C"]
    args = (cd8["h"], cd8["y"], cd8["d"], C.lam, C.rho, C.beta, 2.0, 6)
    n = admm.run_convdict_learn(*args, check_every=2, tau=2.0, mu=1.01)
    f = fast.run_convdict_learn(*args, check_every=2, tau=2.0, mu=1.01)
    assert n[5] == f[5]
    assert rel(f[4], n[4]) < 1e-10 and rel(f[0], n[0]) < 1e-10


def test_convdict_x_update_minimises_the_synthesis_objective(cd8):
    """Reading R9: the x-update of Alg. 2 (Eq. solx_synt_DFT, t = 1) is the minimiser over x of
    beta/2 ||y - Hx||^2 + 1/2 ||D~z - x||^2 (+ lam ||z||_1, constant in x): perturbations of x
    raise the objective, by the quadratic amount the Hessian beta H^T H + I predicts."""
    C = cd8["C"]
    z, t, u = cd8["z"], cd8["t"], cd8["u"]
    x, _, _, _ = admm.convdict_step(C, z, t, u)
    f = lambda xx: admm.convdict_objective(xx, z, cd8["d"], cd8["h"], cd8["y"], C.lam, C.beta)
    f0 = f(x)
    rng = np.random.default_rng(21)
    for _ in range(5):
        dx = 1e-2 * rng.standard_normal(x.shape)
        quad = 0.5 * C.beta * float(np.sum(admm.forward_H(dx, cd8["h"]) ** 2)) + 0.5 * float(np.sum(dx * dx))
        assert abs(f(x + dx) - f0 - quad) < 1e-9 * max(1.0, abs(f0))


def test_filter_admm_reaches_a_kkt_point_and_the_printed_dual_sign_diverges():
    """Reading R22.  For fixed x and codes z, repeating the filter step with e <- e + d - g reaches
    a fixed point that satisfies the optimality conditions of Eq. Constrained2: d = g, g on the
    P x P support with unit norm, and the multiplier sigma e equal to Z^H (x - Z g) (the d-step's
    normal equation at d = g), the same multiplier for two values of sigma.  With the sign as
    printed (e <- e + g - d) the same iteration diverges."""
    rng = np.random.default_rng(2)
    N, L, S, P = 16, 3, 2, 5
    z = rng.standard_normal((L, S, N, N)) * (rng.random((L, S, N, N)) < 0.1)
    x = rng.standard_normal((S, N, N))
    g0 = admm.project_filters(rng.standard_normal((L, N, N)), P)
    mult = []
    for sigma in (100.0, 1000.0):
        g, e = g0.copy(), np.zeros_like(g0)
        for _ in range(2000):
            d, g, e = fast.dict_update(x, z, g, e, sigma, P)
        assert rel(d, g) < 1e-10
        assert np.allclose(np.sqrt(np.sum(admm.crop_filters(g, P) ** 2, axis=(1, 2))), 1.0)
        mask = admm.embed_filters(np.ones((1, P, P)), N)[0] != 0
        assert np.all(g[:, ~mask] == 0)
        r = x - np.stack([sum(admm.circconv2(z[l, s], g[l]) for l in range(L)) for s in range(S)])
        zh_r = np.stack([sum(admm.circcorr2(r[s], z[l, s]) for s in range(S)) for l in range(L)])
        assert rel(sigma * e, zh_r) < 1e-8
        mult.append(sigma * e)
    assert rel(mult[0], mult[1]) < 1e-8
    g, e = g0.copy(), np.zeros_like(g0)
    for _ in range(300):
        d, g_new, _ = fast.dict_update(x, z, g, e, 100.0, P)
        e = e + g_new - d
        g = g_new
    assert np.linalg.norm(e) > 1e6 * np.linalg.norm(mult[0]) / 100.0


def test_convdict3d_x_update_is_stationary(cd3):
    """3D case of the x-update: beta/2 ||y - Hx||^2 + 1/2 ||D~z - x||^2 with D~ the circular 3D
    convolution is minimised (first-order term zero, quadratic term as the Hessian predicts)."""
    C, N, S, L = cd3["C"], cd3["N"], cd3["S"], cd3["L"]
    z = cd3["z"]
    x, _, _, _ = admm.convdict3d_step(C, z, cd3["t"], cd3["u"])
    de = admm.embed_filters3d(cd3["d3"], N, S)
    Dz = sum(conv3_brute(z[l], de[l]) for l in range(L))
    f = lambda xx: 0.5 * C.beta * float(np.sum((cd3["y"] - admm.forward_H(xx, cd3["h"])) ** 2)) + \
        0.5 * float(np.sum((Dz - xx) ** 2))
    f0 = f(x)
    rng = np.random.default_rng(4)
    for _ in range(4):
        dx = 1e-2 * rng.standard_normal(x.shape)
        quad = 0.5 * C.beta * float(np.sum(admm.forward_H(dx, cd3["h"]) ** 2)) + 0.5 * float(np.sum(dx * dx))
        assert abs(f(x + dx) - f0 - quad) < 1e-9 * max(1.0, abs(f0))

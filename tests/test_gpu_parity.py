"""CUDA path vs the FP64 oracle through the C ABI.  GPU only.

Tolerances: relative L2 per step <= 1e-5 and on the final x <= 1e-4 for the
complex64 path (FP64-formed factor and data term); <= 1e-10 for the FP64 path."""
import numpy as np
import pytest

from oracle import admm, fast
from paper_2006_08303_gb300 import inputs

pytestmark = pytest.mark.gpu

STEP_TOL = {"f32": 1e-5, "f64": 1e-10}
FINAL_TOL = {"f32": 1e-4, "f64": 1e-10}


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    return torch


def tdev(torch, a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32 if dtype == "f32" else torch.float64).cuda()


def make_plan(torch, h, y, prior, lam, rho, beta, dtype, **kw):
    from paper_2006_08303_gb300 import api
    K, M, N, _ = h.shape
    P = api.Plan(N, K, M, dtype, **kw)
    P.set_prior(prior, lam, rho, beta)
    P.set_psfs(tdev(torch, h, dtype))
    P.set_measurements(tdev(torch, y, dtype))
    return P


def problem(seed, N, K, M, kind="gauss"):
    """Rectangles + Gaussian PSFs (kind 'gauss') or spectral image + disk-plus-Gaussian PSFs ('disk')."""
    rng = np.random.default_rng(seed)
    if kind == "gauss":
        x = inputs.rectangles_image(rng, N, M, n_rect=6)
        h = inputs.gaussian_psf_bank(N, K, M)
    else:
        x = inputs.spectral_image(rng, N, M)
        h = inputs.disk_gaussian_psf_bank(N, K, M)
    y, _ = inputs.measure(rng, x, h, 30.0)
    return rng, h, y


def u_err(ug, u1, x1, prior):
    """u' = u + w - soft(w + u, tau) is evaluated on w = T x at the scale of w, so its error is measured
    relative to max(||u'||, ||T x||) (the update is 1-Lipschitz in w)."""
    fwd, _ = admm.PRIORS[prior]
    scale = max(np.linalg.norm(u1), np.linalg.norm(fwd(x1)))
    return float(np.linalg.norm(ug - u1) / scale)


def oracle_states(h, y, prior, lam, rho, ls, naive):
    """Oracle iterates (t^l, u^l) at the requested l and the oracle's next step from each."""
    mod = admm if naive else fast
    S = mod.analysis_setup(h, y, prior, lam, rho, 1.0)
    K, M, N, _ = h.shape
    nc = 2 if prior in ("tv", "tv_iso") else 1
    t = np.zeros((M, nc, N, N))
    u = np.zeros_like(t)
    out = []
    for l in range(max(ls) + 1):
        x1, t1, u1, _ = mod.analysis_step(S, t, u)
        if l in ls:
            out.append((l, t, u, x1, u1))
        t, u = t1, u1
    return out


STEP_CASES = [
    # prior, N, K, M, dtype, lam, rho, kind, states l
    ("tv", 64, 3, 3, "f64", 1e-2, 1.0, "gauss", (0, 1, 10, 49)),
    ("tv", 64, 3, 3, "f32", 1e-2, 1.0, "gauss", (0, 1, 10, 49)),
    ("dct8", 64, 2, 3, "f32", 1e-3, 1e-2, "disk", (0, 1, 10, 40)),
    ("l1", 64, 3, 2, "f32", 1e-2, 0.5, "gauss", (0, 1, 10)),
    ("dct8", 128, 3, 3, "f64", 1e-3, 0.1, "disk", (0, 10)),
    ("tv", 256, 5, 5, "f32", 1e-2, 1.0, "disk", (0, 1, 10, 30)),
    ("dct8", 256, 10, 10, "f32", 1e-3, 1e-2, "disk", (0, 1, 10, 30)),
    ("tv", 128, 1, 3, "f32", 1e-2, 1.0, "gauss", (0, 10)),     # K < M: rank-deficient Lambda^H Lambda
    ("tv", 128, 5, 2, "f32", 1e-2, 1.0, "gauss", (0, 10)),     # K > M
    ("l1", 2048, 1, 1, "f32", 1e-2, 1.0, "gauss", (0, 5)),     # largest N
    ("tv", 1024, 3, 3, "f32", 1e-2, 1.0, "gauss", (0, 5)),
    ("tv_iso", 64, 3, 3, "f64", 1e-2, 1.0, "gauss", (0, 1, 10, 49)),   # isotropic TV (reading R20)
    ("tv_iso", 64, 3, 3, "f32", 1e-2, 1.0, "gauss", (0, 1, 10, 49)),
    ("tv_iso", 512, 5, 5, "f32", 1e-2, 1.0, "disk", (0, 1, 10)),
    # Kronecker Symmlet-8 (x) channel DCT (Section V, readings R24-R26)
    ("wdct", 64, 3, 3, "f64", 1e-2, 0.5, "disk", (0, 1, 10, 40)),
    ("wdct", 64, 3, 3, "f32", 1e-2, 0.5, "disk", (0, 1, 10, 40)),
    ("wdct", 512, 10, 10, "f32", 1e-3, 1e-2, "disk", (0, 1, 10)),
    ("wdct", 128, 2, 16, "f32", 1e-2, 0.5, "gauss", (0, 5)),    # 16 channels
    ("wdct", 256, 1, 1, "f32", 1e-2, 0.5, "gauss", (0, 5)),     # one channel (C = 1)
]


@pytest.mark.parametrize("prior,N,K,M,dtype,lam,rho,kind,ls", STEP_CASES)
def test_step_parity_on_oracle_states(torch, prior, N, K, M, dtype, lam, rho, kind, ls):
    """One GPU iteration of Alg. 1 from the oracle's (t^l, u^l) against the oracle's iteration l+1:
    x (Eq. solx_Trans_DFT) and u (Eqs. solt_trans, subu_trans), relative L2 <= 1e-5 (complex64 path)."""
    rng, h, y = problem(100 + N + M + K, N, K, M, kind)
    P = make_plan(torch, h, y, prior, lam, rho, 1.0, dtype)
    for l, t, u, x1, u1 in oracle_states(h, y, prior, lam, rho, ls, naive=(N <= 64)):
        P.state_import(tdev(torch, t, dtype), tdev(torch, u, dtype))
        assert P.iterate(1) == 1
        xg = P.get_x().double().cpu().numpy()
        ug = P.get_u().double().cpu().numpy()
        ex = rel(xg, x1)
        eu = u_err(ug, u1, x1, prior)
        assert ex <= STEP_TOL[dtype], (l, ex)
        assert eu <= STEP_TOL[dtype], (l, eu)
    P.close()


@pytest.mark.parametrize("column_pass", [1, 2])
@pytest.mark.parametrize("prior,N,K,M,kind", [("tv", 128, 3, 3, "gauss"), ("dct8", 256, 10, 10, "disk"),
                                               ("tv", 64, 2, 16, "gauss")])
def test_column_pass_forms(torch, column_pass, prior, N, K, M, kind):
    """The fused (cluster) and split column passes both give Alg. 1's iterates: one step from oracle
    states within 1e-5 (f32), for M up to the 16-channel limit."""
    rng, h, y = problem(300 + N + M, N, K, M, kind)
    lam, rho = (1e-2, 1.0) if prior == "tv" else (1e-3, 1e-2)
    P = make_plan(torch, h, y, prior, lam, rho, 1.0, "f32", column_pass=column_pass)
    assert P.config()["column_pass"] == {1: "fused", 2: "split"}[column_pass]
    for l, t, u, x1, u1 in oracle_states(h, y, prior, lam, rho, (0, 5), naive=(N <= 64)):
        P.state_import(tdev(torch, t, "f32"), tdev(torch, u, "f32"))
        P.iterate(1)
        assert rel(P.get_x().double().cpu().numpy(), x1) <= 1e-5
        assert u_err(P.get_u().double().cpu().numpy(), u1, x1, prior) <= 1e-5
    P.close()


@pytest.mark.parametrize("prior_fft", [8, 16])
@pytest.mark.parametrize("prior,N,K,M,kind", [("tv", 256, 3, 3, "gauss"), ("dct8", 512, 4, 4, "disk"),
                                               ("tv_iso", 512, 3, 3, "gauss"), ("l1", 1024, 2, 2, "gauss"),
                                               ("tv", 1024, 2, 2, "gauss")])
def test_prior_pass_fft_widths(torch, prior_fft, prior, N, K, M, kind):
    """Both prior-pass kernels the autotuner chooses between (8 or 16 FFT elements per thread)
    give Alg. 1's iterates: one step from oracle states within 1e-5, and the plan reports the width
    it was given."""
    rng, h, y = problem(400 + N + M, N, K, M, kind)
    lam, rho = (1e-3, 1e-2) if prior == "dct8" else (1e-2, 1.0)
    P = make_plan(torch, h, y, prior, lam, rho, 1.0, "f32", prior_fft=prior_fft)
    assert P.config()["prior_fft_elems"] == prior_fft
    for l, t, u, x1, u1 in oracle_states(h, y, prior, lam, rho, (0, 5), naive=False):
        P.state_import(tdev(torch, t, "f32"), tdev(torch, u, "f32"))
        P.iterate(1)
        assert rel(P.get_x().double().cpu().numpy(), x1) <= 1e-5
        assert u_err(P.get_u().double().cpu().numpy(), u1, x1, prior) <= 1e-5
    P.close()


def test_autotuned_prior_width_is_reported(torch):
    """With everything autotuned the plan runs one of the two widths and reports it; an invalid
    width is refused at plan creation."""
    from paper_2006_08303_gb300 import api
    rng, h, y = problem(7, 512, 2, 2, "disk")
    P = make_plan(torch, h, y, "dct8", 1e-3, 1e-2, 1.0, "f32")
    assert P.config()["prior_fft_elems"] in (8, 16)
    P.close()
    with pytest.raises(api.CipError):
        api.Plan(512, 2, 2, "f32", prior_fft=4)


@pytest.mark.parametrize("prior,N,rho", [("tv", 64, 1.0), ("dct8", 64, 0.3), ("l1", 128, 0.5)])
def test_step_random_state(torch, prior, N, rho):
    """Property at white-noise (t, u): the complex64 step stays within 1e-4 of the FP64 oracle."""
    rng, h, y = problem(7 + N, N, 3, 3, "gauss")
    t, u = inputs.random_state(rng, prior, 3, N, scale=0.05)
    mod = admm if N <= 64 else fast
    S = mod.analysis_setup(h, y, prior, 1e-2, rho, 1.0)
    x1, _, u1, _ = mod.analysis_step(S, t, u)
    P = make_plan(torch, h, y, prior, 1e-2, rho, 1.0, "f32")
    P.state_import(tdev(torch, t, "f32"), tdev(torch, u, "f32"))
    P.iterate(1)
    assert rel(P.get_x().double().cpu().numpy(), x1) <= 1e-4
    assert u_err(P.get_u().double().cpu().numpy(), u1, x1, prior) <= 1e-4
    P.close()


@pytest.fixture(scope="module")
def spectral_full():
    """The 512 x 512 x 10 spectral-imaging DCT workload and its FP64 oracle run (fast form)."""
    Pr = inputs.spectral_dct()
    S = fast.analysis_setup(Pr.h, Pr.y, Pr.prior, Pr.lam, Pr.rho, Pr.beta)
    t = np.zeros((Pr.M, 1, Pr.N, Pr.N))
    u = np.zeros_like(t)
    keep = {}
    x = None
    for l in range(Pr.iters):
        if l in (0, 10, 100):
            keep[l] = (t, u)
        x, t, u, _ = fast.analysis_step(S, t, u)
    return Pr, S, keep, x, u


def test_full_size_step_parity(torch, spectral_full):
    """512 x 512 x 10 DCT workload in the benchmark's launch configuration: one step from the oracle's
    states l = 0, 10, 100 within 1e-5."""
    Pr, S, keep, _, _ = spectral_full
    P = make_plan(torch, Pr.h, Pr.y, Pr.prior, Pr.lam, Pr.rho, Pr.beta, "f32")
    for l, (t, u) in keep.items():
        x1, _, u1, _ = fast.analysis_step(S, t, u)
        P.state_import(tdev(torch, t, "f32"), tdev(torch, u, "f32"))
        P.iterate(1)
        ex = rel(P.get_x().double().cpu().numpy(), x1)
        eu = u_err(P.get_u().double().cpu().numpy(), u1, x1, Pr.prior)
        assert ex <= 1e-5 and eu <= 1e-5, (l, ex, eu)
    P.close()


def test_full_size_final_x(torch, spectral_full):
    """512 x 512 x 10 DCT workload: x after 200 free-running GPU iterations within 1e-4 of the oracle's."""
    Pr, S, keep, x_ref, u_ref = spectral_full
    P = make_plan(torch, Pr.h, Pr.y, Pr.prior, Pr.lam, Pr.rho, Pr.beta, "f32")
    assert P.iterate(Pr.iters) == Pr.iters
    xg = P.get_x().double().cpu().numpy()
    P.close()
    assert rel(xg, x_ref) <= 1e-4, rel(xg, x_ref)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_tiny_tv_full_run(torch, dtype):
    """64x64x3 TV instance, 50 iterations of Alg. 1 from t = u = 0."""
    Pr = inputs.tiny_tv()
    S = admm.analysis_setup(Pr.h, Pr.y, Pr.prior, Pr.lam, Pr.rho, Pr.beta)
    x_ref, t_ref, u_ref, hist = admm.run_analysis(S, Pr.iters, keep_history=True)
    P = make_plan(torch, Pr.h, Pr.y, Pr.prior, Pr.lam, Pr.rho, Pr.beta, dtype)
    assert P.iterate(Pr.iters) == Pr.iters
    xg = P.get_x().double().cpu().numpy()
    ug = P.get_u().double().cpu().numpy()
    r, s = P.residuals()
    P.close()
    assert rel(xg, x_ref) <= FINAL_TOL[dtype]
    assert rel(ug, u_ref) <= 10 * FINAL_TOL[dtype]
    assert abs(r - hist[-1].r_rel) <= 1e-3 * hist[-1].r_rel + 1e-7
    assert abs(s - hist[-1].s_rel) <= 1e-3 * hist[-1].s_rel + 1e-7


def test_first_iterate_is_factor_times_rhs(torch):
    """x^1 from t = u = 0 is F^H Psi^{-1} beta Lambda^H F y: checks setup (PSF DFT, factor incl. the
    DC pseudo-inverse of TV, data term) through the C ABI."""
    Pr = inputs.tiny_tv(iters=1)
    S = admm.analysis_setup(Pr.h, Pr.y, "tv", Pr.lam, Pr.rho, Pr.beta)
    x1 = admm.x_update(S, np.zeros((3, 2, 64, 64)), np.zeros((3, 2, 64, 64)))
    for dtype in ("f64", "f32"):
        P = make_plan(torch, Pr.h, Pr.y, "tv", Pr.lam, Pr.rho, Pr.beta, dtype)
        P.iterate(1)
        assert rel(P.get_x().double().cpu().numpy(), x1) <= STEP_TOL[dtype]
        P.close()


def test_host_pointers_match_device_pointers(torch):
    """The C ABI accepts host buffers (copied in stream order) with identical results."""
    from paper_2006_08303_gb300 import api
    Pr = inputs.tiny_tv(iters=5)
    Pd = make_plan(torch, Pr.h, Pr.y, "tv", Pr.lam, Pr.rho, Pr.beta, "f32")
    Pd.iterate(5)
    xd = Pd.get_x().cpu().numpy()
    Ph = api.Plan(Pr.N, Pr.K, Pr.M, "f32")
    Ph.set_prior("tv", Pr.lam, Pr.rho, Pr.beta)
    Ph.set_psfs(Pr.h.astype(np.float32))
    Ph.set_measurements(torch.as_tensor(Pr.y, dtype=torch.float32).pin_memory())
    Ph.iterate(5)
    xh = np.empty((Pr.M, Pr.N, Pr.N), np.float32)
    Ph.get_x(xh)
    assert np.array_equal(xd, xh)
    Pd.close()
    Ph.close()


def test_checkpoint_resume_is_bitwise(torch):
    Pr = inputs.tiny_tv(iters=20)
    P = make_plan(torch, Pr.h, Pr.y, "tv", Pr.lam, Pr.rho, Pr.beta, "f32")
    P.iterate(7)
    ck = P.state_export()
    P.iterate(9)
    xa = P.get_x().cpu().numpy()
    P.state_restore(ck)
    assert P.iteration() == 7
    P.iterate(9)
    xb = P.get_x().cpu().numpy()
    P.close()
    assert np.array_equal(xa, xb)


def test_run_is_deterministic(torch):
    Pr = inputs.tiny_tv(iters=15)
    xs = []
    for _ in range(2):
        P = make_plan(torch, Pr.h, Pr.y, "tv", Pr.lam, Pr.rho, Pr.beta, "f32")
        P.iterate(15)
        xs.append(P.get_x().cpu().numpy())
        xs.append(np.array(P.residuals()))
        P.close()
    assert np.array_equal(xs[0], xs[2]) and np.array_equal(xs[1], xs[3])


def test_tolerance_stop_matches_oracle(torch):
    """cip_iterate with tol > 0 stops at the first check (every 10 iterations) where both relative
    residuals (Eq. paramS quantities) are below tol, like the oracle evaluated at the same checks."""
    Pr = inputs.tiny_tv(iters=300)
    S = fast.analysis_setup(Pr.h, Pr.y, Pr.prior, Pr.lam, Pr.rho, Pr.beta)
    tol = 1e-3
    t = np.zeros((3, 2, 64, 64))
    u = np.zeros_like(t)
    n_or = None
    for it in range(1, 301):
        x, t_new, u_new, w = fast.analysis_step(S, t, u)
        if it % 10 == 0:
            r = np.linalg.norm(w - t_new) / max(np.linalg.norm(w), np.linalg.norm(t_new))
            s = np.linalg.norm(t_new - t) / np.linalg.norm(u_new)
            if r < tol and s < tol:
                n_or = it
                break
        t, u = t_new, u_new
    assert n_or is not None
    P = make_plan(torch, Pr.h, Pr.y, Pr.prior, Pr.lam, Pr.rho, Pr.beta, "f64")
    n = P.iterate(300, tol=tol)
    P.close()
    assert n == n_or


def test_errors_are_statuses(torch):
    from paper_2006_08303_gb300 import api
    P = api.Plan(64, 2, 2, "f32")
    with pytest.raises(api.CipError) as e:
        P.iterate(1)
    assert e.value.status == 5
    P.set_prior("tv", 1e-2, 1.0, 1.0)
    with pytest.raises(api.CipError):
        P.set_measurements(torch.zeros((2, 64, 64), device="cuda"))
    with pytest.raises(api.CipError):
        P.set_prior("tv", -1.0, 1.0, 1.0)
    P.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_isotropic_tv_full_run(torch, dtype):
    """Isotropic TV (coupled shrinkage, reading R20): 50 free-running iterations of the tiny
    instance from t = u = 0 against the FP64 oracle, final x within FINAL_TOL."""
    P = inputs.tiny_tv(dtype="f64")
    S = fast.analysis_setup(P.h, P.y, "tv_iso", P.lam, P.rho, P.beta)
    x_or, _, _, _, _ = fast.run_analysis(S, 50)
    plan = make_plan(torch, P.h, P.y, "tv_iso", P.lam, P.rho, P.beta, dtype)
    plan.iterate(50)
    x = plan.get_x().double().cpu().numpy()
    S_an = fast.analysis_setup(P.h, P.y, "tv", P.lam, P.rho, P.beta)
    x_an, _, _, _, _ = fast.run_analysis(S_an, 50)
    assert rel(x, x_or) <= FINAL_TOL[dtype], rel(x, x_or)
    assert rel(x_an, x_or) > 100 * FINAL_TOL["f32"]  # the isotropic iterates really differ
    plan.close()


@pytest.mark.parametrize("dtype,N,M,iters", [("f64", 64, 3, 50), ("f32", 128, 5, 60)])
def test_wdct_full_run(torch, dtype, N, M, iters):
    """Kronecker wavelet (x) DCT prior: free-running iterations from t = u = 0 against the FP64
    oracle, final x within FINAL_TOL (1e-9 for the FP64 path: the wavelet chain rounds more often)."""
    rng, h, y = problem(77 + N, N, M, M, "disk")
    S = fast.analysis_setup(h, y, "wdct", 1e-2, 0.5, 1.0)
    x_or = fast.run_analysis(S, iters)[0]
    P = make_plan(torch, h, y, "wdct", 1e-2, 0.5, 1.0, dtype)
    P.iterate(iters)
    x = P.get_x().double().cpu().numpy()
    P.close()
    assert rel(x, x_or) <= (1e-9 if dtype == "f64" else FINAL_TOL["f32"]), rel(x, x_or)


def test_wdct_tolerance_stop_matches_oracle(torch):
    """The residual partial sums of the wavelet prior's shrinkage kernel: cip_iterate with tol stops
    at the same check as the oracle (relative residuals of Eq. paramS, every 10 iterations)."""
    rng, h, y = problem(5, 64, 3, 3, "gauss")
    S = fast.analysis_setup(h, y, "wdct", 1e-2, 0.5, 1.0)
    tol = 1e-3
    t = np.zeros((3, 1, 64, 64))
    u = np.zeros_like(t)
    n_or = None
    for it in range(1, 301):
        x, t_new, u_new, w = fast.analysis_step(S, t, u)
        if it % 10 == 0:
            r = np.linalg.norm(w - t_new) / max(np.linalg.norm(w), np.linalg.norm(t_new))
            s = np.linalg.norm(t_new - t) / np.linalg.norm(u_new)
            if r < tol and s < tol:
                n_or = it
                break
        t, u = t_new, u_new
    assert n_or is not None
    P = make_plan(torch, h, y, "wdct", 1e-2, 0.5, 1.0, "f64")
    n = P.iterate(300, tol=tol)
    r_rel, s_rel = P.residuals()
    P.close()
    assert n == n_or
    assert r_rel < tol and s_rel < tol

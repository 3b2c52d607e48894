"""CUDA path vs the FP64 oracle through the C ABI.  GPU only.

Tolerances: relative L2 per step <= 1e-5 and on the final x <= 1e-4 for the
complex64 path (FP64-formed factor); <= 1e-10 for the FP64 path."""
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


def problem(seed, N, K, M, unit_sum=True):
    rng = np.random.default_rng(seed)
    x = inputs.rectangles_image(rng, N, M, n_rect=6)
    if unit_sum:
        h = inputs.gaussian_psf_bank(N, K, M)
    else:
        h = rng.uniform(0, 1, (K, M, N, N)) * (rng.random((K, M, N, N)) < 0.02)
        h[:, :, 0, 0] += 1.0
    y, _ = inputs.measure(rng, x, h, 30.0)
    return rng, h, y


CASES = [
    # prior, N, K, M, dtype, lam, rho
    ("tv", 64, 3, 3, "f64", 1e-2, 1.0),
    ("tv", 64, 3, 3, "f32", 1e-2, 1.0),
    ("dct8", 64, 2, 3, "f32", 1e-3, 0.1),
    ("l1", 64, 3, 2, "f32", 1e-2, 0.5),
    ("dct8", 128, 3, 3, "f64", 1e-3, 0.1),
    ("tv", 256, 5, 5, "f32", 1e-2, 1.0),
    ("dct8", 256, 4, 10, "f32", 1e-3, 1e-2),
    ("tv", 1024, 3, 3, "f32", 1e-2, 1.0),
    ("l1", 2048, 1, 1, "f32", 1e-2, 1.0),
]


@pytest.mark.parametrize("prior,N,K,M,dtype,lam,rho", CASES)
def test_one_step_from_imported_state(torch, prior, N, K, M, dtype, lam, rho):
    """Alg. 1 one iteration from a random (t, u): x (Eq. solx_Trans_DFT), u (Eqs. solt_trans, subu_trans)."""
    rng, h, y = problem(100 + N + M, N, K, M, unit_sum=(prior == "tv"))
    t, u = inputs.random_state(rng, prior, M, N, scale=0.05)
    if N <= 64:
        S = admm.analysis_setup(h, y, prior, lam, rho, 1.0)
        x1, t1, u1, _ = admm.analysis_step(S, t, u)
    else:
        S = fast.analysis_setup(h, y, prior, lam, rho, 1.0)
        x1, t1, u1, _ = fast.analysis_step(S, t, u)
    P = make_plan(torch, h, y, prior, lam, rho, 1.0, dtype)
    P.state_import(tdev(torch, t, dtype), tdev(torch, u, dtype))
    assert P.iterate(1) == 1
    xg = P.get_x().double().cpu().numpy()
    ug = P.get_u().double().cpu().numpy()
    P.close()
    assert rel(xg, x1) <= STEP_TOL[dtype], rel(xg, x1)
    assert rel(ug, u1) <= STEP_TOL[dtype], rel(ug, u1)


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
    DC pseudo-inverse of TV, rhs) through the C ABI."""
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
    Pd.close(); Ph.close()


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
    # oracle: residuals at iterations 10, 20, ...
    t = np.zeros((3, 2, 64, 64)); u = np.zeros_like(t)
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

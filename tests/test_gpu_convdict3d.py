"""Convolutional dictionary with 3D filters (Section IV-B, 3D case) on the GPU vs the FP64 oracle.

One GPU iteration from the oracle's (z^l, t^l, u^l) is compared with the oracle's iteration l+1
(x: Eq. solx_synt_DFT with the channel DFT of its last term; z: Eq. solz_DFT_SM in every 3D bin;
u: Eqs. softADMM, subu_dic) at relative L2 <= 1e-5 (complex64) / 1e-10 (FP64), and the
free-running x after the stated iterations at <= 1e-4.  With one channel tap (Q = 1) the 3D
dictionary is the 2D one, which the library computes by a different kernel.  GPU only."""
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


def plan3(torch, pr, dtype="f32", d3=None):
    from paper_2006_08303_gb300 import api
    tdt = torch.float32 if dtype == "f32" else torch.float64
    f = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=tdt).cuda()
    P = api.Plan(pr.N, pr.K, pr.M, dtype)
    P.set_prior("convdict", pr.lam, pr.rho, pr.beta)
    P.set_dictionary_3d(f(pr.filters if d3 is None else d3))
    P.set_psfs(f(pr.h))
    P.set_measurements(f(pr.y))
    return P, f


@pytest.mark.parametrize("dtype,tol", [("f32", 1e-5), ("f64", 1e-10)])
def test_convdict3d_step_parity(torch, dtype, tol):
    pr = inputs.convdict3d_problem(N=64, M=4, L=3, Q=3, P=5)
    C = fast.convdict3d_setup(pr.h, pr.y, pr.filters, pr.lam, pr.rho, pr.beta)
    P, f = plan3(torch, pr, dtype)
    L, M, N = pr.filters.shape[0], pr.M, pr.N
    z = np.zeros((L, M, N, N)); t = np.zeros_like(z); u = np.zeros_like(z)
    for l in range(6):
        x1, z1, t1, u1 = fast.convdict3d_step(C, z, t, u)
        if l in (0, 1, 5):
            P.state_import_coefficients(f(gl(z)), f(gl(t)), f(gl(u)))
            P.iterate(1)
            xg = P.get_x().double().cpu().numpy()
            zg = P.get_coefficients().double().cpu().numpy()
            ug = P.get_u().double().cpu().numpy()
            assert rel(xg, x1) <= tol, (l, rel(xg, x1))
            assert rel(zg, gl(z1)) <= tol, (l, rel(zg, gl(z1)))
            scale = max(np.linalg.norm(u1), np.linalg.norm(z1))
            assert np.linalg.norm(ug - gl(u1)) / scale <= tol, (l, np.linalg.norm(ug - gl(u1)) / scale)
        z, t, u = z1, t1, u1
    P.close()


def test_convdict3d_free_running_256x256x16(torch):
    """The spectral-experiment shape of Section V (6 filters of 5 channel taps, here 11 x 11 in the
    plane) at 256 x 256 x 16: 30 free-running iterations from z = t = u = 0."""
    pr = inputs.convdict3d_problem(N=256, M=16, L=6, Q=5, P=11, iters=30)
    C = fast.convdict3d_setup(pr.h, pr.y, pr.filters, pr.lam, pr.rho, pr.beta)
    z = np.zeros((6, 16, 256, 256)); t = np.zeros_like(z); u = np.zeros_like(z)
    for _ in range(pr.iters):
        x_or, z, t, u = fast.convdict3d_step(C, z, t, u)
    P, _ = plan3(torch, pr)
    P.iterate(pr.iters)
    xg = P.get_x().double().cpu().numpy()
    zg = P.get_coefficients().double().cpu().numpy()
    P.close()
    assert rel(xg, x_or) <= 1e-4, rel(xg, x_or)
    assert rel(zg, gl(z)) <= 1e-3, rel(zg, gl(z))


def test_convdict3d_one_channel_tap_is_the_2d_dictionary(torch):
    """Q = 1: the 3D kernel (channel DFTs around a per-3D-bin solve) against the 2D kernel (per
    channel solve) on the same 2D filters, 20 free-running iterations."""
    from paper_2006_08303_gb300 import api
    pr = inputs.convdict3d_problem(N=128, M=5, L=4, Q=1, P=7)
    P3, f = plan3(torch, pr)
    P3.iterate(20)
    x3 = P3.get_x().double().cpu().numpy()
    z3 = P3.get_coefficients().double().cpu().numpy()
    P3.close()
    P2 = api.Plan(pr.N, pr.K, pr.M, "f32")
    P2.set_prior("convdict", pr.lam, pr.rho, pr.beta)
    P2.set_dictionary(f(pr.filters[:, 0]))
    P2.set_psfs(f(pr.h))
    P2.set_measurements(f(pr.y))
    P2.iterate(20)
    x2 = P2.get_x().double().cpu().numpy()
    z2 = P2.get_coefficients().double().cpu().numpy()
    P2.close()
    assert rel(x3, x2) <= 1e-5, rel(x3, x2)
    assert rel(z3, z2) <= 1e-4, rel(z3, z2)


def test_convdict3d_rejections(torch):
    """Host-side checks: depth beyond the channel count; the 2D-only options."""
    from paper_2006_08303_gb300 import api
    pr = inputs.convdict3d_problem(N=64, M=4, L=3, Q=3, P=5)
    f = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32).cuda()
    P = api.Plan(pr.N, pr.K, pr.M, "f32")
    P.set_prior("convdict", pr.lam, pr.rho, pr.beta)
    with pytest.raises(api.CipError):
        P.set_dictionary_3d(f(np.zeros((3, 5, 5, 5))))  # Q = 5 > M = 4
    P.set_dictionary_3d(f(pr.filters))
    with pytest.raises(api.CipError):
        P.set_code_gradient_weight(0.1)
    with pytest.raises(api.CipError):
        P.set_dictionary_learning(10.0)
    P.close()

"""Gradients of L = w^T K~ z (pttk_grad and the torch.autograd.Function) against the oracle's
analytic gradients on the same TT, central finite differences (h = 1e-6, FP64) and, at
nu = 3/2, the dense FP64 kernel gradient. Tolerances: FP64 path 1e-10 vs the oracle's
analytic gradient and 1e-7 vs finite differences; FP32 path 1e-4 relative."""
import dataclasses
import math

import numpy as np
import pytest

import oracle.pttk_oracle as o
from paper_2406_06344_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_06344_gb300 import pttk as P
    P.load()
    return torch, P


_tts = {}


def _tt(P, w):
    key = (w.name, w.n, w.d)
    if key not in _tts:
        _tts[key] = P.TT.build_offline(w.kernel, w.d, w.src_box, w.tgt_box, w.dtheta, w.theta_box, w.n, w.tol, "fp64")
    return _tts[key]


CASES = [("c1", None), ("c2", None), ("c3", 6)]


def _case(name, n):
    w = W.WORKLOADS[name]
    return dataclasses.replace(w, n=n) if n else w


@pytest.mark.parametrize("name,n", CASES)
def test_grad_fp64_matches_oracle_and_fd(env, name, n):
    torch, P = env
    w = _case(name, n)
    tt = _tt(P, w)
    gc = tt.cores()
    X, Y = W.sources(w, 400), W.targets(w, 350)
    wv, _ = W.weights(400)
    _, zv = W.weights(350)
    th = W.thetas(w, 1)[0]
    dev = lambda a: torch.tensor(a, device="cuda", dtype=torch.float64)
    L, dth, dX = P.grad(tt, th, dev(X), dev(Y), dev(wv), dev(zv), "fp64")
    Lo = o.loss(*o.instantiate(gc, w.d, w.dtheta, w.mode_boxes(), th, X, Y), wv, zv)
    gth, gX = o.loss_grad(gc, w.d, w.dtheta, w.mode_boxes(), th, X, Y, wv, zv)
    assert L == pytest.approx(Lo, rel=1e-12)
    assert np.allclose(dth, gth, rtol=1e-10, atol=1e-12 * abs(Lo))
    assert np.linalg.norm(dX.cpu().numpy() - gX) <= 1e-10 * np.linalg.norm(gX)
    # central differences of the GPU loss itself
    h = 1e-6
    for j in range(w.dtheta):
        e = np.zeros(w.dtheta)
        e[j] = h
        Lp = P.grad(tt, th + e, dev(X), dev(Y), dev(wv), dev(zv), "fp64", want_dX=False)[0]
        Lm = P.grad(tt, th - e, dev(X), dev(Y), dev(wv), dev(zv), "fp64", want_dX=False)[0]
        assert dth[j] == pytest.approx((Lp - Lm) / (2 * h), rel=1e-7, abs=1e-9)
    rng = np.random.default_rng(4)
    v = rng.standard_normal(X.shape) * 0.01
    Lp = P.grad(tt, th, dev(X + h * v), dev(Y), dev(wv), dev(zv), "fp64", want_dX=False)[0]
    Lm = P.grad(tt, th, dev(X - h * v), dev(Y), dev(wv), dev(zv), "fp64", want_dX=False)[0]
    assert float(np.sum(dX.cpu().numpy() * v)) == pytest.approx((Lp - Lm) / (2 * h), rel=1e-6, abs=1e-9)


@pytest.mark.parametrize("form", ["fp32", "tf32x3", "fp16x3"])
@pytest.mark.parametrize("name,n", CASES)
def test_grad_fp32_forms(env, form, name, n):
    torch, P = env
    w = _case(name, n)
    tt = _tt(P, w)
    gc = tt.cores()
    X, Y = W.sources(w, 3000), W.targets(w, 2500)
    wv, _ = W.weights(3000)
    _, zv = W.weights(2500)
    th = W.thetas(w, 1)[0]
    f32 = lambda a: torch.tensor(a, device="cuda", dtype=torch.float32)
    Xf = f32(X)
    L, dth, dX = P.grad(tt, th, Xf, f32(Y), f32(wv), f32(zv), form)
    X32, Y32 = Xf.double().cpu().numpy(), f32(Y).double().cpu().numpy()
    w32, z32 = f32(wv).double().cpu().numpy(), f32(zv).double().cpu().numpy()
    gth, gX = o.loss_grad(gc, w.d, w.dtheta, w.mode_boxes(), th, X32, Y32, w32, z32)
    Lo = o.loss(*o.instantiate(gc, w.d, w.dtheta, w.mode_boxes(), th, X32, Y32), w32, z32)
    assert L == pytest.approx(Lo, rel=1e-4)
    assert np.linalg.norm(dth - gth) <= 1e-4 * np.linalg.norm(gth)
    assert np.linalg.norm(dX.double().cpu().numpy() - gX) <= 1e-4 * np.linalg.norm(gX)


def test_autograd_function_and_dense_matern32_gradient(env):
    """torch.autograd through PTTKLoss at nu = 3/2 (d = 1): gradients against the dense FP64
    kernel gradient dk/dl = a^2 e^{-a}/l, grad_x k = -3 e^{-a}(x - y)/l^2, a = sqrt(3) r / l."""
    torch, P = env
    w = dataclasses.replace(W.C2, d=1, dtheta=1, n=24, src_box=((0.0, 1.0),), tgt_box=((2.0, 3.0),),
                            theta_box=((0.5, 2.0),))
    tt = _tt(P, w)
    rng = np.random.default_rng(5)
    X, Y = rng.random((500, 1)), 2 + rng.random((400, 1))
    wv, zv = rng.standard_normal(500), rng.standard_normal(400)
    l = 1.3
    theta = torch.tensor([l], dtype=torch.float64, requires_grad=True)
    Xd = torch.tensor(X, device="cuda", requires_grad=True)
    L = P.pttk_loss(theta, Xd, torch.tensor(Y, device="cuda"), torch.tensor(wv, device="cuda"),
                    torch.tensor(zv, device="cuda"), tt, "fp64")
    (2.0 * L).backward()
    diff = X[:, None, 0] - Y[None, :, 0]
    a = math.sqrt(3) * np.abs(diff) / l
    dK_dl = a ** 2 * np.exp(-a) / l
    dK_dx = -3 * np.exp(-a) * diff / l ** 2
    assert theta.grad.item() == pytest.approx(2.0 * (wv @ dK_dl @ zv), rel=1e-8)
    gx = 2.0 * wv * (dK_dx @ zv)
    assert np.linalg.norm(Xd.grad.cpu().numpy()[:, 0] - gx) <= 1e-8 * np.linalg.norm(gx)


def test_grad_full_size_c3_500k(env):
    """The adjoint workload: the d = 3 Matern-nu TT, N_s = N_t = 500k, w, z ~ N(0, 1) in FP32;
    the loss and dtheta against the oracle on the same cores (sampled-free: the loss is a sum
    over all points, computed by the oracle in FP64 from its own chain), dX on sampled rows."""
    torch, P = env
    w = W.C3
    tt = P.TT.build_offline(w.kernel, w.d, w.src_box, w.tgt_box, w.dtheta, w.theta_box, w.n, w.tol, "fp64")
    gc = tt.cores()
    N = W.CA_POINTS
    X, Y = W.sources(w, N), W.targets(w, N)
    wv, zv = W.weights(N)
    th = W.thetas(w, 1)[0]
    f32 = lambda a: torch.tensor(a, device="cuda", dtype=torch.float32)
    Xf, Yf, wf, zf = f32(X), f32(Y), f32(wv), f32(zv)
    L, dth, dX = P.grad(tt, th, Xf, Yf, wf, zf, "tf32x3")
    X32, Y32 = Xf.double().cpu().numpy(), Yf.double().cpu().numpy()
    w32, z32 = wf.double().cpu().numpy(), zf.double().cpu().numpy()
    # a = U^T w and b = V^T z by the oracle in chunks (500k points)
    Mo = o.core_matrix_H(gc, w.d, w.dtheta, th, w.theta_box)
    a = np.zeros(Mo.shape[0])
    b = np.zeros(Mo.shape[1])
    for s0 in range(0, N, 50000):
        sl = slice(s0, s0 + 50000)
        a += o.source_factor(gc, w.d, o.chebyshev_basis(X32[sl], w.src_box, w.n)).T @ w32[sl]
        b += o.target_factor(gc, w.d, o.chebyshev_basis(Y32[sl], w.tgt_box, w.n)).T @ z32[sl]
    Lo = a @ Mo @ b
    assert L == pytest.approx(Lo, rel=1e-4)
    gth = np.array([a @ o.core_matrix_dH(gc, w.d, w.dtheta, th, w.theta_box, j) @ b for j in range(w.dtheta)])
    assert np.linalg.norm(dth - gth) <= 1e-4 * np.linalg.norm(gth)
    rows = np.sort(np.random.default_rng(6).choice(N, 200, replace=False))
    g = Mo @ b
    B = o.chebyshev_basis(X32[rows], w.src_box, w.n)
    for i, (lo, hi) in enumerate(w.src_box):
        Bi = list(B)
        Bi[i] = o.cheb_dvector(o.interval_map_inv(X32[rows, i], lo, hi), w.n) * (2.0 / (lo - hi))
        ref = w32[rows] * (o.source_factor(gc, w.d, Bi) @ g)
        got = dX[rows, i].double().cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-4 * np.linalg.norm(ref)

"""Pins of the oracle's Gaussian-process pieces (log marginal likelihood, its gradient,
the PTTK-Global preconditioner, preconditioned CG), each against a closed form, another
library route or brute force, plus planted mistakes."""
import math

import numpy as np
import pytest

import oracle.pttk_gp as gp
import oracle.pttk_oracle as o


def _se(X, l):
    r2 = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
    return np.exp(-r2 / l ** 2), 2.0 * r2 / l ** 3 * np.exp(-r2 / l ** 2)   # K, dK/dl


def test_lml_of_one_point_is_the_closed_form():
    k, s2, y = 0.7, 0.1, 1.3
    want = -0.5 * y * y / (k + s2) - 0.5 * math.log(k + s2) - 0.5 * math.log(2 * math.pi)
    assert abs(gp.log_marginal_likelihood(np.array([[k]]), np.array([y]), s2) - want) <= 1e-15


def test_lml_matches_slogdet_and_solve():
    rng = np.random.default_rng(90)
    X = rng.uniform(0, 1, (80, 2))
    K, _ = _se(X, 0.6)
    y = rng.standard_normal(80)
    s2 = 1e-2
    A = K + s2 * np.eye(80)
    want = -0.5 * y @ np.linalg.solve(A, y) - 0.5 * np.linalg.slogdet(A)[1] - 40 * math.log(2 * math.pi)
    assert abs(gp.log_marginal_likelihood(K, y, s2) - want) <= 1e-10 * abs(want)


def test_lml_gradient_matches_central_differences():
    rng = np.random.default_rng(91)
    X = rng.uniform(0, 1, (60, 2))
    y = rng.standard_normal(60)
    s2, l, h = 1e-2, 0.6, 1e-6
    K, dK = _se(X, l)
    g = gp.log_marginal_likelihood_grad(K, [dK], y, s2)[0]
    fd = (gp.log_marginal_likelihood(_se(X, l + h)[0], y, s2) -
          gp.log_marginal_likelihood(_se(X, l - h)[0], y, s2)) / (2 * h)
    assert abs(g - fd) <= 1e-6 * abs(fd)


def test_global_preconditioner_is_the_inverse():
    rng = np.random.default_rng(92)
    Z, _ = np.linalg.qr(rng.standard_normal((50, 8)))
    B = rng.standard_normal((8, 8))
    W = B @ B.T
    s2 = 0.3
    v = rng.standard_normal(50)
    want = np.linalg.solve(Z @ W @ Z.T + s2 * np.eye(50), v)
    assert np.linalg.norm(gp.global_preconditioner(Z, W, s2)(v) - want) <= 1e-12 * np.linalg.norm(want)


def test_pcg_solves_and_an_exact_preconditioner_takes_one_step():
    rng = np.random.default_rng(93)
    X = rng.uniform(0, 1, (100, 2))
    K, _ = _se(X, 0.5)
    A = K + 1e-2 * np.eye(100)
    b = rng.standard_normal(100)
    x, it, _ = gp.pcg(lambda v: A @ v, b, tol=1e-12)
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-9 * np.linalg.norm(x)
    Ainv = np.linalg.inv(A)
    x1, it1, _ = gp.pcg(lambda v: A @ v, b, lambda v: Ainv @ v, tol=1e-10)
    assert it1 == 1


def test_global_factors_precondition_the_se_system():
    # PTTK-Global-1 of the SE kernel (d = 2, l = 0.7, N = 300) as a preconditioner for
    # (K + s2 I) x = b: CG needs far fewer steps than without it
    boxes = [(0.0, 1.0), (0.0, 1.0), (0.3, 1.4), (0.0, 1.0), (0.0, 1.0)]
    cores, _, _ = o.build_offline(o.GAUSS, 2, 1, boxes, 12, 1e-10)
    X = np.random.default_rng(94).uniform(0.0, 1.0, (300, 2))
    S, H, T = o.instantiate(cores, 2, 1, boxes, (0.7,), X, X)
    Z, W = o.global_factors(S, T, H)
    K = o.kernel_matrix(o.GAUSS, X, X, (0.7,))
    s2 = 1e-3
    A = lambda v: K @ v + s2 * v
    b = np.random.default_rng(95).standard_normal(300)
    _, it0, _ = gp.pcg(A, b, tol=1e-8, maxit=5000)
    x, it1, _ = gp.pcg(A, b, gp.global_preconditioner(Z, W, s2), tol=1e-8)
    assert np.linalg.norm(A(x) - b) <= 1e-8 * np.linalg.norm(b)
    assert it1 * 5 <= it0


# --- planted mistakes ------------------------------------------------------------------------

def _woodbury_without_shift(Z, W, s2):
    inner = np.linalg.inv(W)
    return lambda v: Z @ (inner @ (Z.T @ v)) + (v - Z @ (Z.T @ v)) / s2


def _grad_without_half(K, dK, y, s2):
    return 2.0 * _orig_grad(K, dK, y, s2)


def _lml_without_logdet(K, y, s2):
    A = K + s2 * np.eye(len(y))
    return float(-0.5 * y @ np.linalg.solve(A, y) - 0.5 * len(y) * math.log(2 * math.pi))


_orig_grad = gp.log_marginal_likelihood_grad

MUTATIONS = {
    "Woodbury inner matrix without s2": ("global_preconditioner", _woodbury_without_shift,
                                         test_global_preconditioner_is_the_inverse),
    "gradient without the 1/2": ("log_marginal_likelihood_grad", _grad_without_half,
                                 test_lml_gradient_matches_central_differences),
    "likelihood without log det": ("log_marginal_likelihood", _lml_without_logdet,
                                   test_lml_matches_slogdet_and_solve),
}


@pytest.mark.parametrize("name", list(MUTATIONS))
def test_gp_pins_catch_planted_mistakes(name, monkeypatch):
    attr, fn, pin = MUTATIONS[name]
    pin()
    monkeypatch.setattr(gp, attr, fn)
    with pytest.raises(AssertionError):
        pin()

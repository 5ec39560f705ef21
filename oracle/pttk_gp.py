"""Plain FP64 CPU oracle for the Gaussian-process use of PTTK named in Section 1 of arXiv
2406.06344: hyperparameters chosen by maximising the log marginal likelihood, which needs
K(X, X; theta) and its derivatives at many theta, and the parametric low-rank form used as a
preconditioner for conjugate gradients on the kernel system.

TEST INFRASTRUCTURE ONLY. The GPU library never imports or calls this module and shares no
code with it. Only the tests, ``__graft_entry__.smoke()`` and the CPU baseline leg of
``bench.py`` may use it.

The paper names these uses without formulas. The ones here are the textbook definitions
(Rasmussen and Williams, "Gaussian Processes for Machine Learning", 2006, Eqs. 2.30 and 5.9;
Hestenes and Stiefel's conjugate gradients with a preconditioner). Readings:
  G1  The noise model is K(X, X; theta) + s2 I with a fixed noise variance s2 > 0.
  G2  The preconditioner is (Z W Z^T + s2 I)^{-1}, with Z W Z^T the PTTK-Global factorisation
      of Algorithm 4 (Z with orthonormal columns). By the Woodbury identity it equals
      Z (W + s2 I)^{-1} Z^T + (I - Z Z^T) / s2.
  G3  CG stops when ||r_j||_2 <= tol ||b||_2, r_j the unpreconditioned residual.
"""
from __future__ import annotations

import math

import numpy as np


def log_marginal_likelihood(K: np.ndarray, y: np.ndarray, s2: float) -> float:
    """log p(y | X, theta) = -1/2 y^T (K + s2 I)^{-1} y - 1/2 log det(K + s2 I) - N/2 log(2 pi)
    (Rasmussen and Williams, Eq. 2.30), through a Cholesky factor."""
    N = len(y)
    L = np.linalg.cholesky(K + s2 * np.eye(N))
    alpha = np.linalg.solve(L.T, np.linalg.solve(L, y))
    return float(-0.5 * y @ alpha - np.sum(np.log(np.diag(L))) - 0.5 * N * math.log(2.0 * math.pi))


def log_marginal_likelihood_grad(K: np.ndarray, dK: list, y: np.ndarray, s2: float) -> np.ndarray:
    """d/d theta_j log p(y | X, theta) = 1/2 tr((alpha alpha^T - (K + s2 I)^{-1}) dK_j),
    alpha = (K + s2 I)^{-1} y (Rasmussen and Williams, Eq. 5.9)."""
    N = len(y)
    Ainv = np.linalg.inv(K + s2 * np.eye(N))
    alpha = Ainv @ y
    inner = np.outer(alpha, alpha) - Ainv
    return np.array([0.5 * np.sum(inner * dKj.T) for dKj in dK])


def global_preconditioner(Z: np.ndarray, W: np.ndarray, s2: float):
    """v -> (Z W Z^T + s2 I)^{-1} v for Z with orthonormal columns (reading G2): the Woodbury
    form Z (W + s2 I)^{-1} Z^T v + (v - Z Z^T v) / s2."""
    inner = np.linalg.inv(W + s2 * np.eye(W.shape[0]))

    def apply(v):
        c = Z.T @ v
        return Z @ (inner @ c) + (v - Z @ c) / s2
    return apply


def pcg(A, b: np.ndarray, Minv=None, tol: float = 1e-10, maxit: int = 1000):
    """Preconditioned conjugate gradients for A x = b, A symmetric positive definite, given as
    a function v -> A v; Minv: v -> M^{-1} v (identity when None). Stops when
    ||b - A x_j|| <= tol ||b|| (reading G3). Returns (x, iterations, residual norms)."""
    Minv = Minv or (lambda v: v)
    x = np.zeros_like(b)
    r = b.copy()
    z = Minv(r)
    p = z.copy()
    rz = r @ z
    bn = np.linalg.norm(b)
    hist = [np.linalg.norm(r)]
    it = 0
    while hist[-1] > tol * bn and it < maxit:
        Ap = A(p)
        a = rz / (p @ Ap)
        x = x + a * p
        r = r - a * Ap
        z = Minv(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
        hist.append(np.linalg.norm(r))
    return x, it, hist

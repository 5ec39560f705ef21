"""Pins of the FP64 oracle against facts fixed by the paper or by mathematics.

Each test checks the oracle through a route other than its own code: a closed
form, a library routine applied differently, a textbook identity, a value the
paper prints, or brute force on tiny inputs. They are chosen so that a dropped
term, a transposed operand, a wrong index order or a wrong sign in the oracle
fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
from scipy import special

import oracle.pttk_oracle as o

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --- Section 2.4: nodes, transform, basis -----------------------------------

@pytest.mark.parametrize("n", [2, 5, 12, 16, 20])
def test_nodes_are_roots_of_T_n(n):
    e = np.zeros(n + 1)
    e[n] = 1.0
    roots = np.sort(np.polynomial.chebyshev.chebroots(e).real)
    assert np.allclose(np.sort(o.cheb_nodes(n)), roots, atol=1e-13)


@pytest.mark.parametrize("n", [3, 12, 16, 20])
def test_transform_inverts_node_values(n):
    # discrete orthogonality of T_k at the roots of T_n: T A = A T = I, T[i, k] = T_k(zeta_i)
    zeta = o.cheb_nodes(n)
    T = np.stack([np.polynomial.chebyshev.chebval(zeta, np.eye(n)[k]) for k in range(n)], axis=1)
    A = o.cheb_transform_matrix(n)
    assert np.allclose(T @ A, np.eye(n), atol=1e-13)
    assert np.allclose(A @ T, np.eye(n), atol=1e-13)


@pytest.mark.parametrize("a,b", [(0.0, 1.0), (2.0, 3.0), (0.2, 2.0), (-1.0, 1.0)])
def test_basis_is_nodal_and_matches_coefficient_form(a, b):
    n = 9
    eta = o.interval_map(o.cheb_nodes(n), a, b)
    # phi(eta_i, eta_j) = delta_ij (Section 2.4, proof of Lemma cheb_bound)
    assert np.allclose(o.basis_q(eta, a, b, n), np.eye(n), atol=1e-13)
    x = np.linspace(a, b, 37)
    q = o.basis_q(x, a, b, n)
    # q(x) = T(xhat)^T A with T evaluated by numpy's Chebyshev series (reading R3)
    xh = o.interval_map_inv(x, a, b)
    T = np.stack([np.polynomial.chebyshev.chebval(xh, np.eye(n)[k]) for k in range(n)], axis=1)
    assert np.allclose(q, T @ o.cheb_transform_matrix(n), atol=1e-13)
    assert np.allclose(q.sum(axis=1), 1.0, atol=1e-13)       # constants are reproduced


@pytest.mark.parametrize("n", [4, 12, 16, 20, 32])
def test_lebesgue_bound(n):
    # Lemma cheb_bound: max_x sum_k |phi(zeta_k, x)| <= (2/pi) log n + 1
    x = np.linspace(-1.0, 1.0, 4001)
    lam = np.abs(o.basis_q(x, -1.0, 1.0, n)).sum(axis=1).max()
    assert lam <= 2.0 / math.pi * math.log(n) + 1.0


def test_interval_map_is_the_printed_one():
    # Section 2.4 prints phi_[a,b](x) = ((a-b)/2) x + (a+b)/2: +1 -> a, -1 -> b
    assert o.interval_map(1.0, 2.0, 3.0) == 2.0
    assert o.interval_map(-1.0, 2.0, 3.0) == 3.0
    assert o.interval_map_inv(o.interval_map(0.3, 2.0, 5.0), 2.0, 5.0) == pytest.approx(0.3)


@pytest.mark.parametrize("n", [12, 16])
def test_coefficients_of_separable_exponential(n):
    # exp(s t) = I_0(s) + 2 sum_k I_k(s) T_k(t) (textbook Chebyshev expansion; modified Bessel I).
    # A product over modes with a different s per mode pins the mode order of C = M x_k A.
    s = [0.7, -1.3, 0.4]
    boxes = [(0.0, 1.0), (0.5, 2.0), (2.0, 3.0)]
    eta = o.node_vectors(boxes, n)
    grids = np.meshgrid(*[o.interval_map_inv(e, a, b) for e, (a, b) in zip(eta, boxes)], indexing="ij")
    M = np.exp(sum(sj * g for sj, g in zip(s, grids)))
    C = o.coefficient_tensor(M, n)
    # interpolation at the n roots of T_n aliases T_{2n-k} onto -T_k and T_{2n+k} onto -T_k
    # (T_{2n +- k}(zeta_i) = -T_k(zeta_i)), so the discrete coefficient is
    # a_k - a_{2n-k} - a_{2n+k} + ...; two alias terms suffice at these s and n.
    def discrete(sj):
        a = lambda k: (1.0 if k == 0 else 2.0) * special.iv(k, sj)
        return np.array([a(k) - a(2 * n - k) - a(2 * n + k) for k in range(n)])
    expected = np.einsum("i,j,k->ijk", *[discrete(sj) for sj in s])
    assert np.allclose(C, expected, atol=2e-16 * n ** 3)


# --- Table kern-table: kernels -----------------------------------------------

@pytest.mark.parametrize("l", [0.5, 1.0, 2.0])
def test_matern_general_nu_reduces_to_closed_forms(l):
    r = np.linspace(0.05, 6.0, 200)
    a = r / l
    exp_ = np.exp(-a)                                                     # nu = 1/2
    m32 = (1 + math.sqrt(3) * a) * np.exp(-math.sqrt(3) * a)              # nu = 3/2
    m52 = (1 + math.sqrt(5) * a + 5 * a ** 2 / 3) * np.exp(-math.sqrt(5) * a)  # nu = 5/2
    assert np.allclose(o.kernel_of_r(o.MATERN_NU, r, (l, 0.5)), exp_, rtol=1e-13, atol=0)
    assert np.allclose(o.kernel_of_r(o.MATERN_NU, r, (l, 1.5)), m32, rtol=1e-13, atol=0)
    assert np.allclose(o.kernel_of_r(o.MATERN_NU, r, (l, 2.5)), m52, rtol=1e-13, atol=0)
    assert np.allclose(o.kernel_of_r(o.MATERN32, r, (l,)), m32, rtol=1e-14, atol=0)
    # normalisation 2^(1-nu)/Gamma(nu): kappa -> 1 as r -> 0 for every nu
    for nu in (0.7, 1.9, 2.5):
        assert o.kernel_of_r(o.MATERN_NU, np.array([1e-9]), (l, nu))[0] == pytest.approx(1.0, abs=1e-6)


def test_gaussian_has_no_half():
    # Table kern-table: exp(-(r/l)^2); at r = l the value is exp(-1)
    assert o.kernel_of_r(o.GAUSS, np.array([1.3]), (1.3,))[0] == pytest.approx(math.exp(-1.0), rel=1e-15)


def test_grid_entries_are_kernel_values_at_nodes():
    # Eq. mdc: m_{i} = f_kappa(eta) with xi = (x, theta, y); checked against the dense kernel
    d, dth, n = 2, 2, 4
    boxes = [(0, 1), (0, 1), (0.5, 2.0), (0.5, 2.5), (3, 4), (0, 1)]
    M = o.grid_tensor(o.kernel_f(o.MATERN_NU), d, dth, boxes, n)
    eta = o.node_vectors(boxes, n)
    rng = np.random.default_rng(0)
    for _ in range(20):
        i = rng.integers(0, n, size=6)
        x = np.array([eta[0][i[0]], eta[1][i[1]]])
        th = (eta[2][i[2]], eta[3][i[3]])
        y = np.array([eta[4][i[4]], eta[5][i[5]]])
        assert M[tuple(i)] == pytest.approx(o.kernel_matrix(o.MATERN_NU, x, y, th)[0, 0], rel=1e-14)


def test_grid_sizes_printed_in_appendix_c():
    rows = [l.split("#")[0].split() for l in open(os.path.join(GOLDEN, "appendix_c_grid_sizes.txt"))]
    rows = [list(map(int, r)) for r in rows if r]
    assert len(rows) == 4
    for d, dth, n, count in rows:
        assert n ** (2 * d + dth) == count
        # the oracle's grid has that many entries (checked at n = 2 to keep it small)
        boxes = [(0.0, 1.0)] * (2 * d + dth)
        M = o.grid_tensor(lambda x, th, y: 1.0 + 0.0 * x[0], d, dth, boxes, 2)
        assert M.size == 2 ** (2 * d + dth)


# --- Section 2.3: TT-SVD -----------------------------------------------------

def _random_tt(dims, ranks, rng):
    return [rng.standard_normal((ranks[k], dims[k], ranks[k + 1])) for k in range(len(dims))]


def test_tt_svd_recovers_known_ranks():
    rng = np.random.default_rng(1)
    dims, ranks = (5, 6, 4, 5, 3), [1, 3, 4, 5, 2, 1]
    X = o.tt_full(_random_tt(dims, ranks, rng))
    cores, r = o.tt_svd(X, 1e-12)
    assert r == ranks
    assert o.rel_fro(X, o.tt_full(cores)) < 1e-13
    for G in cores[:-1]:                                  # left-orthonormal cores
        G2 = o.unfold2(G)
        assert np.allclose(G2.T @ G2, np.eye(G2.shape[1]), atol=1e-12)


def _odeco(dims, sigma, rng):
    """sum_i sigma_i u_i (x) v_i (x) ... with orthonormal factor columns: every
    unfolding has singular values exactly sigma."""
    Qs = [np.linalg.qr(rng.standard_normal((n, len(sigma))))[0] for n in dims]
    X = 0
    for i, s in enumerate(sigma):
        t = np.array(s)
        for Q in Qs:
            t = np.multiply.outer(t, Q[:, i])
        X = X + t
    return X


def test_tt_svd_threshold_uses_sqrt_D_minus_1():
    # delta = eps / sqrt(D-1) ||X||_F (Algorithm 1). Put delta at 0.8 x the tail after rank 3:
    # the correct rule keeps rank 4 at every bond; dropping sqrt(D-1) (= sqrt 3) would keep 3.
    rng = np.random.default_rng(2)
    sigma = np.array([1.0, 1e-2, 1e-4, 1e-6, 1e-8])
    X = _odeco((6, 6, 6, 6), sigma, rng)
    tail3 = math.sqrt(float(np.sum(sigma[3:] ** 2)))
    eps = 0.8 * tail3 * math.sqrt(3) / np.linalg.norm(X)
    cores, r = o.tt_svd(X, eps)
    assert r == [1, 4, 4, 4, 1]
    assert o.rel_fro(X, o.tt_full(cores)) <= eps
    eps_loose = 1.2 * tail3 * math.sqrt(3) / np.linalg.norm(X)
    assert o.tt_svd(X, eps_loose)[1] == [1, 3, 3, 3, 1]


@pytest.mark.parametrize("eps", [1e-1, 1e-2, 1e-4])
def test_tt_svd_error_bound_and_rank_caps(eps):
    rng = np.random.default_rng(3)
    X = rng.standard_normal((4, 5, 3, 4, 5))
    cores, r = o.tt_svd(X, eps)
    assert o.rel_fro(X, o.tt_full(cores)) <= eps * (1 + 1e-12)
    dims = X.shape
    for k in range(1, len(dims)):
        assert r[k] <= min(np.prod(dims[:k]), np.prod(dims[k:]))


def test_tt_svd_order_two_is_eckart_young():
    # for D = 2 the TT-SVD is a truncated SVD; its error must equal the optimal tail
    rng = np.random.default_rng(4)
    X = rng.standard_normal((30, 20)) @ np.diag(0.5 ** np.arange(20)) @ rng.standard_normal((20, 20))
    cores, r = o.tt_svd(X, 1e-3)
    s = np.linalg.svd(X, compute_uv=False)
    tail = math.sqrt(float(np.sum(s[r[1]:] ** 2)))
    assert np.linalg.norm(X - o.tt_full(cores)) == pytest.approx(tail, rel=1e-8)
    assert math.sqrt(float(np.sum(s[r[1] - 1:] ** 2))) > 1e-3 * np.linalg.norm(X)


def test_separable_function_has_unit_ranks():
    f = lambda x, th, y: np.exp(x[0]) * np.cos(th[0]) * (1 + y[0] ** 2)
    boxes = [(0, 1), (0.5, 2), (2, 3)]
    cores, r, C = o.build_offline(o.GAUSS, 1, 1, boxes, 10, 1e-12, f=f)
    assert r == [1, 1, 1, 1]


# --- Algorithms 2-3: online stage and factor chain ---------------------------

def test_polynomial_kernel_is_reproduced_exactly():
    # Proposition compress (p = n): a kernel of degree < n in every variable is interpolated exactly
    f = lambda x, th, y: (1.0 + x[0] * y[0] + x[1] * y[1] + th[0]) ** 3
    d, dth = 2, 1
    boxes = [(0, 1), (0, 1), (0.2, 2.0), (2, 3), (0, 1)]
    rng = np.random.default_rng(5)
    X = rng.random((40, 2))
    Y = np.column_stack([2 + rng.random(40), rng.random(40)])
    theta = (1.37,)
    exact = (1.0 + X @ Y.T + theta[0]) ** 3
    cores, r, C = o.build_offline(None, d, dth, boxes, 5, 1e-13, f=f)
    assert max(r) <= 10
    U, M, V = o.instantiate(cores, d, dth, boxes, theta, X, Y)
    assert o.rel_fro(exact, U @ M @ V.T) < 1e-13
    # with too few nodes (n = 3, degree 3 needs 4) the same pipeline is not exact
    cores3, _, _ = o.build_offline(None, d, dth, boxes, 3, 1e-13, f=f)
    U, M, V = o.instantiate(cores3, d, dth, boxes, theta, X, Y)
    assert o.rel_fro(exact, U @ M @ V.T) > 1e-6


def test_factor_chain_equals_full_interpolant():
    # mixed-product identities (Eq. mixedprod) behind Phase 3: S H T^T = F_s C_F^{d}(theta) F_t^T
    rng = np.random.default_rng(6)
    d, dth, n = 2, 2, 5
    ranks = [1, 3, 7, 4, 6, 5, 2, 1][: 2 * d + dth + 1]
    ranks[-1] = 1
    cores = _random_tt((n,) * (2 * d + dth), ranks, rng)
    boxes = [(0, 1), (0, 1), (0.5, 2), (0.5, 2.5), (3, 4), (0, 1)]
    X = rng.random((17, 2))
    Y = np.column_stack([3 + rng.random(13), rng.random(13)])
    theta = (1.1, 0.9)
    U, M, V = o.instantiate(cores, d, dth, boxes, theta, X, Y)
    full = o.full_interpolant(o.tt_full(cores), d, dth, boxes, theta, X, Y)
    assert np.allclose(U @ M @ V.T, full, rtol=1e-12, atol=1e-12 * np.abs(full).max())
    assert U.shape == (17, ranks[d]) and V.shape == (13, ranks[d + dth]) and M.shape == (ranks[d], ranks[d + dth])


def test_dense_kernel_brute_force_c1():
    # end to end on tiny inputs: K~ vs dense K; the error is the interpolation floor
    # (Proposition error: E(n) plus an amplified TT term that is negligible at tol 1e-10)
    from paper_2406_06344_gb300 import workloads as W
    w = W.C1
    cores, r, C = o.build_offline(w.kernel, w.d, w.dtheta, w.mode_boxes(), w.n, w.tol)
    X, Y = W.sources(w, 300), W.targets(w, 300)
    for th, bound in (((1.9,), 1e-6), ((1.2,), 1e-5), ((0.5,), 1e-3)):
        K = o.kernel_matrix(w.kernel, X, Y, th)
        U, M, V = o.instantiate(cores, w.d, w.dtheta, w.mode_boxes(), th, X, Y)
        Kf = o.full_interpolant(C, w.d, w.dtheta, w.mode_boxes(), th, X, Y)
        assert o.rel_fro(K, U @ M @ V.T) < bound
        # the TT truncation error is absolute (delta ~ 1e-10 ||C||_F), far below the floor
        assert np.abs(Kf - U @ M @ V.T).max() < 1e-9
    # exponential convergence in n at fixed theta
    errs = []
    for n in (8, 12, 16, 24):
        cores, _, _ = o.build_offline(w.kernel, w.d, w.dtheta, w.mode_boxes(), n, 1e-12)
        U, M, V = o.instantiate(cores, w.d, w.dtheta, w.mode_boxes(), (1.2,), X, Y)
        errs.append(o.rel_fro(o.kernel_matrix(w.kernel, X, Y, (1.2,)), U @ M @ V.T))
    assert errs[0] > errs[1] > errs[2] > errs[3] and errs[3] < 1e-9


def test_error_bound_of_proposition_error():
    # ||K~_full - K~_TT||_C <= lambda^D ||M - M^||_C  (proof of Proposition error, Eq. inter2)
    from paper_2406_06344_gb300 import workloads as W
    w = W.C1
    n = w.n
    cores, r, C = o.build_offline(w.kernel, w.d, w.dtheta, w.mode_boxes(), n, 1e-4)
    Ainv = np.linalg.inv(o.cheb_transform_matrix(n))
    M = C
    Mhat = o.tt_full(cores)
    for k in range(3):
        M = o.mode_product(M, Ainv, k)
        Mhat = o.mode_product(Mhat, Ainv, k)
    lam = 2.0 / math.pi * math.log(n) + 1.0
    X, Y = W.sources(w, 100), W.targets(w, 100)
    for th in ((0.7,), (1.6,)):
        U, Mh, V = o.instantiate(cores, w.d, w.dtheta, w.mode_boxes(), th, X, Y)
        Kf = o.full_interpolant(C, w.d, w.dtheta, w.mode_boxes(), th, X, Y)
        assert np.abs(Kf - U @ Mh @ V.T).max() <= lam ** 3 * np.abs(M - Mhat).max()


def test_orientation_of_interval_map_does_not_change_the_interpolant():
    # reading R1: reversing every box (b, a) turns the printed map into the usual one
    from paper_2406_06344_gb300 import workloads as W
    w = W.C2
    boxes = w.mode_boxes()
    n = 8
    X, Y = W.sources(w, 50), W.targets(w, 50)
    th = (0.9,)
    c1, _, _ = o.build_offline(w.kernel, w.d, w.dtheta, boxes, n, 1e-12)
    c2, _, _ = o.build_offline(w.kernel, w.d, w.dtheta, boxes[:, ::-1], n, 1e-12)
    K1 = np.linalg.multi_dot(o.instantiate(c1, w.d, w.dtheta, boxes, th, X, Y)[:2] + (o.instantiate(c1, w.d, w.dtheta, boxes, th, X, Y)[2].T,))
    U2, M2, V2 = o.instantiate(c2, w.d, w.dtheta, boxes[:, ::-1], th, X, Y)
    assert o.rel_fro(K1, U2 @ M2 @ V2.T) < 1e-12


def test_apply_matches_dense_product():
    rng = np.random.default_rng(7)
    U, M, V, w = rng.random((30, 5)), rng.random((5, 4)), rng.random((20, 4)), rng.random(20)
    assert np.allclose(o.apply(U, M, V, w), (U @ M @ V.T) @ w, rtol=1e-14)


# --- gradients of L = w^T K~ z -----------------------------------------------

def _small_tt(kind, d, dth, boxes, n):
    return o.build_offline(kind, d, dth, boxes, n, 1e-12)[0]


def test_gradients_match_central_differences():
    d, dth, n = 2, 2, 7
    boxes = [(0, 1), (0, 1), (0.5, 2.0), (0.5, 2.5), (3, 4), (0, 1)]
    cores = _small_tt(o.MATERN_NU, d, dth, boxes, n)
    rng = np.random.default_rng(8)
    X = rng.random((25, 2))
    Y = np.column_stack([3 + rng.random(30), rng.random(30)])
    w, z = rng.standard_normal(25), rng.standard_normal(30)
    theta = np.array([1.3, 1.7])
    gth, gX = o.loss_grad(cores, d, dth, boxes, theta, X, Y, w, z)
    L = lambda th, XX: o.loss(*o.instantiate(cores, d, dth, boxes, th, XX, Y), w, z)
    h = 1e-6
    for j in range(dth):
        e = np.zeros(dth)
        e[j] = h
        fd = (L(theta + e, X) - L(theta - e, X)) / (2 * h)
        assert gth[j] == pytest.approx(fd, rel=1e-7, abs=1e-9)
    for _ in range(4):
        v = rng.standard_normal(X.shape)
        fd = (L(theta, X + h * v) - L(theta, X - h * v)) / (2 * h)
        assert float(np.sum(gX * v)) == pytest.approx(fd, rel=1e-7, abs=1e-9)


def test_gradients_match_dense_matern32_closed_form():
    # at nu = 3/2: dkappa/dl = a^2 e^{-a} / l, grad_x kappa = -3 e^{-a} (x - y) / l^2, a = sqrt(3) r / l
    d, dth, n = 1, 1, 24          # n = 24: the interpolation floor is ~1e-13 here
    boxes = [(0, 1), (0.5, 2.0), (2, 3)]
    cores = _small_tt(o.MATERN32, d, dth, boxes, n)
    rng = np.random.default_rng(9)
    X, Y = rng.random((40, 1)), 2 + rng.random((50, 1))
    w, z = rng.standard_normal(40), rng.standard_normal(50)
    l = 1.4
    gth, gX = o.loss_grad(cores, d, dth, boxes, np.array([l]), X, Y, w, z)
    diff = X[:, None, 0] - Y[None, :, 0]
    r = np.abs(diff)
    a = math.sqrt(3) * r / l
    dK_dl = a ** 2 * np.exp(-a) / l
    dK_dx = -3 * np.exp(-a) * diff / l ** 2
    assert gth[0] == pytest.approx(w @ dK_dl @ z, rel=1e-9)
    gx = w * (dK_dx @ z)
    assert np.linalg.norm(gX[:, 0] - gx) <= 1e-10 * np.linalg.norm(gx)


# --- the other kernels of Table kern-table --------------------------------------

@pytest.mark.parametrize("l", [0.5, 1.3])
def test_exponential_and_matern52_are_matern_at_half_and_five_halves(l):
    # the closed forms against the general-nu Matern evaluated through scipy's K_nu
    r = np.linspace(0.05, 6.0, 101)
    assert np.allclose(o.kernel_of_r(o.EXPONENTIAL, r, (l,)), o.kernel_of_r(o.MATERN_NU, r, (l, 0.5)),
                       rtol=1e-13, atol=0)
    assert np.allclose(o.kernel_of_r(o.MATERN52, r, (l,)), o.kernel_of_r(o.MATERN_NU, r, (l, 2.5)),
                       rtol=1e-13, atol=0)


def test_multiquadric_and_thin_plate_family_identities():
    r = np.linspace(0.1, 5.0, 50)
    for l in (0.4, 1.0, 2.5):
        # multiquadric = hypot(1, r/l)
        assert np.allclose(o.kernel_of_r(o.MULTIQUADRIC, r, (l,)), np.hypot(1.0, r / l), rtol=1e-15)
        # thin-plate spline (r/l)^2 log((r/l)^2) = 2 x thin-plate at r/l
        assert np.allclose(o.kernel_of_r(o.THIN_PLATE_SPLINE, r, (l,)), 2.0 * o.kernel_of_r(o.THIN_PLATE, r / l, ()),
                           rtol=1e-13, atol=1e-15)
    # thin-plate r^2 log r = -r^2 x Laplace-2D; bi-harmonic = Laplace-3D squared
    assert np.allclose(o.kernel_of_r(o.THIN_PLATE, r, ()), -r * r * o.kernel_of_r(o.LAPLACE2D, r, ()), rtol=1e-15)
    assert np.allclose(o.kernel_of_r(o.BIHARMONIC, r, ()), o.kernel_of_r(o.LAPLACE3D, r, ()) ** 2, rtol=1e-15)
    assert o.kernel_of_r(o.THIN_PLATE_SPLINE, np.array([0.0]), (1.0,))[0] == 0.0   # the limit at r = 0


def test_kernel_without_parameter_end_to_end():
    # TTK (d_theta = 0): the pipeline runs with an empty theta and H = I; the interpolation of
    # the Laplace-3D kernel on admissible boxes converges to the dense matrix
    d, boxes = 2, [(0.0, 1.0), (0.0, 1.0), (2.0, 3.0), (0.0, 1.0)]
    X = np.random.default_rng(11).random((60, 2))
    Y = np.column_stack([2 + np.random.default_rng(12).random(50), np.random.default_rng(13).random(50)])
    K = o.kernel_matrix(o.LAPLACE3D, X, Y, ())
    errs = []
    for n in (6, 10, 14):
        cores, r, C = o.build_offline(o.LAPLACE3D, d, 0, boxes, n, 1e-13)
        U, M, V = o.instantiate(cores, d, 0, boxes, (), X, Y)
        assert M.shape[0] == M.shape[1] and np.array_equal(M, np.eye(M.shape[0]))
        errs.append(o.rel_fro(K, U @ M @ V.T))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-8


# --- TT-Round (Algorithm 1) -------------------------------------------------------

def tt_sum(a, b):
    """Cores of the TT of X_a + X_b: concatenated end cores, block-diagonal middle cores."""
    N = len(a)
    out = []
    for i, (A, B) in enumerate(zip(a, b)):
        if i == 0:
            out.append(np.concatenate([A, B], axis=2))
        elif i == N - 1:
            out.append(np.concatenate([A, B], axis=0))
        else:
            C = np.zeros((A.shape[0] + B.shape[0], A.shape[1], A.shape[2] + B.shape[2]))
            C[:A.shape[0], :, :A.shape[2]] = A
            C[A.shape[0]:, :, A.shape[2]:] = B
            out.append(C)
    return out


def test_tt_round_undoes_rank_inflation():
    # X + X has a TT with doubled ranks; rounding finds the ranks of X and the tensor 2X
    rng = np.random.default_rng(21)
    dims, ranks = (4, 5, 3, 6, 4), [1, 3, 4, 3, 2, 1]
    G = _random_tt(dims, ranks, rng)
    X = o.tt_full(G)
    S = tt_sum(G, G)
    assert [c.shape[2] for c in S][:-1] == [2 * r for r in ranks[1:-1]]
    R, rr = o.tt_round(S, 1e-12)
    assert rr == ranks
    assert o.rel_fro(2 * X, o.tt_full(R)) < 1e-13
    for g in R[:-1]:                                       # left-orthonormal cores
        g2 = o.unfold2(g)
        assert np.allclose(g2.T @ g2, np.eye(g2.shape[1]), atol=1e-12)


@pytest.mark.parametrize("eps", [1e-2, 1e-5])
def test_tt_round_meets_its_tolerance(eps):
    # a low-rank tensor plus small noise in TT format with inflated ranks: the rounded TT
    # stays within eps of it and its ranks do not exceed the input's
    rng = np.random.default_rng(22)
    dims = (5, 4, 6, 5)
    G = _random_tt(dims, [1, 2, 3, 2, 1], rng)
    Nz = [0.01 * c for c in _random_tt(dims, [1, 4, 5, 3, 1], rng)]
    S = tt_sum(G, Nz)
    X = o.tt_full(S)
    R, rr = o.tt_round(S, eps)
    assert o.rel_fro(X, o.tt_full(R)) <= eps
    assert all(a <= b for a, b in zip(rr, [1] + [c.shape[2] for c in S]))


@pytest.mark.parametrize("eps", [1e-3, 1e-6])
def test_tt_round_matches_tt_svd_of_the_full_tensor(eps):
    # After the right-to-left orthogonalisation, the left-to-right sweep of TT-Round sees the
    # singular values of the full tensor's unfoldings, as the TT-SVD does, and both cut at the
    # same delta. So rounding a TT of X with inflated ranks gives the TT-SVD's ranks and error.
    # Test tensor: 1/(1 + i1 + i2 + 1.3 i3 + i4 + i5), whose unfoldings decay gradually.
    dims = (6, 5, 7, 6, 5)
    idx = np.indices(dims)
    X = 1.0 / (1.0 + idx.sum(axis=0) + 0.3 * idx[2])
    G, ranks = o.tt_svd(X, eps)
    E, _ = o.tt_svd(X, 1e-15)
    S = tt_sum([E[0] / 3] + E[1:], [2 * E[0] / 3] + E[1:])        # X with doubled ranks
    R, rr = o.tt_round(S, eps)
    assert rr == ranks
    e_svd, e_round = o.rel_fro(X, o.tt_full(G)), o.rel_fro(X, o.tt_full(R))
    assert abs(e_svd - e_round) <= 1e-6 * e_svd


# --- PTTK-Global (Algorithm 4) --------------------------------------------------------------

def test_global_1_is_the_psd_part_of_the_symmetric_part():
    # Q W Q^T of PTTK-Global-1 is the symmetric part (S H T^T + T H^T S^T)/2 of the plain
    # approximation with its negative eigenvalues set to zero; without that step (an indefinite
    # kernel) it is the symmetric part itself. Checked against an eigendecomposition of the
    # N x N matrix, a different and larger problem than the k x k one the oracle solves.
    rng = np.random.default_rng(30)
    N, rs, rt = 40, 5, 7
    S, T, H = rng.standard_normal((N, rs)), rng.standard_normal((N, rt)), rng.standard_normal((rs, rt))
    K1 = S @ H @ T.T
    Ks = 0.5 * (K1 + K1.T)
    lam, V = np.linalg.eigh(Ks)
    assert lam.min() < -1e-3 * lam.max()                      # the case has negative eigenvalues
    Kpsd = V @ np.diag(np.maximum(lam, 0.0)) @ V.T
    Z, W = o.global_factors(S, T, H)
    assert o.rel_fro(Kpsd, Z @ W @ Z.T) <= 1e-12
    Z, W = o.global_factors(S, T, H, definite=False)
    assert o.rel_fro(Ks, Z @ W @ Z.T) <= 1e-12
    Q, R = o.global_offline(S, T)
    assert np.allclose(Q.T @ Q, np.eye(Q.shape[1]), atol=1e-13)
    assert o.rel_fro(np.hstack([S, T]), Q @ R) <= 1e-14


@pytest.mark.parametrize("definite", [True, False])
@pytest.mark.parametrize("eps", [3e-2, 1e-3])
def test_global_2_keeps_the_fewest_terms(definite, eps):
    # PTTK-Global-2 keeps the shortest prefix (by |lambda|) of eigenpairs of the symmetric part
    # meeting ||Z W Z^T - S H T^T||_F <= eps ||S H T^T||_F. Brute force on the N x N matrices:
    # for each m, the m largest eigenpairs of (S H T^T + T H^T S^T)/2 (the positive ones only
    # for a definite kernel), and the error measured directly.
    # S H T^T = F C F^T + 1e-4 F B F2^T: symmetric with a graded, partly negative spectrum, plus a
    # small non-symmetric part, the structure of the kernel case
    rng = np.random.default_rng(32)
    N, rs, rt = 50, 6, 8
    F = rng.standard_normal((N, rs))
    Qc, _ = np.linalg.qr(rng.standard_normal((rs, rs)))
    C = Qc @ np.diag([4.0, 2.0, -0.002, 1.0, 0.3, 0.05]) @ Qc.T
    S, T = F, np.hstack([F, rng.standard_normal((N, rt - rs))])
    H = np.hstack([C, 1e-4 * rng.standard_normal((rs, rt - rs))])
    K1 = S @ H @ T.T
    lam, V = np.linalg.eigh(0.5 * (K1 + K1.T))
    order = np.argsort(-np.abs(lam), kind="stable")
    lam, V = lam[order], V[:, order]
    if definite:
        lam, V = lam[lam > 0], V[:, lam > 0]
    errs = [np.linalg.norm(V[:, :m] @ np.diag(lam[:m]) @ V[:, :m].T - K1) for m in range(len(lam) + 1)]
    ok = [m for m, e in enumerate(errs) if e <= eps * np.linalg.norm(K1)]
    m_brute = ok[0] if ok else len(lam)
    assert 0 < m_brute < len(lam)                               # a real choice at this eps
    Z, W = o.global_factors(S, T, H, eps, compress=True, definite=definite)
    assert Z.shape[1] == m_brute
    assert np.allclose(W, np.diag(np.diag(W)))                  # W = Lambda^, diagonal
    assert abs(np.linalg.norm(Z @ W @ Z.T - K1) - errs[m_brute]) <= 1e-10 * np.linalg.norm(K1)
    assert np.allclose(Z.T @ Z, np.eye(Z.shape[1]), atol=1e-12)  # Q U^ has orthonormal columns


def _global_case(kind):
    boxes = [(0.0, 1.0), (0.0, 1.0), (0.3, 1.4), (0.0, 1.0), (0.0, 1.0)]
    cores, _, _ = o.build_offline(kind, 2, 1, boxes, 12, 1e-10)
    X = np.random.default_rng(31).uniform(0.0, 1.0, (300, 2))
    th = (0.7,)
    S, H, T = o.instantiate(cores, 2, 1, boxes, th, X, X)
    return S, H, T, o.kernel_matrix(kind, X, X, th)


def test_global_on_the_squared_exponential_kernel():
    # SE is positive definite: PTTK-Global-1 is symmetric positive semi-definite and as close to
    # K as the plain interpolant S H T^T is (the symmetric PSD part can only move it closer)
    S, H, T, K = _global_case(o.GAUSS)
    plain = o.rel_fro(K, S @ H @ T.T)
    Z, W = o.global_factors(S, T, H)
    Kg = Z @ W @ Z.T
    assert o.rel_fro(K, Kg) <= plain * (1 + 1e-9)
    assert np.abs(Kg - Kg.T).max() <= 1e-14 * np.abs(Kg).max()
    ev = np.linalg.eigvalsh(0.5 * (Kg + Kg.T))
    assert ev.min() >= -1e-13 * ev.max()
    # PTTK-Global-2 at eps = 1e-4: far fewer terms, within the tolerance of S H T^T
    Z2, W2 = o.global_factors(S, T, H, 1e-4, compress=True)
    assert Z2.shape[1] < Z.shape[1] // 4
    assert o.rel_fro(S @ H @ T.T, Z2 @ W2 @ Z2.T) <= 1e-4


def test_global_on_the_indefinite_multiquadric_kernel():
    # The Multiquadric matrix is indefinite: zeroing negative eigenvalues loses > 10 % of it,
    # and without that step PTTK-Global-1 is as accurate as the plain interpolant
    S, H, T, K = _global_case(o.MULTIQUADRIC)
    plain = o.rel_fro(K, S @ H @ T.T)
    Z, W = o.global_factors(S, T, H, definite=False)
    assert o.rel_fro(K, Z @ W @ Z.T) <= plain * (1 + 1e-6)
    Z, W = o.global_factors(S, T, H, definite=True)
    assert o.rel_fro(K, Z @ W @ Z.T) >= 0.1


# --- Algorithm 2, Phase 4: TT-Round of the twisted TT [T1(S), G_theta.., T3(T^T)] ----------

def _phase4_case(dtheta=1, Ns=23, Nt=19, n=6, seed=5):
    """Factors S (Ns x rs) and T (Nt x rt) and theta cores with known structure: S and T have
    more columns than rank (products through a smaller inner dimension), so rounding must
    reduce them."""
    rng = np.random.default_rng(seed)
    rs, rt, inner = 7, 6, 3
    S = rng.standard_normal((Ns, inner)) @ rng.standard_normal((inner, rs))
    T = rng.standard_normal((Nt, inner)) @ rng.standard_normal((inner, rt))
    ranks = [rs] + [5] * (dtheta - 1) + [rt]
    cores = [rng.standard_normal((ranks[j], n, ranks[j + 1])) for j in range(dtheta)]
    return S, cores, T


def _full_twisted(S, cores, T):
    """x[i, k.., j] = sum S[i,a] G_1[a,k_1,b] .. T[j,c] by brute-force einsum (not tt_full)."""
    if len(cores) == 1:
        return np.einsum("ia,akb,jb->ikj", S, cores[0], T)
    return np.einsum("ia,akb,blc,jc->iklj", S, cores[0], cores[1], T)


@pytest.mark.parametrize("dtheta", [1, 2])
def test_twisted_tt_represents_S_H_T(dtheta):
    S, cores, T = _phase4_case(dtheta)
    tw = o.twisted_tt(S, cores, T)
    assert np.allclose(o.tt_full(tw), _full_twisted(S, cores, T), atol=1e-12)
    # contracting the theta modes with the Chebyshev vectors gives S H(theta) T^T (Eq. hmat)
    box = [(0.5, 2.0)] * dtheta
    th = [0.8, 1.7][:dtheta]
    full = _full_twisted(S, cores, T)
    n = cores[0].shape[1]
    for j, (t, (a, b)) in enumerate(zip(th, box)):
        v = np.polynomial.chebyshev.chebvander(np.array([(2 * t - a - b) / (a - b)]), n - 1)[0]
        full = np.tensordot(full, v, axes=([1], [0]))
    assert np.allclose(full, S @ o.theta_core_matrix(cores, th, box) @ T.T, atol=1e-10)


@pytest.mark.parametrize("eps", [1e-12, 1e-3])
def test_phase4_meets_its_tolerance_and_tt_svd_ranks(eps):
    S, cores, T = _phase4_case(2)
    X = _full_twisted(S, cores, T)
    S2, c2, T2, ranks = o.phase4(S, cores, T, eps)
    X2 = _full_twisted(S2, c2, T2)
    assert np.linalg.norm(X2 - X) <= eps * np.linalg.norm(X) * (1 + 1e-10) + 1e-13
    assert ranks == o.tt_svd(X, eps)[1]
    # the first core is left-orthonormal after the left-to-right sweep
    assert np.allclose(S2.T @ S2, np.eye(S2.shape[1]), atol=1e-12)


def test_phase4_removes_redundant_columns():
    # S and T have 7 and 6 columns but rank 3: at a tight tolerance the outer ranks become 3
    S, cores, T = _phase4_case(1)
    S2, c2, T2, ranks = o.phase4(S, cores, T, 1e-12)
    assert S2.shape[1] == 3 and T2.shape[1] == 3
    assert ranks == [1, 3, 3, 1]


def test_phase4_per_theta_error_bound():
    # |T_k| <= 1 on [-1, 1], so the matrix at any theta moves by at most
    # sqrt(n^dtheta) ||X - X'||_F <= sqrt(n^dtheta) eps ||X||_F
    S, cores, T = _phase4_case(2, seed=9)
    eps = 1e-2
    X = _full_twisted(S, cores, T)
    S2, c2, T2, _ = o.phase4(S, cores, T, eps)
    box = [(0.5, 2.0), (0.5, 2.5)]
    n = cores[0].shape[1]
    for th in ([0.5, 0.5], [1.3, 2.2], [2.0, 2.5]):
        K = S @ o.theta_core_matrix(cores, th, box) @ T.T
        K2 = S2 @ o.theta_core_matrix(c2, th, box) @ T2.T
        assert np.linalg.norm(K - K2) <= math.sqrt(n ** 2) * eps * np.linalg.norm(X)

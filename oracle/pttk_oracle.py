"""Plain FP64 CPU oracle for the parametric tensor-train kernel (PTTK) method of
Khan & Saibaba, "Parametric kernel low-rank approximations using tensor train
decomposition" (arXiv 2406.06344).

TEST INFRASTRUCTURE ONLY. The GPU library never imports or calls this module and
shares no code with it. Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use it.

Everything is FP64 numpy, written for readability rather than speed. Library
primitives (matrix products, the SVD, the Bessel function K_nu and the gamma
function) serve as single steps; nothing is blocked, fused or reordered beyond
what each cited passage states.

Conventions (all from Section 2 of the paper):
  * tensors are numpy arrays indexed [i_1, ..., i_D]; unfoldings use the
    little-endian (column-major, i_1 fastest) flattening of Section 2.2, i.e.
    numpy ``order='F'`` reshapes;
  * a TT core G_k has shape (r_{k-1}, n, r_k); G^{2} is its
    (r_{k-1} n) x r_k unfolding and G^{1} its r_{k-1} x (n r_k) unfolding;
  * the variable order is xi = (x, theta, y) (Eq. fkappa), D = 2d + dtheta.

Readings of the paper taken here (where the paper is silent, ambiguous or garbled):
  R1  The interval map is used exactly as printed in Section 2.4,
      phi_[a,b](t) = ((a-b)/2) t + (a+b)/2 (it sends +1 to a). The
      interpolant does not depend on this orientation (test pin).
  R2  Nodes are the roots of T_n (first kind), zeta_i = cos((2i-1) pi / (2n)).
  R3  The TT is built from the Chebyshev coefficient tensor
      C = M x_1 A x_2 A ... x_D A, A[k, i] = (c_k / n) T_k(zeta_i),
      c_0 = 1, c_k = 2 (Eq. cheb_trans rewritten: q(x) = T(xhat)^T A).
      Contracting a core of C with T(xhat) equals contracting the matching
      core of the nodal TT with q(x), so Algorithms 2 and 3 are unchanged
      with q replaced by the Chebyshev vector T(xhat).
  R4  The TT is computed by TT-SVD (Oseledets 2011, Algorithm 1, cited in
      Section 2.3) with the truncation threshold of Algorithm 1 (TT-Round):
      delta = eps / sqrt(D-1) * ||C||_F; r_k is the smallest r >= 1 whose
      discarded tail satisfies sqrt(sum_{i>r} sigma_i^2) <= delta.
  R5  Matern normalisation reads 2^(1-nu) / Gamma(nu) (the table prints
      Gamma(l)); SE is exp(-(r/l)^2) without a factor 1/2 (Table kern-table).
  R6  Phase 3 of Algorithm 2 (the factor chain) runs per instantiation:
      instantiate(TT, theta, X, Y) -> (U, M, V) = (S, H(theta), T).
  R7  PTTK-Global (Algorithm 4): the compression test compares with
      S H(theta) T^T (the printed S H(theta) T lacks the transpose). The
      eigenpairs kept are a prefix of the order |lambda_1| >= |lambda_2| >= ...
      (negative eigenvalues removed first when the kernel is definite), the
      shortest prefix that meets the test; all of them when none does.
"""
from __future__ import annotations

import math
import numpy as np
from scipy import special

GAUSS, MATERN32, MATERN_NU = 0, 1, 2
EXPONENTIAL, MATERN52, MULTIQUADRIC, THIN_PLATE_SPLINE = 3, 4, 5, 6
BIHARMONIC, LAPLACE3D, LAPLACE2D, THIN_PLATE = 7, 8, 9, 10     # no parameter (d_theta = 0)


# ---------------------------------------------------------------------------
# Section 2.4: Chebyshev nodes, interval map, basis
# ---------------------------------------------------------------------------

def cheb_nodes(n: int) -> np.ndarray:
    """Roots of T_n on [-1, 1]: zeta_i = cos((2i-1) pi / (2n)), i = 1..n (Section 2.4)."""
    i = np.arange(1, n + 1, dtype=np.float64)
    return np.cos((2.0 * i - 1.0) * np.pi / (2.0 * n))


def interval_map(t, a: float, b: float):
    """phi_[a,b](t) = ((a-b)/2) t + (a+b)/2, as printed in Section 2.4 (reading R1)."""
    return 0.5 * (a - b) * np.asarray(t, dtype=np.float64) + 0.5 * (a + b)


def interval_map_inv(x, a: float, b: float):
    """phi_[a,b]^{-1}(x) = (2x - a - b) / (a - b)."""
    return (2.0 * np.asarray(x, dtype=np.float64) - a - b) / (a - b)


def cheb_T(k, t):
    """T_k(t) = cos(k arccos t) for |t| <= 1 (definition in Section 2.4)."""
    t = np.clip(np.asarray(t, dtype=np.float64), -1.0, 1.0)
    return np.cos(np.multiply.outer(np.arccos(t), np.asarray(k, dtype=np.float64)))


def cheb_vector(t, n: int) -> np.ndarray:
    """[T_0(t), ..., T_{n-1}(t)] for each t: shape t.shape + (n,)."""
    return cheb_T(np.arange(n), t)


def cheb_dvector(t, n: int) -> np.ndarray:
    """[T_0'(t), ..., T_{n-1}'(t)] via numpy's Chebyshev-series derivative (library routine)."""
    t = np.asarray(t, dtype=np.float64)
    out = np.empty(t.shape + (n,))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        out[..., k] = np.polynomial.chebyshev.chebval(t, np.polynomial.chebyshev.chebder(e)) if k else 0.0
    return out


def cheb_transform_matrix(n: int) -> np.ndarray:
    """A[k, i] = (c_k / n) T_k(zeta_i), c_0 = 1, c_{k>=1} = 2 (Eq. cheb_trans, reading R3)."""
    zeta = cheb_nodes(n)
    c = np.full(n, 2.0)
    c[0] = 1.0
    return (c[:, None] / n) * cheb_T(np.arange(n), zeta).T


def basis_q(x, a: float, b: float, n: int) -> np.ndarray:
    """q(x) = [phi^{[a,b]}(eta_1, x), ..., phi^{[a,b]}(eta_n, x)] written out term by term
    from Eq. cheb_trans: 1/n + (2/n) sum_{k=1}^{n-1} T_k(phi^{-1}(eta_i)) T_k(phi^{-1}(x))
    (Eqs. q_s_t, q_p). Shape x.shape + (n,)."""
    eta = interval_map(cheb_nodes(n), a, b)
    zeta_i = interval_map_inv(eta, a, b)               # = the nodes on [-1, 1]
    xh = interval_map_inv(x, a, b)
    out = np.full(np.shape(x) + (n,), 1.0 / n)
    for k in range(1, n):
        out += (2.0 / n) * np.multiply.outer(cheb_T(k, xh), cheb_T(k, zeta_i))
    return out


# ---------------------------------------------------------------------------
# Table kern-table: kernels
# ---------------------------------------------------------------------------

def kernel_of_r(kind: int, r, theta) -> np.ndarray:
    """kappa as a function of r = ||x - y||_2 and theta (Table kern-table, reading R5).

    GAUSS              theta = (l,):      exp(-(r/l)^2)
    MATERN32           theta = (l,):      (1 + sqrt(3) r/l) exp(-sqrt(3) r/l)
    MATERN_NU          theta = (l, nu):   2^(1-nu)/Gamma(nu) (sqrt(2 nu) r/l)^nu K_nu(sqrt(2 nu) r/l)
    EXPONENTIAL        theta = (l,):      exp(-r/l)
    MATERN52           theta = (l,):      (1 + sqrt(5) r/l + 5 (r/l)^2 / 3) exp(-sqrt(5) r/l)
    MULTIQUADRIC       theta = (l,):      (1 + (r/l)^2)^(1/2)
    THIN_PLATE_SPLINE  theta = (l,):      (r/l)^2 log((r/l)^2)
    BIHARMONIC         theta = ():        r^-2
    LAPLACE3D          theta = ():        r^-1
    LAPLACE2D          theta = ():        -log(r)
    THIN_PLATE         theta = ():        r^2 log(r)
    """
    r = np.asarray(r, dtype=np.float64)
    if kind == GAUSS:
        l = theta[0]
        return np.exp(-(r / l) ** 2)
    if kind == MATERN32:
        l = theta[0]
        a = math.sqrt(3.0) * r / l
        return (1.0 + a) * np.exp(-a)
    if kind == EXPONENTIAL:
        return np.exp(-r / theta[0])
    if kind == MATERN52:
        a = math.sqrt(5.0) * r / theta[0]
        return (1.0 + a + a * a / 3.0) * np.exp(-a)
    if kind == MULTIQUADRIC:
        return np.sqrt(1.0 + (r / theta[0]) ** 2)
    if kind == THIN_PLATE_SPLINE:
        q = (r / theta[0]) ** 2
        with np.errstate(divide="ignore", invalid="ignore"):
            return np.where(q > 0.0, q * np.log(np.where(q > 0.0, q, 1.0)), 0.0)
    if kind == BIHARMONIC:
        return r ** -2.0
    if kind == LAPLACE3D:
        return 1.0 / r
    if kind == LAPLACE2D:
        return -np.log(r)
    if kind == THIN_PLATE:
        return r * r * np.log(r)
    if kind == MATERN_NU:
        l, nu = theta[0], theta[1]
        z = np.sqrt(2.0 * nu) * r / l
        return np.power(2.0, 1.0 - nu) / special.gamma(nu) * np.power(z, nu) * special.kv(nu, z)
    raise ValueError(f"unknown kernel {kind}")


def kernel_matrix(kind: int, X, Y, theta) -> np.ndarray:
    """Dense K(X, Y; theta), [K]_ij = kappa(x_i, y_j; theta) (Eq. matparamkernel)."""
    X = np.atleast_2d(X)
    Y = np.atleast_2d(Y)
    r = np.sqrt(((X[:, None, :] - Y[None, :, :]) ** 2).sum(-1))
    return kernel_of_r(kind, r, theta)


# ---------------------------------------------------------------------------
# Section 2.4 "Multivariate approximation": the grid tensor M and coefficients C
# ---------------------------------------------------------------------------

def node_vectors(mode_boxes, n: int) -> list:
    """eta^{(j)}_i = phi_[alpha_j, beta_j](zeta_i) for j = 1..D."""
    zeta = cheb_nodes(n)
    return [interval_map(zeta, a, b) for (a, b) in mode_boxes]


def grid_tensor(f, d: int, dtheta: int, mode_boxes, n: int) -> np.ndarray:
    """m_{i_1..i_D} = f_kappa(eta^{(1)}_{i_1}, ..., eta^{(D)}_{i_D}) (Eq. mdc).

    ``f(x, theta, y)`` receives broadcastable arrays: x and y are lists of d
    coordinate arrays, theta a list of dtheta arrays (variable order of Eq. fkappa).
    Evaluated one slab of the last mode at a time to bound memory.
    """
    D = 2 * d + dtheta
    eta = node_vectors(mode_boxes, n)
    out = np.empty((n,) * D, dtype=np.float64)
    grids = np.ix_(*eta[:-1])
    for last in range(n):
        coords = list(grids) + [np.full((1,) * (D - 1), eta[-1][last])]
        x = coords[:d]
        th = coords[d:d + dtheta]
        y = coords[d + dtheta:]
        out[..., last] = np.broadcast_to(f(x, th, y), (n,) * (D - 1))
    return out


def kernel_f(kind: int):
    """f_kappa(xi) = kappa(x, y; theta) with xi = (x, theta, y) (Eq. fkappa)."""
    def f(x, th, y):
        r2 = 0.0
        for xj, yj in zip(x, y):
            r2 = r2 + (xj - yj) ** 2
        r = np.sqrt(r2)
        if kind == MATERN_NU:
            l, nu = th
            z = np.sqrt(2.0 * nu) * r / l
            return np.power(2.0, 1.0 - nu) / special.gamma(nu) * np.power(z, nu) * special.kv(nu, z)
        return kernel_of_r(kind, r, tuple(th[:1]))
    return f


def mode_product(X: np.ndarray, A: np.ndarray, k: int) -> np.ndarray:
    """Y = X x_k A, y_{..j..} = sum_{i_k} x_{..i_k..} a_{j, i_k} (Section 2.2)."""
    return np.moveaxis(np.tensordot(A, X, axes=([1], [k])), 0, k)


def coefficient_tensor(M: np.ndarray, n: int) -> np.ndarray:
    """C = M x_1 A x_2 A ... x_D A (reading R3)."""
    A = cheb_transform_matrix(n)
    C = M
    for k in range(M.ndim):
        C = mode_product(C, A, k)
    return C


# ---------------------------------------------------------------------------
# Section 2.3: TT format and TT-SVD
# ---------------------------------------------------------------------------

def truncation_rank(s: np.ndarray, delta: float) -> int:
    """Smallest r >= 1 with sqrt(sum_{i>r} s_i^2) <= delta (reading R4)."""
    for r in range(1, len(s) + 1):
        if math.sqrt(float(np.sum(s[r:] ** 2))) <= delta:
            return r
    return len(s)


def tt_svd(C: np.ndarray, eps: float):
    """TT-SVD (Oseledets 2011, Algorithm 1; Section 2.3) with delta = eps/sqrt(D-1) ||C||_F.

    Returns (cores, ranks): cores[k] has shape (r_k, n_{k+1}, r_{k+1}), ranks = [1, r_1, ..., r_{D-1}, 1].
    """
    D = C.ndim
    dims = C.shape
    delta = eps / math.sqrt(D - 1) * float(np.linalg.norm(C.ravel()))
    cores = []
    ranks = [1]
    X = C.reshape(-1, order="F")
    r_prev = 1
    for k in range(D - 1):
        X = X.reshape(r_prev * dims[k], -1, order="F")
        U, s, Vt = np.linalg.svd(X, full_matrices=False)
        r = truncation_rank(s, delta)
        cores.append(U[:, :r].reshape(r_prev, dims[k], r, order="F"))
        X = s[:r, None] * Vt[:r, :]
        ranks.append(r)
        r_prev = r
    cores.append(X.reshape(r_prev, dims[-1], 1, order="F"))
    ranks.append(1)
    return cores, ranks


def tt_round(cores, eps: float):
    """TT-Round (Algorithm 1, Section 2.3): right-to-left orthogonalisation by thin QR of
    (G_i^{1})^T, then left-to-right truncated SVDs of G_i^{2} with delta = eps/sqrt(N-1) ||X||_F.
    Reading: the update of G_{i-1} is the one that leaves the tensor unchanged,
    G_{i-1}^{2} <- G_{i-1}^{2} R^T (G_i^{1} = R^T Q^T).
    Returns (cores, ranks)."""
    G = [np.array(c, dtype=np.float64) for c in cores]
    N = len(G)
    for i in range(N - 1, 0, -1):
        r0, n, r1 = G[i].shape
        Q, R = np.linalg.qr(unfold1(G[i]).T)                 # (n r1) x k, k x r0
        k = Q.shape[1]
        G[i] = Q.T.reshape(k, n, r1, order="F")
        a, m, _ = G[i - 1].shape
        G[i - 1] = (unfold2(G[i - 1]) @ R.T).reshape(a, m, k, order="F")
    delta = eps / math.sqrt(N - 1) * float(np.linalg.norm(G[0])) if N > 1 else 0.0
    for i in range(N - 1):
        r0, n, r1 = G[i].shape
        U, s, Vt = np.linalg.svd(unfold2(G[i]), full_matrices=False)
        r = truncation_rank(s, delta)
        G[i] = U[:, :r].reshape(r0, n, r, order="F")
        _, n2, r2 = G[i + 1].shape
        G[i + 1] = ((s[:r, None] * Vt[:r]) @ unfold1(G[i + 1])).reshape(r, n2, r2, order="F")
    return G, [1] + [g.shape[2] for g in G]


def tt_full(cores) -> np.ndarray:
    """x_{i_1..i_N} = sum_s G_1[1,i_1,s_1] G_2[s_1,i_2,s_2] ... G_N[s_{N-1},i_N,1] (Section 2.3)."""
    T = cores[0]                                  # (1, n_1, r_1)
    for G in cores[1:]:
        T = np.tensordot(T, G, axes=([T.ndim - 1], [0]))
    return T.reshape(T.shape[1:-1])


def unfold2(G: np.ndarray) -> np.ndarray:
    """G^{2}: (r_{k-1} n) x r_k unfolding, row index a + r_{k-1} j."""
    return G.reshape(G.shape[0] * G.shape[1], G.shape[2], order="F")


def unfold1(G: np.ndarray) -> np.ndarray:
    """G^{1}: r_{k-1} x (n r_k) unfolding, column index j + n b."""
    return G.reshape(G.shape[0], G.shape[1] * G.shape[2], order="F")


# ---------------------------------------------------------------------------
# Section 2.1 products used by Phase 3
# ---------------------------------------------------------------------------

def face_split(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """A ⋉ B: row p is A[p,:] (Kronecker) B[p,:], column index j * cols(B) + a (Section 2.1)."""
    return np.einsum("pj,pa->pja", A, B).reshape(A.shape[0], A.shape[1] * B.shape[1])


def khatri_rao(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """A ⋊ B: column q is A[:,q] (Kronecker) B[:,q], row index a * rows(B) + j (Section 2.1)."""
    return np.einsum("aq,jq->ajq", A, B).reshape(A.shape[0] * B.shape[0], A.shape[1])


# ---------------------------------------------------------------------------
# Algorithm 3 (online stage) and Algorithm 2 Phase 3 (factor chain)
# ---------------------------------------------------------------------------

def theta_hat(theta, theta_box) -> np.ndarray:
    return np.array([interval_map_inv(t, a, b) for t, (a, b) in zip(theta, theta_box)])


def core_matrix_H(cores, d: int, dtheta: int, theta, theta_box) -> np.ndarray:
    """H(theta) = H_1(theta_1) ... H_dtheta(theta_dtheta), H_j = G_{d+j} x_2 T(theta_hat_j)
    (Eq. hmat and Algorithm 3, in the coefficient form of reading R3)."""
    n = cores[d].shape[1]
    th = theta_hat(theta, theta_box)
    H = np.eye(cores[d].shape[0])
    for j in range(dtheta):
        G = cores[d + j]
        Hj = np.tensordot(G, cheb_vector(th[j], n), axes=([1], [0]))
        H = H @ Hj
    return H


def core_matrix_dH(cores, d: int, dtheta: int, theta, theta_box, which: int) -> np.ndarray:
    """d H(theta) / d theta_which: the factor H_which is replaced by
    sum_k G[:,k,:] T_k'(theta_hat) * dtheta_hat/dtheta, dtheta_hat/dtheta = 2/(a - b)."""
    n = cores[d].shape[1]
    th = theta_hat(theta, theta_box)
    H = np.eye(cores[d].shape[0])
    for j in range(dtheta):
        G = cores[d + j]
        if j == which:
            a, b = theta_box[j]
            v = cheb_dvector(th[j], n) * (2.0 / (a - b))
        else:
            v = cheb_vector(th[j], n)
        H = H @ np.tensordot(G, v, axes=([1], [0]))
    return H


def chebyshev_basis(points: np.ndarray, box, n: int) -> list:
    """B_i[p, k] = T_k(phi^{-1}(points[p, i])): the coefficient-form factor matrices
    U_i / V_i of Eq. uv_factor (reading R3). One N x n matrix per spatial dimension."""
    return [cheb_vector(interval_map_inv(points[:, i], a, b), n) for i, (a, b) in enumerate(box)]


def source_factor(cores, d: int, B: list) -> np.ndarray:
    """Algorithm 2 Phase 3, source side: S <- U_1 G_1^{2}; S <- (U_i ⋉ S) G_i^{2}, i = 2..d."""
    S = B[0] @ unfold2(cores[0])
    for i in range(1, d):
        S = face_split(B[i], S) @ unfold2(cores[i])
    return S


def target_factor(cores, d: int, Bt: list) -> np.ndarray:
    """Algorithm 2 Phase 3, target side: T <- G_D^{1} V_d^T;
    T <- G_{D-i}^{1} (T ⋊ V_{d-i}^T), i = 1..d-1; T <- T^T."""
    D = len(cores)
    T = unfold1(cores[D - 1]) @ Bt[d - 1].T
    for i in range(1, d):
        T = unfold1(cores[D - 1 - i]) @ khatri_rao(T, Bt[d - 1 - i].T)
    return T.T


def instantiate(cores, d: int, dtheta: int, mode_boxes, theta, X, Y):
    """instantiate(TT, theta, X, Y) -> (U, M, V) with K ~= U M V^T (reading R6):
    U = S (source factor), M = H(theta) (Algorithm 3), V = T (target factor)."""
    n = cores[0].shape[1]
    mode_boxes = [tuple(b) for b in mode_boxes]
    src_box = mode_boxes[:d]
    th_box = mode_boxes[d:d + dtheta]
    tgt_box = mode_boxes[d + dtheta:]
    U = source_factor(cores, d, chebyshev_basis(np.atleast_2d(X), src_box, n))
    V = target_factor(cores, d, chebyshev_basis(np.atleast_2d(Y), tgt_box, n))
    M = core_matrix_H(cores, d, dtheta, theta, th_box)
    return U, M, V


def twisted_tt(S: np.ndarray, theta_cores, T: np.ndarray) -> list:
    """[T^(1)(S), G_{d+1}, ..., G_{d+dtheta}, T^(3)(T^T)] (Eq. twist; Section 3.1, Phase 4):
    an order-(dtheta + 2) TT with mode sizes (N_s, n, ..., n, N_t) whose first core holds S
    ([T^(1)(S)]_{1,i,j} = s_ij) and whose last holds T^T ([T^(3)(T^T)]_{i,j,1} = t_ji)."""
    first = S.reshape(1, S.shape[0], S.shape[1])
    last = T.T.reshape(T.shape[1], T.shape[0], 1)
    return [first] + [np.array(g, dtype=np.float64) for g in theta_cores] + [last]


def phase4(S: np.ndarray, theta_cores, T: np.ndarray, eps: float):
    """Phase 4 of Algorithm 2: TT-Round (Algorithm 1) of the twisted TT of S, the theta cores
    and T^T at tolerance eps. Returns (S', theta cores', T', ranks): the compressed factors
    with K(X, Y; theta) ~= S' H'(theta) T'^T, H' from the rounded theta cores by Eq. hmat."""
    G, ranks = tt_round(twisted_tt(S, theta_cores, T), eps)
    S2 = G[0].reshape(G[0].shape[1], G[0].shape[2])
    T2 = G[-1].reshape(G[-1].shape[0], G[-1].shape[1]).T
    return S2, G[1:-1], T2, ranks


def theta_core_matrix(theta_cores, theta, theta_box) -> np.ndarray:
    """H(theta) of Eq. hmat from the theta cores alone (Algorithm 3)."""
    return core_matrix_H(list(theta_cores), 0, len(theta_cores), theta, theta_box)


def apply(U, M, V, w) -> np.ndarray:
    """out = U (M (V^T w)): the low-rank matrix-vector product of Eq. paramlowrank."""
    return U @ (M @ (V.T @ w))


# ---------------------------------------------------------------------------
# Eq. paramkernelmatrix: the direct full-tensor interpolant (no TT)
# ---------------------------------------------------------------------------

def face_split_chain(B: list) -> np.ndarray:
    """F = B_d ⋉ B_{d-1} ⋉ ... ⋉ B_1 (Eq. fs), column index i_1 + n i_2 + ... (little-endian)."""
    F = B[0]
    for Bi in B[1:]:
        F = face_split(Bi, F)
    return F


def full_interpolant(C: np.ndarray, d: int, dtheta: int, mode_boxes, theta, X, Y) -> np.ndarray:
    """K~_full = F_s C_F^{d}(theta) F_t^T with C_F(theta) = C x_{d+j} T(theta_hat_j)
    (Eqs. ilowrank and paramkernelmatrix in coefficient form, reading R3)."""
    n = C.shape[0]
    mode_boxes = [tuple(b) for b in mode_boxes]
    th = theta_hat(theta, mode_boxes[d:d + dtheta])
    Ct = C
    for j in range(dtheta):                      # contract the theta modes one at a time
        Ct = np.tensordot(Ct, cheb_vector(th[j], n), axes=([d], [0]))
    MF = Ct.reshape(n ** d, n ** d, order="F")
    Fs = face_split_chain(chebyshev_basis(np.atleast_2d(X), mode_boxes[:d], n))
    Ft = face_split_chain(chebyshev_basis(np.atleast_2d(Y), mode_boxes[d + dtheta:], n))
    return Fs @ MF @ Ft.T


# ---------------------------------------------------------------------------
# Offline stage entry point and error metric
# ---------------------------------------------------------------------------

def build_offline(kind: int, d: int, dtheta: int, mode_boxes, n: int, eps: float, f=None):
    """Grid -> coefficients -> TT-SVD (Algorithm 2 Phases 1-2 with TT-SVD in place of
    greedy-cross, reading R4). Returns (cores, ranks, C)."""
    f = kernel_f(kind) if f is None else f
    M = grid_tensor(f, d, dtheta, mode_boxes, n)
    C = coefficient_tensor(M, n)
    cores, ranks = tt_svd(C, eps)
    return cores, ranks, C


def rel_fro(A, B) -> float:
    """||A - B||_F / ||A||_F (relative error of Section 4, Frobenius norm)."""
    return float(np.linalg.norm(A - B) / np.linalg.norm(A))


# ---------------------------------------------------------------------------
# Gradients of the scalar loss L = w^T K~ z (the adjoint form)
# ---------------------------------------------------------------------------

def loss(U, M, V, w, z) -> float:
    return float(w @ (U @ (M @ (V.T @ z))))


def loss_grad(cores, d: int, dtheta: int, mode_boxes, theta, X, Y, w, z):
    """dL/dtheta and dL/dX for L = w^T U(X) H(theta) V(Y)^T z.

    dL/dtheta_j = (U^T w)^T dH/dtheta_j (V^T z).
    dL/dx_{p,i} = w_p * (dU[p,:]/dx_{p,i}) . (H V^T z), where dU/dx_{:,i} is the
    Phase-3 chain with the basis of dimension i replaced by T'(xhat) * 2/(a-b)
    (each x_{p,i} enters U[p,:] only through that basis row)."""
    n = cores[0].shape[1]
    mode_boxes = [tuple(b) for b in mode_boxes]
    src_box = mode_boxes[:d]
    th_box = mode_boxes[d:d + dtheta]
    X = np.atleast_2d(X)
    U, M, V = instantiate(cores, d, dtheta, mode_boxes, theta, X, Y)
    a = U.T @ w
    b = V.T @ z
    dtheta_out = np.array([a @ core_matrix_dH(cores, d, dtheta, theta, th_box, j) @ b
                           for j in range(dtheta)])
    g = M @ b
    B = chebyshev_basis(X, src_box, n)
    dX = np.empty_like(X)
    for i, (lo, hi) in enumerate(src_box):
        Bi = list(B)
        Bi[i] = cheb_dvector(interval_map_inv(X[:, i], lo, hi), n) * (2.0 / (lo - hi))
        dX[:, i] = w * (source_factor(cores, d, Bi) @ g)
    return dtheta_out, dX


# --- PTTK-Global (Algorithm 4, Section 3 "Global low-rank approximation") ----------------

def global_offline(S: np.ndarray, T: np.ndarray):
    """Offline stage of PTTK-Global (Algorithm 4): with X = Y and B_s = B_t, S = U(X) and
    T = V(X) are the two factors of Algorithm 2 on the one point set; the thin QR
    [S T] = Q R is stored. Returns (Q, R), Q: N x k orthonormal, R: k x (r_s + r_t)."""
    Q, R = np.linalg.qr(np.hstack([S, T]), mode="reduced")
    return Q, R


def global_hhat(H: np.ndarray) -> np.ndarray:
    """H^ of Eq. pttk1: the symmetric block matrix [[0, H/2], [H^T/2, 0]], so that
    [S T] H^ [S T]^T = (S H T^T + T H^T S^T) / 2."""
    rs, rt = H.shape
    Hh = np.zeros((rs + rt, rs + rt))
    Hh[:rs, rs:] = 0.5 * H
    Hh[rs:, :rs] = 0.5 * H.T
    return Hh


def global_online(R: np.ndarray, H: np.ndarray, eps: float = 0.0, compress: bool = False,
                  definite: bool = True):
    """Online stage of PTTK-Global (Algorithm 4) for H = H(theta) (r_s x r_t).

    Eigendecomposition R H^ R^T = U Lambda U^T, eigenpairs ordered by decreasing |lambda|;
    for a definite kernel the negative eigenvalues are zeroed and their eigenvectors dropped
    (the paper drops this step for indefinite kernels such as the Multiquadric).
    Without compression: returns (None, W), W = U Lambda U^T (k x k), K ~= Q W Q^T.
    With compression: keeps the shortest prefix of eigenpairs with
    ||Q U^ Lambda^ (Q U^)^T - S H T^T||_F <= eps ||S H T^T||_F (reading R7; with Q orthonormal
    and S H T^T = Q (R E R^T) Q^T, E = [[0, H], [0, 0]], both norms are taken on k x k
    matrices); returns (U^, Lambda^) with K ~= (Q U^) Lambda^ (Q U^)^T."""
    rs = H.shape[0]
    lam, U = np.linalg.eigh(R @ global_hhat(H) @ R.T)
    order = np.argsort(-np.abs(lam), kind="stable")
    lam, U = lam[order], U[:, order]
    if definite:
        keep = lam > 0
        lam, U = lam[keep], U[:, keep]
    if not compress:
        return None, U @ np.diag(lam) @ U.T
    E = np.zeros((R.shape[1], R.shape[1]))
    E[:rs, rs:] = H
    target = R @ E @ R.T
    bound = eps * np.linalg.norm(target)
    m = len(lam)
    for j in range(len(lam) + 1):
        if np.linalg.norm(U[:, :j] @ np.diag(lam[:j]) @ U[:, :j].T - target) <= bound:
            m = j
            break
    return U[:, :m], np.diag(lam[:m])


def global_factors(S: np.ndarray, T: np.ndarray, H: np.ndarray, eps: float = 0.0,
                   compress: bool = False, definite: bool = True):
    """Both stages of Algorithm 4 on one point set: returns (Z, W) with K(X, X; theta) ~=
    Z W Z^T; Z = Q (PTTK-Global-1, compress False) or Q U^ (PTTK-Global-2)."""
    Q, R = global_offline(S, T)
    Uh, W = global_online(R, H, eps, compress, definite)
    return (Q if Uh is None else Q @ Uh), W

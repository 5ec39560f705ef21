"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in the oracle (on the CPU, by replacing one of its functions for
the duration of the test) and checks that at least one of the pins in test_oracle_pins.py now
fails. The mistakes are the ones a reader of the paper could plausibly make: a dropped or
doubled coefficient, the wrong node family, a reversed map, a missing factor in a kernel or in
the truncation threshold, an off-by-one rank, a transposed unfolding, a swapped Kronecker
index, a wrong sign or scale in a derivative.
"""
import math

import numpy as np
import pytest
from scipy import special

import oracle.pttk_oracle as o
from tests import test_oracle_pins as pins

_orig = {name: getattr(o, name) for name in dir(o) if callable(getattr(o, name))}


def _transform_c0_two(n):
    zeta = o.cheb_nodes(n)
    return (2.0 / n) * o.cheb_T(np.arange(n), zeta).T


def _nodes_extrema(n):
    return np.cos(np.arange(n) * np.pi / max(n - 1, 1))


def _map_usual(t, a, b):
    return 0.5 * (b - a) * np.asarray(t, dtype=np.float64) + 0.5 * (a + b)


def _kernel_half(kind, r, theta):
    if kind == o.GAUSS:
        return np.exp(-0.5 * (np.asarray(r) / theta[0]) ** 2)
    return _orig["kernel_of_r"](kind, r, theta)


def _kernel_gamma_l(kind, r, theta):
    if kind == o.MATERN_NU:
        l, nu = theta[0], theta[1]
        z = np.sqrt(2.0 * nu) * np.asarray(r) / l
        return np.power(2.0, 1.0 - nu) / special.gamma(l) * np.power(z, nu) * special.kv(nu, z)
    return _orig["kernel_of_r"](kind, r, theta)


def _tt_svd_no_sqrt(C, eps):
    # delta without the 1/sqrt(D-1) factor: equivalent to calling the right rule with eps sqrt(D-1)
    return _orig["tt_svd"](C, eps * math.sqrt(C.ndim - 1))


def _rank_plus_one(s, delta):
    return min(_orig["truncation_rank"](s, delta) + 1, len(s))


def _rank_minus_one(s, delta):
    return max(_orig["truncation_rank"](s, delta) - 1, 1)


def _face_split_swapped(A, B):
    return np.einsum("pj,pa->paj", A, B).reshape(A.shape[0], A.shape[1] * B.shape[1])


def _unfold2_c_order(G):
    return G.reshape(G.shape[0] * G.shape[1], G.shape[2], order="C")


def _target_factor_transposed(cores, d, Bt):
    # the target chain read with the source-side unfolding of each core
    D = len(cores)
    T = Bt[d - 1] @ o.unfold2(np.transpose(cores[D - 1], (2, 1, 0)))
    for i in range(1, d):
        T = o.face_split(Bt[d - 1 - i], T) @ o.unfold2(cores[D - 1 - i])
    return T


def _H_wrong_sign(cores, d, dtheta, theta, theta_box):
    return _orig["core_matrix_H"](cores, d, dtheta, theta, [(b, a) for a, b in theta_box])


def _dH_wrong_scale(cores, d, dtheta, theta, theta_box, which):
    return -_orig["core_matrix_dH"](cores, d, dtheta, theta, theta_box, which)


def _mode_product_transposed(X, A, k):
    return np.moveaxis(np.tensordot(A.T, X, axes=([1], [k])), 0, k)


def _grid_order_swapped(f, d, dtheta, mode_boxes, n):
    # variables handed to f in the order (x, y, theta) instead of xi = (x, theta, y)
    return _orig["grid_tensor"](lambda x, th, y: f(x, y, th), d, dtheta, mode_boxes, n)


def _apply_reversed_points(U, M, V, w):
    # the target points taken in reverse order
    return U @ (M @ (V[::-1].T @ w))


def _dvector_missing_two(t, n):
    return 0.5 * _orig["cheb_dvector"](t, n)


def _chebT_shifted(k, t):
    return _orig["cheb_T"](np.asarray(k) + 1, t)


def _laplace2d_sign(kind, r, theta):
    if kind == o.LAPLACE2D:
        return np.log(np.asarray(r))
    return _orig["kernel_of_r"](kind, r, theta)


def _H_theta_swapped(cores, d, dtheta, theta, theta_box):
    # theta_1 contracted with the core of theta_2 and the other way round
    th = list(theta)[::-1]
    box = list(theta_box)[::-1]
    n = cores[d].shape[1]
    H = np.eye(cores[d].shape[0])
    that = o.theta_hat(th, box)
    for j in range(dtheta):
        H = H @ np.tensordot(cores[d + j], o.cheb_vector(that[j], n), axes=([1], [0]))
    return H


def _biharmonic_power(kind, r, theta):
    if kind == o.BIHARMONIC:
        return 1.0 / np.asarray(r)
    return _orig["kernel_of_r"](kind, r, theta)


def _tt_round_variant(cores, eps, r_update="RT", sqrt_d=True, orthogonalise=True, delta_first=False):
    """The oracle's TT-Round with one step changed: the update of the left neighbour, the
    sqrt(N-1) of the threshold, the orthogonalisation sweep, or the norm delta is taken from."""
    G = [np.array(c, dtype=np.float64) for c in cores]
    N = len(G)
    norm_before = float(np.linalg.norm(G[0]))
    if orthogonalise:
        for i in range(N - 1, 0, -1):
            r0, n, r1 = G[i].shape
            Q, R = np.linalg.qr(o.unfold1(G[i]).T)
            k = Q.shape[1]
            G[i] = Q.T.reshape(k, n, r1, order="F")
            a, m, _ = G[i - 1].shape
            G[i - 1] = (o.unfold2(G[i - 1]) @ (R.T if r_update == "RT" else R)).reshape(a, m, k, order="F")
    nrm = norm_before if delta_first else float(np.linalg.norm(G[0]))
    delta = eps / (math.sqrt(N - 1) if sqrt_d else 1.0) * nrm
    for i in range(N - 1):
        r0, n, r1 = G[i].shape
        U, s, Vt = np.linalg.svd(o.unfold2(G[i]), full_matrices=False)
        r = o.truncation_rank(s, delta)
        G[i] = U[:, :r].reshape(r0, n, r, order="F")
        _, n2, r2 = G[i + 1].shape
        G[i + 1] = ((s[:r, None] * Vt[:r]) @ o.unfold1(G[i + 1])).reshape(r, n2, r2, order="F")
    return G, [1] + [g.shape[2] for g in G]


def _round_with(**kw):
    return lambda cores, eps: _tt_round_variant(cores, eps, **kw)


_ROUND_PINS = [(pins.test_tt_round_undoes_rank_inflation, {}),
               (pins.test_tt_round_meets_its_tolerance, {"eps": 1e-2}),
               (pins.test_tt_round_matches_tt_svd_of_the_full_tensor, {"eps": 1e-3}),
               (pins.test_tt_round_matches_tt_svd_of_the_full_tensor, {"eps": 1e-6})]


def _hhat_no_half(H):
    return 2.0 * _orig["global_hhat"](H)


def _hhat_h_twice(H):
    rs, rt = H.shape
    Hh = np.zeros((rs + rt, rs + rt))
    Hh[:rs, rs:] = 0.5 * H
    Hh[rs:, :rs] = 0.5 * H            # H where H^T belongs
    return Hh


def _global_keeps_negatives(R, H, eps=0.0, compress=False, definite=True):
    return _orig["global_online"](R, H, eps, compress, False)


def _global_one_term_short(R, H, eps=0.0, compress=False, definite=True):
    Uh, W = _orig["global_online"](R, H, eps, compress, definite)
    if Uh is None:
        return Uh, W
    return Uh[:, :-1], W[:-1, :-1]


_GLOBAL_PINS = [(pins.test_global_1_is_the_psd_part_of_the_symmetric_part, {}),
                (pins.test_global_2_keeps_the_fewest_terms, {"definite": True, "eps": 1e-3}),
                (pins.test_global_2_keeps_the_fewest_terms, {"definite": False, "eps": 3e-2})]


def _twisted_last_untransposed(S, theta_cores, T):
    # the last core filled from T instead of T^T (same shape only when the ranks allow it:
    # a reshape of T's memory as r_t x N_t)
    last = np.asarray(T).reshape(T.shape[1], T.shape[0], 1)
    return [S.reshape(1, S.shape[0], S.shape[1])] + [np.array(g) for g in theta_cores] + [last]


def _twisted_first_transposed(S, theta_cores, T):
    first = np.asarray(S).T.reshape(1, S.shape[0], S.shape[1])
    return [first] + [np.array(g) for g in theta_cores] + [T.T.reshape(T.shape[1], T.shape[0], 1)]


_PHASE4_PINS = [(pins.test_twisted_tt_represents_S_H_T, {"dtheta": 1}),
                (pins.test_twisted_tt_represents_S_H_T, {"dtheta": 2})]


# name -> (replacements, pins that should catch it as (function, kwargs))
CASES = {
    "transform c_0 = 2": ({"cheb_transform_matrix": _transform_c0_two},
                          [(pins.test_transform_inverts_node_values, {"n": 12}),
                           (pins.test_coefficients_of_separable_exponential, {"n": 12})]),
    "extrema instead of roots": ({"cheb_nodes": _nodes_extrema},
                                 [(pins.test_nodes_are_roots_of_T_n, {"n": 5})]),
    "usual interval map": ({"interval_map": _map_usual},
                           [(pins.test_interval_map_is_the_printed_one, {}),
                            (pins.test_basis_is_nodal_and_matches_coefficient_form, {"a": 0.0, "b": 1.0})]),
    "gaussian with 1/2": ({"kernel_of_r": _kernel_half}, [(pins.test_gaussian_has_no_half, {})]),
    "matern gamma(l)": ({"kernel_of_r": _kernel_gamma_l},
                        [(pins.test_matern_general_nu_reduces_to_closed_forms, {"l": 0.5})]),
    "threshold without sqrt(D-1)": ({"tt_svd": _tt_svd_no_sqrt},
                                    [(pins.test_tt_svd_threshold_uses_sqrt_D_minus_1, {})]),
    "rank one too high": ({"truncation_rank": _rank_plus_one},
                          [(pins.test_tt_svd_recovers_known_ranks, {}),
                           (pins.test_tt_svd_threshold_uses_sqrt_D_minus_1, {})]),
    "rank one too low": ({"truncation_rank": _rank_minus_one},
                         [(pins.test_tt_svd_recovers_known_ranks, {}),
                          (pins.test_tt_svd_error_bound_and_rank_caps, {"eps": 1e-2})]),
    "swapped Kronecker index in the face-split product": (
        {"face_split": _face_split_swapped}, [(pins.test_factor_chain_equals_full_interpolant, {})]),
    "row-major core unfolding": ({"unfold2": _unfold2_c_order},
                                 [(pins.test_tt_svd_recovers_known_ranks, {}),
                                  (pins.test_factor_chain_equals_full_interpolant, {})]),
    "target chain on transposed cores": ({"target_factor": _target_factor_transposed},
                                         [(pins.test_factor_chain_equals_full_interpolant, {})]),
    "theta map reversed in H": ({"core_matrix_H": _H_wrong_sign},
                                [(pins.test_factor_chain_equals_full_interpolant, {})]),
    "wrong sign of dtheta_hat/dtheta": ({"core_matrix_dH": _dH_wrong_scale},
                                        [(pins.test_gradients_match_central_differences, {})]),
    "derivative basis scaled": ({"cheb_dvector": _dvector_missing_two},
                                [(pins.test_gradients_match_central_differences, {})]),
    "transposed transform in the mode product": ({"mode_product": _mode_product_transposed},
                                                 [(pins.test_coefficients_of_separable_exponential, {"n": 12})]),
    "grid variables in the order (x, y, theta)": ({"grid_tensor": _grid_order_swapped},
                                                  [(pins.test_grid_entries_are_kernel_values_at_nodes, {})]),
    "apply with the target points reversed": ({"apply": _apply_reversed_points},
                                       [(pins.test_apply_matches_dense_product, {})]),
    "Chebyshev index off by one": ({"cheb_T": _chebT_shifted},
                                   [(pins.test_transform_inverts_node_values, {"n": 12})]),
    "Laplace-2D with the wrong sign": ({"kernel_of_r": _laplace2d_sign},
                                       [(pins.test_multiquadric_and_thin_plate_family_identities, {})]),
    "theta components swapped in H": ({"core_matrix_H": _H_theta_swapped},
                                      [(pins.test_factor_chain_equals_full_interpolant, {})]),
    "bi-harmonic as r^-1": ({"kernel_of_r": _biharmonic_power},
                            [(pins.test_multiquadric_and_thin_plate_family_identities, {})]),
    "TT-Round: left neighbour times R, not R^T": ({"tt_round": _round_with(r_update="R")}, _ROUND_PINS),
    "TT-Round: threshold without sqrt(N-1)": ({"tt_round": _round_with(sqrt_d=False)}, _ROUND_PINS),
    "TT-Round: no orthogonalisation sweep": ({"tt_round": _round_with(orthogonalise=False)}, _ROUND_PINS),
    "TT-Round: delta from the first core before the sweep": (
        {"tt_round": _round_with(delta_first=True)}, _ROUND_PINS),
    "PTTK-Global: H^ without the 1/2": ({"global_hhat": _hhat_no_half}, _GLOBAL_PINS),
    "PTTK-Global: H in place of H^T in H^": ({"global_hhat": _hhat_h_twice}, _GLOBAL_PINS),
    "PTTK-Global: negative eigenvalues kept for a definite kernel": (
        {"global_online": _global_keeps_negatives}, _GLOBAL_PINS),
    "PTTK-Global: compression one term short": ({"global_online": _global_one_term_short}, _GLOBAL_PINS),
    "Phase 4: last core from T, not T^T": ({"twisted_tt": _twisted_last_untransposed}, _PHASE4_PINS),
    "Phase 4: first core from S read transposed": ({"twisted_tt": _twisted_first_transposed}, _PHASE4_PINS),
}


def _fails(fn, kwargs):
    try:
        fn(**kwargs)
    except (AssertionError, ValueError, IndexError, np.linalg.LinAlgError):
        return True
    return False


@pytest.mark.parametrize("name", list(CASES))
def test_pins_catch_planted_mistakes(name, monkeypatch):
    repl, catchers = CASES[name]
    # the unmutated oracle passes every catcher
    for fn, kw in catchers:
        assert not _fails(fn, kw), f"{fn.__name__} fails on the unmutated oracle"
    for attr, fn in repl.items():
        monkeypatch.setattr(o, attr, fn)
    assert any(_fails(fn, kw) for fn, kw in catchers), f"no pin catches: {name}"

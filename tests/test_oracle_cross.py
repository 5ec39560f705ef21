"""Pins of the oracle's TT greedy-cross (Algorithms 5, 6 and 7) and of its random numbers.

The cross approximation is a heuristic; what the mathematics fixes is checked instead:
  * SplitMix64 against the outputs of its published reference code;
  * a matrix of rank r is reproduced exactly once Algorithm 5 has added r pivots;
  * a tensor with exact TT ranks is reproduced exactly, with those ranks;
  * with nested index sets the TT-cross interpolation reproduces the tensor on every fibre
    X(I<=k-1, :, I>k) it was built from (and so on every cross), however far it has converged;
  * on a smooth tensor the error falls with eps, and on the c1 kernel grid the cross build
    agrees with the TT-SVD build.
"""
import json
import os

import numpy as np
import pytest

import oracle.pttk_cross as x
import oracle.pttk_oracle as o

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.json")


def test_splitmix64_matches_the_published_outputs():
    g = json.load(open(GOLDEN))["outputs"]
    for seed, outs in g.items():
        for c, v in enumerate(outs):
            assert x.splitmix64(int(seed), c) == int(v, 0)
    r = x.CounterRNG(0)
    assert [r.u64() for _ in range(2)] == [int(v, 0) for v in g["0"][:2]]


def test_counter_rng_draws_are_uniform():
    r = x.CounterRNG(99)
    counts = np.bincount([r.below(10) for _ in range(50000)], minlength=10)
    assert np.abs(counts / 5000.0 - 1.0).max() < 0.05
    bits = [r.bit() for _ in range(20000)]
    assert abs(np.mean(bits) - 0.5) < 0.02


def _array_phi(X):
    return lambda idx: X[tuple(np.atleast_2d(idx).T)]


def test_update_cross_reproduces_a_rank_r_matrix():
    rng = np.random.default_rng(50)
    A = rng.standard_normal((30, 4)) @ rng.standard_normal((4, 25))
    entry = lambda i, j: A[i, j]
    I, J = [int(np.argmax(np.abs(A).max(axis=1)))], []
    J = [int(np.argmax(np.abs(A[I[0]])))]
    r = x.CounterRNG(5)
    while True:
        piv = x.update_cross(entry, 30, 25, I, J, r)
        if piv is None:
            break
        I.append(piv[0])
        J.append(piv[1])
    assert len(I) == 4
    skel = A[:, J] @ np.linalg.solve(A[np.ix_(I, J)], A[I, :])
    assert o.rel_fro(A, skel) <= 1e-12


def test_greedy_cross_reproduces_an_exact_tt():
    rng = np.random.default_rng(51)
    dims, ranks = (5, 6, 4, 5), [1, 2, 3, 2, 1]
    X = o.tt_full([rng.standard_normal((ranks[k], dims[k], ranks[k + 1])) for k in range(4)])
    cores, rr, left, right, _ = x.tt_greedy_cross(_array_phi(X), dims, 1e-12, x.CounterRNG(11))
    assert rr == ranks
    assert o.rel_fro(X, o.tt_full(cores)) <= 1e-12


def _smooth(dims):
    idx = np.indices(dims)
    return 1.0 / (1.0 + idx.sum(0) + 0.3 * idx[2])


@pytest.mark.parametrize("max_sweeps", [0, 1, 3])
def test_cross_interpolates_on_its_fibres(max_sweeps):
    dims = (6, 5, 7, 6)
    X = _smooth(dims)
    cores, rr, left, right, sw = x.tt_greedy_cross(_array_phi(X), dims, 1e-14, x.CounterRNG(12),
                                                   max_sweeps=max_sweeps)
    Xh = o.tt_full(cores)
    N = len(dims)
    for k in range(1, N + 1):
        for l in left[k - 1]:
            for r in right[k]:
                for i in range(dims[k - 1]):
                    e = l + (i,) + r
                    assert abs(Xh[e] - X[e]) <= 1e-12 * np.abs(X).max()
    # and the nested sets are what the formula needs
    for k in range(1, N):
        assert all(l[:-1] in left[k - 1] for l in left[k])
        assert all(r[1:] in right[k + 1] for r in right[k])
        assert len(left[k]) == len(right[k]) == rr[k]


def test_cross_error_falls_with_eps():
    dims = (6, 5, 7, 6)
    X = _smooth(dims)
    errs, ranks = [], []
    for eps in (1e-3, 1e-6, 1e-9):
        cores, rr, _, _, _ = x.tt_greedy_cross(_array_phi(X), dims, eps, x.CounterRNG(13))
        errs.append(o.rel_fro(X, o.tt_full(cores)))
        ranks.append(sum(rr))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] <= 1e-8
    assert ranks[0] <= ranks[1] <= ranks[2]


def test_greedy_init_gives_nested_invertible_crosses():
    dims = (6, 5, 7, 6)
    X = _smooth(dims)
    left, right = x.greedy_init(_array_phi(X), dims, x.CounterRNG(14))
    for k in range(1, len(dims)):
        assert len(left[k]) == len(right[k]) == 2
        assert left[k][0] != left[k][1] and right[k][0] != right[k][1]
        if k > 1:
            assert all(l[:-1] in left[k - 1] for l in left[k])
        if k < len(dims) - 1:
            assert all(r[1:] in right[k + 1] for r in right[k])
        P = np.array([[X[l + r] for r in right[k]] for l in left[k]])
        assert np.linalg.cond(P) < 1e6


def test_cross_build_of_the_c1_kernel_agrees_with_tt_svd():
    # Gaussian, d = 1, [0,1] vs [2,3], l in [0.5, 2], n = 16: the cross build reaches the
    # coefficient tensor of the full grid, and TT-Round brings its ranks to the TT-SVD's
    boxes = [(0.0, 1.0), (0.5, 2.0), (2.0, 3.0)]
    cc, rr, _ = x.build_offline_cross(o.GAUSS, 1, 1, boxes, 16, 1e-10, 13)
    cs, rs, C = o.build_offline(o.GAUSS, 1, 1, boxes, 16, 1e-10)
    assert o.rel_fro(C, o.tt_full(cc)) <= 1e-10
    _, rr2 = o.tt_round(cc, 1e-10)
    assert all(a <= b + 1 for a, b in zip(rr2, rs))
    X = np.random.default_rng(52).uniform(0.0, 1.0, (200, 1))
    Y = np.random.default_rng(53).uniform(2.0, 3.0, (150, 1))
    Uc, Mc, Vc = o.instantiate(cc, 1, 1, boxes, (1.1,), X, Y)
    Us, Ms, Vs = o.instantiate(cs, 1, 1, boxes, (1.1,), X, Y)
    assert o.rel_fro(Us @ Ms @ Vs.T, Uc @ Mc @ Vc.T) <= 1e-9


# --- planted mistakes, each caught by one of the pins above ----------------------------------

def _cores_inverse_transposed(phi, dims, left, right):
    N = len(dims)
    cores = []
    for k in range(1, N + 1):
        L, Rt = left[k - 1], right[k]
        idx = [l + (i,) + r for r in Rt for i in range(dims[k - 1]) for l in L]
        T = phi(np.array(idx, dtype=np.int64)).reshape(len(L), dims[k - 1], len(Rt), order="F")
        if k < N:
            Pk = phi(np.array([l + r for r in right[k] for l in left[k]], dtype=np.int64))
            Pk = Pk.reshape(len(left[k]), len(right[k]), order="F")
            T = (o.unfold2(T) @ np.linalg.inv(Pk).T).reshape(T.shape, order="F")
        cores.append(T)
    return cores


def _splitmix_wrong_shift(key, counter):
    M = (1 << 64) - 1
    z = (key + (counter + 1) * 0x9E3779B97F4A7C15) & M
    z = ((z ^ (z >> 31)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return z ^ (z >> 31)


MUTATIONS = {
    "P^{-T} in place of P^{-1} in the interpolation": ("cross_cores", _cores_inverse_transposed,
                                                        [(test_cross_interpolates_on_its_fibres, {"max_sweeps": 1}),
                                                         (test_greedy_cross_reproduces_an_exact_tt, {})]),
    "SplitMix64 with a wrong shift": ("splitmix64", _splitmix_wrong_shift,
                                      [(test_splitmix64_matches_the_published_outputs, {})]),
}


@pytest.mark.parametrize("name", list(MUTATIONS))
def test_cross_pins_catch_planted_mistakes(name, monkeypatch):
    attr, fn, catchers = MUTATIONS[name]
    for f, kw in catchers:
        f(**kw)                                            # passes unmutated
    monkeypatch.setattr(x, attr, fn)
    failed = False
    for f, kw in catchers:
        try:
            f(**kw)
        except (AssertionError, ValueError, np.linalg.LinAlgError):
            failed = True
    assert failed, f"no pin catches: {name}"

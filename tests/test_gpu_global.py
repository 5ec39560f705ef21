"""PTTK-Global (Algorithm 4) on the GPU against the oracle's PTTK-Global.

Both sides start from the oracle's TT cores (uploaded with pttk_tt_from_cores), so that the
comparison covers the factor chains on one point set, the thin QR of [S T], H(theta), the
eigendecomposition of R H^ R^T and the selection of eigenpairs. Q and U differ between the
two by rotations (and in directions of [S T] at rounding level), so the tests compare the
products Z W Z^T, the ranks, and the properties of Q.
"""
import math

import numpy as np
import pytest

import oracle.pttk_oracle as o

pytestmark = pytest.mark.gpu

BOXES2 = [(0.0, 1.0), (0.0, 1.0), (0.3, 1.4), (0.0, 1.0), (0.0, 1.0)]   # (x, l, y), d = 2


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_06344_gb300 import pttk as P
    P.load()
    X = np.random.default_rng(40).uniform(0.0, 1.0, (2000, 2))
    cases = {}
    for kern in (o.GAUSS, o.MULTIQUADRIC):
        cores, _, _ = o.build_offline(kern, 2, 1, BOXES2, 12, 1e-10)
        tt = P.TT.from_cores(kern, 2, BOXES2[:2], BOXES2[3:], 1, BOXES2[2:3], 12, cores)
        g = P.Global(tt, torch.tensor(X, device="cuda"))
        tt.free()                       # the Global handle keeps its own copy of the cores
        cases[kern] = (cores, g)
    yield torch, P, X, cases
    for _, g in cases.values():
        g.free()


def _oracle(cores, X, th):
    S, H, T = o.instantiate(cores, 2, 1, BOXES2, th, X, X)
    return S, H, T


@pytest.mark.parametrize("kern,definite,th", [(o.GAUSS, True, 0.7), (o.MULTIQUADRIC, False, 1.2),
                                              (o.GAUSS, False, 1.2)])
def test_global_1_matches_the_oracle(env, kern, definite, th):
    torch, P, X, cases = env
    cores, g = cases[kern]
    S, H, T = _oracle(cores, X, (th,))
    N, k, rs, rt = g.dims
    assert (N, rs, rt) == (len(X), S.shape[1], T.shape[1]) and k == rs + rt
    # Q has orthonormal columns and Q R = [S T]
    Q = g.Q()
    Qh = Q.cpu().numpy()
    assert np.abs(Qh.T @ Qh - np.eye(k)).max() <= 1e-12
    assert o.rel_fro(np.hstack([S, T]), Qh @ g.R()) <= 1e-12
    Zo, Wo = o.global_factors(S, T, H, definite=definite)
    Ko = Zo @ Wo @ Zo.T
    Z, W = g.instantiate((th,), definite=definite)
    assert W.shape == (k, k)
    Kg = (Z @ W @ Z.T).cpu().numpy()
    assert o.rel_fro(Ko, Kg) <= 1e-10
    assert np.abs(Kg - Kg.T).max() <= 1e-13 * np.abs(Kg).max()


@pytest.mark.parametrize("kern,definite,th,eps", [(o.GAUSS, True, 0.7, 1e-4), (o.GAUSS, True, 0.7, 1e-6),
                                                  (o.MULTIQUADRIC, False, 1.2, 1e-4),
                                                  (o.MULTIQUADRIC, False, 1.2, 1e-7)])
def test_global_2_matches_the_oracle(env, kern, definite, th, eps):
    torch, P, X, cases = env
    cores, g = cases[kern]
    S, H, T = _oracle(cores, X, (th,))
    Zo, Wo = o.global_factors(S, T, H, eps, compress=True, definite=definite)
    m = Zo.shape[1]
    K1 = S @ H @ T.T
    nrm = np.linalg.norm(K1)
    # the case is not borderline: one term fewer misses the tolerance by > 1 %
    e_m = np.linalg.norm(Zo @ Wo @ Zo.T - K1) / nrm
    e_less = np.linalg.norm(Zo[:, :-1] @ Wo[:-1, :-1] @ Zo[:, :-1].T - K1) / nrm
    assert e_m <= 0.99 * eps and e_less >= 1.01 * eps
    Z, W = g.instantiate((th,), eps, compress=True, definite=definite)
    assert Z.shape == (len(X), m) and W.shape == (m, m)
    Zh, Wh = Z.cpu().numpy(), W.cpu().numpy()
    assert np.array_equal(Wh, np.diag(np.diag(Wh)))
    assert np.abs(Zh.T @ Zh - np.eye(m)).max() <= 1e-12
    assert o.rel_fro(Zo @ Wo @ Zo.T, Zh @ Wh @ Zh.T) <= 1e-10
    assert np.linalg.norm(Zh @ Wh @ Zh.T - K1) <= eps * nrm


@pytest.mark.parametrize("kern,definite", [(o.GAUSS, True), (o.MULTIQUADRIC, False)])
def test_global_1_batched_over_theta(env, kern, definite):
    """pttk_global_instantiate_batched: W_b of five parameter values in one call against the
    oracle's PTTK-Global-1 at each (1e-10 relative, as the single call), and against the
    single-theta call on the same handle (1e-11: the batch changes only the multisection
    lanes, not the method); B = 0 is a no-op and a theta outside its box is EDOMAIN."""
    torch, P, X, cases = env
    cores, g = cases[kern]
    ths = [0.35, 0.7, 0.95, 1.2, 1.39]
    Wb = g.instantiate_batched(np.array(ths)[:, None], definite=definite)
    Q = g.Q()
    Qh = Q.cpu().numpy()
    for b, th in enumerate(ths):
        S, H, T = _oracle(cores, X, (th,))
        Zo, Wo = o.global_factors(S, T, H, definite=definite)
        Ko = Zo @ Wo @ Zo.T
        Kb = Qh @ Wb[b].cpu().numpy() @ Qh.T
        assert o.rel_fro(Ko, Kb) <= 1e-10, (th, o.rel_fro(Ko, Kb))
        _, W1 = g.instantiate((th,), compress=False, definite=definite)
        assert torch.linalg.norm(W1 - Wb[b]) <= 1e-11 * torch.linalg.norm(W1)
    assert g.instantiate_batched(np.zeros((0, 1))).shape[0] == 0
    with pytest.raises(P.PttkError) as e:
        g.instantiate_batched(np.array([[0.7], [2.0]]))
    assert e.value.status == P.EDOMAIN


def test_global_apply_and_theta_outside_the_box(env):
    torch, P, X, cases = env
    cores, g = cases[o.GAUSS]
    S, H, T = _oracle(cores, X, (0.9,))
    Zo, Wo = o.global_factors(S, T, H, 1e-6, compress=True)
    w = np.random.default_rng(41).standard_normal(len(X))
    Z, W = g.instantiate((0.9,), 1e-6, compress=True)
    y = P.apply(Z, W, Z, torch.tensor(w, device="cuda")).cpu().numpy()
    yo = o.apply(Zo, Wo, Zo, w)
    assert np.linalg.norm(y - yo) <= 1e-10 * np.linalg.norm(yo)
    with pytest.raises(P.PttkError) as ei:
        g.instantiate((1.5,))
    assert ei.value.status == P.EDOMAIN


def test_global_needs_one_box(env):
    torch, P, X, cases = env
    cores, _ = cases[o.GAUSS]
    tt = P.TT.from_cores(o.GAUSS, 2, BOXES2[:2], [(2.0, 3.0), (0.0, 1.0)], 1, BOXES2[2:3], 12, cores)
    with pytest.raises(P.PttkError) as ei:
        P.Global(tt, torch.tensor(X, device="cuda"))
    assert ei.value.status == P.EINVAL
    tt.free()


@pytest.mark.parametrize("N", [1, 100])
def test_global_small_point_sets(env, N):
    # fewer points than columns of [S T] (r_s + r_t = 280): Q is N x N and [S T] is wide
    torch, P, _, cases = env
    cores, _ = cases[o.GAUSS]
    X = np.random.default_rng(42).uniform(0.0, 1.0, (N, 2))
    tt = P.TT.from_cores(o.GAUSS, 2, BOXES2[:2], BOXES2[3:], 1, BOXES2[2:3], 12, cores)
    g = P.Global(tt, torch.tensor(X, device="cuda"))
    tt.free()
    n_, k, rs, rt = g.dims
    assert n_ == N and k == min(N, rs + rt)
    S, H, T = _oracle(cores, X, (0.8,))
    Zo, Wo = o.global_factors(S, T, H)
    Z, W = g.instantiate((0.8,))
    Kg = (Z @ W @ Z.T).cpu().numpy()
    assert o.rel_fro(Zo @ Wo @ Zo.T, Kg) <= 1e-10
    g.free()


def test_global_needs_a_point(env):
    torch, P, _, cases = env
    cores, _ = cases[o.GAUSS]
    tt = P.TT.from_cores(o.GAUSS, 2, BOXES2[:2], BOXES2[3:], 1, BOXES2[2:3], 12, cores)
    with pytest.raises(P.PttkError) as ei:
        P.Global(tt, torch.empty(0, 2, dtype=torch.float64, device="cuda"))
    assert ei.value.status == P.EINVAL
    tt.free()


def test_global_full_size_sampled(env):
    # the paper's synthetic setting in d = 3 (SE kernel, B_s = B_t = [0,1]^3,
    # l in [0.2 sqrt(3), sqrt(3)], N = 1e5, TT tol 1e-5) with n = 12 nodes per mode: Q is 1e5 x 828.
    # Entries of Z W Z^T on a sampled 300 x 300 block.
    torch, P, _, _ = env
    Db = math.sqrt(3.0)
    boxes = [(0.0, 1.0)] * 3 + [(0.2 * Db, Db)] + [(0.0, 1.0)] * 3
    cores, _, _ = o.build_offline(o.GAUSS, 3, 1, boxes, 12, 1e-5)
    X = np.random.default_rng(5).uniform(0.0, 1.0, (100000, 3))
    th = (0.8,)
    S, H, T = o.instantiate(cores, 3, 1, boxes, th, X, X)
    Qo, Ro = o.global_offline(S, T)
    tt = P.TT.from_cores(o.GAUSS, 3, boxes[:3], boxes[4:], 1, boxes[3:4], 12, cores)
    g = P.Global(tt, torch.tensor(X, device="cuda"))
    tt.free()
    I = np.sort(np.random.default_rng(6).choice(len(X), 300, replace=False))
    It = torch.tensor(I, device="cuda")
    _, Wo = o.global_online(Ro, H)
    Z, W = g.instantiate(th)
    Zi = Z[It].cpu().numpy()
    assert o.rel_fro(Qo[I] @ Wo @ Qo[I].T, Zi @ W.cpu().numpy() @ Zi.T) <= 1e-9
    eps = 2e-5                                              # 53 terms, 5 % clear of the next rank
    Uh, W2o = o.global_online(Ro, H, eps, compress=True)
    E = np.zeros((Ro.shape[1], Ro.shape[1]))
    E[:H.shape[0], H.shape[0]:] = H
    C1 = Ro @ E @ Ro.T
    e_m = np.linalg.norm(Uh @ W2o @ Uh.T - C1) / np.linalg.norm(C1)
    e_less = np.linalg.norm(Uh[:, :-1] @ W2o[:-1, :-1] @ Uh[:, :-1].T - C1) / np.linalg.norm(C1)
    assert e_m <= 0.99 * eps and e_less >= 1.01 * eps       # not borderline
    Z2, W2 = g.instantiate(th, eps, compress=True)
    assert Z2.shape[1] == Uh.shape[1]
    Zo2 = Qo[I] @ Uh
    Zi2 = Z2[It].cpu().numpy()
    assert o.rel_fro(Zo2 @ W2o @ Zo2.T, Zi2 @ W2.cpu().numpy() @ Zi2.T) <= 1e-9
    g.free()

"""Algorithm 2 with fixed point sets on the GPU (pttk_fixed_*): Phase 3 (the FP64 factor
chains S = U(X), T = V(Y)) and Phase 4 (TT-Round of the twisted TT [T^(1)(S), G_theta..,
T^(3)(T^T)], Eq. twist), then Algorithm 3 on the rounded theta cores, against the oracle's
phase4 on the same S, T and cores.

Tolerances: the GPU and the oracle round the same tensor X at the same tol, so each represents
X within tol ||X||_F. Their matrices at any theta then differ by at most
2 sqrt(n^d_theta) tol ||X||_F (|T_k| <= 1), checked per theta; ranks are equal. They also take
the same truncation (the GPU's QR stops at 1e-4 delta), so the two rounded matrices agree to
the FP64 bar of 1e-12. With tol = 0 the handle holds the unrounded factors: S H(theta) T^T
within 1e-12 of the oracle's chain.
"""
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


def _case(P, name, n):
    import dataclasses
    w = dataclasses.replace(W.WORKLOADS[name], n=n)
    tt = P.TT.build_offline(w.kernel, w.d, w.src_box, w.tgt_box, w.dtheta, w.theta_box, w.n, w.tol, "fp64")
    return w, tt


def _full_norm(S, cores, T):
    """||X||_F of the twisted tensor, from its cores (no n^D array): the Gram route
    ||X||^2 = trace((S^T S) G (T^T T) G^T) contracted core by core."""
    A = S.T @ S
    for G in cores:
        A = np.einsum("ab,akc,bkd->cd", A, G, G)
    return math.sqrt(float(np.sum(A * (T.T @ T))))


@pytest.mark.parametrize("name,n,Ns,Nt,tol", [("c2", 8, 700, 650, 1e-6), ("c3", 5, 900, 800, 1e-8),
                                              ("c1", 16, 300, 280, 1e-10)])
def test_phase4_matches_oracle(env, name, n, Ns, Nt, tol):
    torch, P = env
    w, tt = _case(P, name, n)
    X, Y = W.sources(w, Ns), W.targets(w, Nt)
    f = P.Fixed(tt, torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda"), tol)
    gc = tt.cores()
    # the oracle's Phase 3 on the GPU's cores, then its Phase 4
    S, T = o.instantiate(gc, w.d, w.dtheta, w.mode_boxes(), W.thetas(w, 1)[0], X, Y)[0::2]
    thc = gc[w.d:w.d + w.dtheta]
    S2, c2, T2, ranks = o.phase4(S, thc, T, tol)
    Ns_, Nt_, dth, gr = f.dims
    assert (Ns_, Nt_, dth) == (Ns, Nt, w.dtheta)
    assert gr == ranks[1:-1], (gr, ranks)
    Sg, Tg = f.factors()
    Sg, Tg = Sg.cpu().numpy(), Tg.cpu().numpy()
    assert np.allclose(Sg.T @ Sg, np.eye(Sg.shape[1]), atol=1e-11)
    Xn = _full_norm(S, thc, T)
    box = w.mode_boxes()[w.d:w.d + w.dtheta]
    for th in W.thetas(w, 4):
        Kg = Sg @ f.theta_core(th).cpu().numpy() @ Tg.T
        Ko = S2 @ o.theta_core_matrix(c2, th, box) @ T2.T
        K = S @ o.theta_core_matrix(thc, th, box) @ T.T
        bound = math.sqrt(n ** w.dtheta) * tol * Xn
        assert np.linalg.norm(Kg - K) <= bound
        assert np.linalg.norm(Kg - Ko) <= 2 * bound
        # both round the same tensor with the same truncation (the GPU's QR stops at 1e-4
        # delta), so they agree far inside the tolerance: the FP64 bar of 1e-12
        assert o.rel_fro(Ko, Kg) <= 1e-12, o.rel_fro(Ko, Kg)
    f.free()


def test_phase4_reduces_ranks_and_tol_zero_keeps_them(env):
    torch, P = env
    w, tt = _case(P, "c2", 8)
    # few points: the factors S (N_s x r_s) have rank <= N_s < r_s, so rounding must reduce r_s
    X, Y = W.sources(w, 9), W.targets(w, 7)
    Xd, Yd = torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda")
    f0 = P.Fixed(tt, Xd, Yd, 0.0)
    r = tt.ranks
    assert f0.dims[3] == [r[w.d], r[w.d + 1]]
    th = W.thetas(w, 1)[0]
    U, M, V = P.instantiate(tt, th, Xd, Yd, "fp64")
    S0, T0 = f0.factors()
    K0 = (S0 @ f0.theta_core(th) @ T0.T).cpu().numpy()
    Ki = (U @ M @ V.T).cpu().numpy()
    assert o.rel_fro(Ki, K0) <= 1e-12
    f1 = P.Fixed(tt, Xd, Yd, 1e-12)
    rr = f1.dims[3]
    assert rr[0] <= 9 and rr[-1] <= 7
    S1, T1 = f1.factors()
    K1 = (S1 @ f1.theta_core(th) @ T1.T).cpu().numpy()
    assert o.rel_fro(Ki, K1) <= 1e-10


def test_phase4_rejects_points_outside_and_bad_tol(env):
    torch, P = env
    w, tt = _case(P, "c2", 6)
    X = torch.tensor(W.sources(w, 20), device="cuda")
    Y = torch.tensor(W.targets(w, 20), device="cuda")
    with pytest.raises(P.PttkError) as e:
        P.Fixed(tt, X, Y, 1.5)
    assert e.value.status == P.EINVAL
    Xo = X.clone()
    Xo[3, 0] = 1.0 + 1e-6
    with pytest.raises(P.PttkError) as e:
        P.Fixed(tt, Xo, Y, 1e-8)
    assert e.value.status == P.EDOMAIN
    # the handle still works afterwards
    f = P.Fixed(tt, X, Y, 1e-8)
    assert f.dims[0] == 20


def test_phase4_kernels_without_parameter(env):
    """d_theta = 0 (the TTK variant): the twisted TT is [T^(1)(S), T^(3)(T^T)], H' = I."""
    torch, P = env
    sb, tb = ((0.0, 1.0),) * 2, ((2.0, 3.0), (0.0, 1.0))
    tt = P.TT.build_offline(W.LAPLACE3D, 2, sb, tb, 0, (), 10, 1e-10, "fp64")
    X, Y = W.points_in_box(sb, 120, 1), W.points_in_box(tb, 110, 2)
    Xd, Yd = torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda")
    f = P.Fixed(tt, Xd, Yd, 1e-9)
    S, T = f.factors()
    Kf = (S @ f.theta_core(()) @ T.T).cpu().numpy()
    U, M, V = P.instantiate(tt, (), Xd, Yd, "fp64")
    Ki = (U @ M @ V.T).cpu().numpy()
    assert o.rel_fro(Ki, Kf) <= 1e-8
    gc = tt.cores()
    So, To = o.instantiate(gc, 2, 0, list(sb) + list(tb), (), X, Y)[0::2]
    ranks = o.phase4(So, [], To, 1e-9)[3]
    assert f.dims[3] == ranks[1:-1]

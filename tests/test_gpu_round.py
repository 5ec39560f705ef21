"""TT-Round (Algorithm 1) on the GPU against the oracle's TT-Round.

The GPU rounds in FP64 with the TT-SVD's factorisation (pivoted QR, one-sided Jacobi), its
QR stopping at 1e-4 delta; the oracle with numpy's QR and SVD. Cores differ by rotations, so
the tests compare ranks, the represented tensor (1e-13) and the instantiated K~ (1e-12).
"""
import numpy as np
import pytest

import oracle.pttk_oracle as o
from paper_2406_06344_gb300 import workloads as W
from tests.test_oracle_pins import tt_sum

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_06344_gb300 import pttk as P
    P.load()
    w = W.Workload("c2n8", W.MATERN32, 2, 1, 8, W.C2.src_box, W.C2.tgt_box, W.C2.theta_box, 2000, 4)
    cores, ranks, _ = o.build_offline(w.kernel, w.d, w.dtheta, w.mode_boxes(), w.n, 1e-10)
    return torch, P, w, cores, ranks


def _from_cores(P, w, cores):
    return P.TT.from_cores(w.kernel, w.d, w.src_box, w.tgt_box, w.dtheta, w.theta_box, w.n, cores)


def test_round_undoes_rank_inflation(env):
    torch, P, w, cores, ranks = env
    S = tt_sum(cores, cores)                         # a TT of 2X with doubled ranks
    tt = _from_cores(P, w, S)
    rt = tt.round(1e-10)
    R, oranks = o.tt_round(S, 1e-10)
    # the original is itself truncated at 1e-10, so rounding 2X at 1e-10 may drop one more
    # direction at the middle bonds (the oracle gives 52 where the TT-SVD kept 53)
    assert rt.ranks == oranks
    assert all(a <= b for a, b in zip(oranks, ranks))
    X2 = 2.0 * o.tt_full(cores)
    G = o.tt_full(rt.cores())
    assert o.rel_fro(X2, G) <= 1e-10                  # the bound Algorithm 1 guarantees
    # the same truncation as the oracle's: TT-Round's QR stops at 1e-4 delta (delta = 1e-10 /
    # sqrt(4) of the norm here), so the kept subspaces agree with the exact SVD's to ~1e-14
    assert o.rel_fro(o.tt_full(R), G) <= 1e-13
    # the rounded handle instantiates like the oracle's rounded TT, at the FP64 bar of 1e-12.
    # Against the original, doubled, K~ moves more than the coefficient tensor: the dropped
    # direction is evaluated through the Chebyshev bases (the oracle's own rounded TT sits at
    # 1.96e-9 there)
    X, Y = W.sources(w, 300), W.targets(w, 200)
    th = W.thetas(w, 1)[0]
    U, M, V = P.instantiate(rt, th, torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda"), "fp64")
    rt.check()
    Kg = U.cpu().numpy() @ M.cpu().numpy() @ V.cpu().numpy().T
    Ur, Mr, Vr = o.instantiate(R, w.d, w.dtheta, w.mode_boxes(), th, X, Y)
    assert o.rel_fro(Ur @ Mr @ Vr.T, Kg) <= 1e-12
    Uo, Mo, Vo = o.instantiate(cores, w.d, w.dtheta, w.mode_boxes(), th, X, Y)
    assert o.rel_fro(2 * Uo @ Mo @ Vo.T, Kg) <= 5e-9
    rt.free()
    tt.free()


@pytest.mark.parametrize("tol", [1e-4, 1e-7])
def test_round_to_a_looser_tolerance(env, tol):
    torch, P, w, cores, ranks = env
    tt = _from_cores(P, w, cores)
    rt = tt.round(tol)
    _, oranks = o.tt_round(cores, tol)
    assert rt.ranks == oranks
    assert all(a <= b for a, b in zip(rt.ranks, ranks))
    X = o.tt_full(cores)
    assert o.rel_fro(X, o.tt_full(rt.cores())) <= tol
    # and the same rounded tensor as the oracle's
    R, _ = o.tt_round(cores, tol)
    assert o.rel_fro(o.tt_full(R), o.tt_full(rt.cores())) <= 1e-13
    rt.free()
    tt.free()

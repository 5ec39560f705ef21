"""Full-size parity on the d = 3 general-nu Matern workload (12^8 = 429,981,696-entry grid,
N_s = N_t = 1M points), in the launch configuration the bench times.

  * The FP64 coefficient tensor C, every element, against the oracle's C (written by
    tests/golden/make_oracle_coeffs.py, which calls only the oracle): within 1e-13 of max|C|,
    the bar of the small-grid coefficient tests.
  * The FP64 TT-SVD: ||C - TT||_F <= tol ||C||_F for the TT the GPU builds, against the GPU's C
    and against the oracle's C (the truncation bound of Section 2.3 with tol = 1e-10), and its
    ranks equal to the oracle's.
  * The FP64 SIMT factor chain at N = 1M per side: sampled rows of U and V, and K~ on them,
    within 1e-12 of the oracle's chain on the same cores (factor rows are unique given the
    cores).
"""
import json
import os
import tempfile

import numpy as np
import pytest

import oracle.pttk_oracle as o
from paper_2406_06344_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "oracle_ranks.json")


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_06344_gb300 import pttk as P
    P.load()
    return torch, P


@pytest.fixture(scope="module")
def c3(env):
    """The GPU's FP64 coefficient tensor (flat, column-major) and TT-SVD at tol 1e-10."""
    torch, P = env
    w = W.C3
    C = P.grid_coeffs(w.kernel, w.d, w.src_box, w.tgt_box, w.dtheta, w.theta_box, w.n, "fp64")
    tt = P.TT.from_coeffs(w.kernel, w.d, w.src_box, w.tgt_box, w.dtheta, w.theta_box, w.n, w.tol, C)
    yield C, tt
    tt.free()


def _tt_full(torch, cores):
    """The full tensor of a TT (cores r_{k-1} x n x r_k) on the GPU in FP64, flattened
    column-major (i_1 fastest)."""
    T = None
    for G in cores:
        g = torch.tensor(G, device="cuda")
        r0, n, r1 = g.shape
        if T is None:
            T = g.reshape(n, r1)
            continue
        P_ = T @ g.reshape(r0, n * r1)                     # [(i_1..i_k), (i_{k+1}, b)]
        T = P_.reshape(T.shape[0], n, r1).permute(1, 0, 2).reshape(-1, r1)  # row i_1.. + n^k i_{k+1}
    return T.reshape(-1)


@pytest.mark.slow
def test_c3_coefficients_every_element_match_oracle(env, c3):
    torch, P = env
    from tests.golden.make_oracle_coeffs import cached
    C, _ = c3
    path = os.path.join(tempfile.gettempdir(), "pttk_oracle_c3_coeffs.npy")
    Co = cached("c3", path)
    assert Co.shape == (C.numel(),)
    Cod = torch.from_numpy(np.asarray(Co)).to("cuda")
    err = (C - Cod).abs().max().item()
    assert err <= 1e-13 * Cod.abs().max().item()


def test_c3_tt_svd_reconstruction_within_tolerance(env, c3):
    torch, P = env
    w = W.C3
    C, tt = c3
    assert tt.ranks == json.load(open(GOLDEN))["c3"]["ranks"]
    full = _tt_full(torch, tt.cores())
    assert full.numel() == C.numel()
    err = (torch.linalg.norm(C - full) / torch.linalg.norm(C)).item()
    assert err <= w.tol, err


@pytest.mark.slow
def test_c3_tt_svd_reconstruction_against_oracle_coefficients(env, c3):
    torch, P = env
    from tests.golden.make_oracle_coeffs import cached
    w = W.C3
    _, tt = c3
    Co = torch.from_numpy(np.asarray(cached("c3", os.path.join(tempfile.gettempdir(), "pttk_oracle_c3_coeffs.npy"))))
    Co = Co.to("cuda")
    full = _tt_full(torch, tt.cores())
    err = (torch.linalg.norm(Co - full) / torch.linalg.norm(Co)).item()
    assert err <= w.tol, err


def test_tt_full_helper_matches_oracle_on_small_tt(env):
    """The reconstruction helper above against the oracle's tt_full on a small random TT."""
    torch, _ = env
    rng = np.random.default_rng(3)
    ranks = [1, 3, 4, 2, 1]
    cores = [rng.standard_normal((ranks[k], 5, ranks[k + 1])) for k in range(4)]
    ref = o.tt_full(cores).ravel(order="F")
    got = _tt_full(torch, cores).cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_c3_fp64_chain_full_size_sampled_rows(env, c3):
    torch, P = env
    w = W.C3
    _, tt = c3
    N = w.n_points
    Xd = torch.tensor(W.sources(w), device="cuda")
    Yd = torch.tensor(W.targets(w), device="cuda")
    th = W.thetas(w, 1)[0]
    U, M, V = P.instantiate(tt, th, Xd, Yd, "fp64")
    assert P.load().pttk_tt_check(tt.handle, None) == P.OK
    rng = np.random.default_rng(21)
    rows = np.sort(rng.choice(N, size=2000, replace=False))
    rows[0], rows[-1] = 0, N - 1
    rt = torch.tensor(rows, device="cuda")
    Xs, Ys = Xd[rt].cpu().numpy(), Yd[rt].cpu().numpy()
    Uo, Mo, Vo = o.instantiate(tt.cores(), w.d, w.dtheta, w.mode_boxes(), th, Xs, Ys)
    Ug, Mg, Vg = U[rt].cpu().numpy(), M.cpu().numpy(), V[rt].cpu().numpy()
    assert o.rel_fro(Uo, Ug) <= 1e-12
    assert o.rel_fro(Vo, Vg) <= 1e-12
    assert o.rel_fro(Uo @ Mo @ Vo.T, Ug @ Mg @ Vg.T) <= 1e-12

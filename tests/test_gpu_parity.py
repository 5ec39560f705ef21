"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances:
  * FP64 forms: the coefficient tensor within 1e-13 of max|C| element-wise; K~ within
    1e-12 relative Frobenius of the oracle's K~ (rounding of a few thousand FP64
    operations per entry, amplified by the TT-SVD's conditioning, stays far below this).
  * FP32 forms: within 1e-5 relative Frobenius of the oracle's FP64 K~ (the FP32 target);
    FP32 coefficients within 2e-6 of max|C| (a few FP32 roundings of exp/K_nu values whose
    arguments reach ~20, times the O(n) transform sums).
"""
import dataclasses
import json
import math
import os

import numpy as np
import pytest

import oracle.pttk_oracle as o
from paper_2406_06344_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "oracle_ranks.json")


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def P(torch_cuda):
    from paper_2406_06344_gb300 import pttk
    pttk.load()
    return pttk


def _boxes(w):
    return w.src_box, w.tgt_box, w.theta_box


def _small(w, n=None, **kw):
    """The same workload with another n (for oracle-size cases)."""
    import dataclasses
    return dataclasses.replace(w, n=n or w.n, **kw)


_oracle_cache = {}


def oracle_build(w):
    key = (w.name, w.n, w.tol)
    if key not in _oracle_cache:
        _oracle_cache[key] = o.build_offline(w.kernel, w.d, w.dtheta, w.mode_boxes(), w.n, w.tol)
    return _oracle_cache[key]


def gpu_coeffs(P, w, prec):
    s, t, p = _boxes(w)
    return P.grid_coeffs(w.kernel, w.d, s, t, w.dtheta, p, w.n, prec).cpu().numpy()


# --- grid + transform ---------------------------------------------------------------

@pytest.mark.parametrize("name,n", [("c1", 16), ("c2", 20), ("c2", 7), ("c3", 4), ("c3", 5)])
def test_coefficients_fp64(P, name, n):
    w = _small(W.WORKLOADS[name], n)
    M = o.grid_tensor(o.kernel_f(w.kernel), w.d, w.dtheta, w.mode_boxes(), w.n)
    C = o.coefficient_tensor(M, w.n).ravel(order="F")
    Cg = gpu_coeffs(P, w, "fp64")
    assert Cg.shape == C.shape
    assert np.abs(Cg - C).max() <= 1e-13 * np.abs(C).max()


@pytest.mark.parametrize("name,n", [("c1", 16), ("c2", 20), ("c3", 5)])
def test_coefficients_fp32(P, name, n):
    w = _small(W.WORKLOADS[name], n)
    M = o.grid_tensor(o.kernel_f(w.kernel), w.d, w.dtheta, w.mode_boxes(), w.n)
    C = o.coefficient_tensor(M, w.n).ravel(order="F")
    Cg = gpu_coeffs(P, w, "fp32")
    assert Cg.dtype == np.float32
    assert np.abs(Cg.astype(np.float64) - C).max() <= 2e-6 * np.abs(C).max()


def test_matern_nu_kernel_values_over_wide_range(P):
    # K_nu over z ~ 0.03 .. 130 and nu in [0.5, 2.5]: a 1-D source box close to a long
    # target box; n = 9 puts nodes through the range (the grid's per-nu table spans ~21 pieces)
    w = dataclasses.replace(W.C3, d=1, src_box=((0.0, 0.05),), tgt_box=((0.1, 30.0),), n=9,
                            theta_box=((0.5, 2.0), (0.5, 2.5)))
    M = o.grid_tensor(o.kernel_f(w.kernel), w.d, w.dtheta, w.mode_boxes(), w.n)
    C = o.coefficient_tensor(M, w.n).ravel(order="F")
    Cg = gpu_coeffs(P, w, "fp64")
    assert np.abs(Cg - C).max() <= 1e-13 * np.abs(C).max()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 2e-6)])
def test_matern_nu_on_nearly_one_box(P, prec, tol):
    """Target box = source box shifted by 0.001 in x_1: node distances reach 0.001, so z
    runs from about 5e-4 (below the per-nu table's floor of 1e-3: those entries take the
    quadrature) to about 4 (the table). The oracle's z^nu K_nu(z) form has no value at
    z = 0 itself, so the boxes are not made identical."""
    w = dataclasses.replace(W.C3, d=2, src_box=((0.0, 1.0), (0.0, 1.0)), tgt_box=((0.001, 1.001), (0.0, 1.0)),
                            n=6, theta_box=((0.5, 2.0), (0.5, 2.5)))
    M = o.grid_tensor(o.kernel_f(w.kernel), w.d, w.dtheta, w.mode_boxes(), w.n)
    C = o.coefficient_tensor(M, w.n).ravel(order="F")
    assert np.all(np.isfinite(C))
    Cg = gpu_coeffs(P, w, prec).astype(np.float64)
    assert np.abs(Cg - C).max() <= tol * np.abs(C).max()


# --- TT-SVD ---------------------------------------------------------------------------

def _tt_full_from_gpu(tt):
    return o.tt_full(tt.cores())


@pytest.mark.parametrize("name", ["c1", "c2"])
def test_tt_svd_matches_oracle(P, name):
    w = W.WORKLOADS[name]
    cores, ranks, C = oracle_build(w)
    s, t, p = _boxes(w)
    tt = P.TT.build_offline(w.kernel, w.d, s, t, w.dtheta, p, w.n, w.tol, "fp64")
    assert tt.ranks == ranks
    Tg = _tt_full_from_gpu(tt)
    assert o.rel_fro(C, Tg) <= w.tol
    # same ranks and separated singular values at every cut: the same truncated tensor
    assert o.rel_fro(o.tt_full(cores), Tg) <= 1e-12
    for G in tt.cores()[:-1]:
        G2 = o.unfold2(G)
        assert np.allclose(G2.T @ G2, np.eye(G2.shape[1]), atol=1e-12)


def test_tt_svd_from_given_coefficients_recovers_known_tt(P, torch_cuda):
    # a tensor with an exact TT of known ranks, passed in directly (tall and wide steps)
    rng = np.random.default_rng(11)
    n, ranks = 6, [1, 4, 9, 5, 3, 1]
    cores = [rng.standard_normal((ranks[k], n, ranks[k + 1])) for k in range(5)]
    X = o.tt_full(cores)
    C = torch_cuda.tensor(X.ravel(order="F"), device="cuda")
    tt = P.TT.from_coeffs(P.GAUSS, 2, ((0, 1), (0, 1)), ((2, 3), (0, 1)), 1, ((0.5, 2),), n, 1e-12, C)
    assert tt.ranks == ranks
    assert o.rel_fro(X, _tt_full_from_gpu(tt)) < 1e-12


def test_tt_svd_tolerance_controls_rank(P):
    w = W.C2
    s, t, p = _boxes(w)
    prev = None
    for tol in (1e-4, 1e-7, 1e-10):
        _, ranks, C = o.build_offline(w.kernel, w.d, w.dtheta, w.mode_boxes(), w.n, tol)
        tt = P.TT.build_offline(w.kernel, w.d, s, t, w.dtheta, p, w.n, tol, "fp64")
        assert tt.ranks == ranks
        assert o.rel_fro(C, _tt_full_from_gpu(tt)) <= tol
        if prev is not None:
            assert sum(ranks) >= sum(prev)
        prev = ranks


# --- online: H(theta), factors, apply -----------------------------------------------

def _gpu_tt(P, w, grid_prec="fp64", tol=None):
    s, t, p = _boxes(w)
    return P.TT.build_offline(w.kernel, w.d, s, t, w.dtheta, p, w.n, tol or w.tol, grid_prec)


@pytest.mark.parametrize("name", ["c1", "c2"])
@pytest.mark.parametrize("npts", [1000, 257])
def test_instantiate_fp64_matches_oracle(P, torch_cuda, name, npts):
    torch = torch_cuda
    w = W.WORKLOADS[name]
    cores, ranks, C = oracle_build(w)
    tt = _gpu_tt(P, w)
    X, Y = W.sources(w, npts), W.targets(w, npts + 31)
    Xd, Yd = torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda")
    gcores = tt.cores()
    for th in W.thetas(w, 3):
        U, M, V = P.instantiate(tt, th, Xd, Yd, "fp64")
        Kg = (U @ M @ V.T).cpu().numpy()
        # the online kernels alone: oracle chain on the GPU's cores
        Uo, Mo, Vo = o.instantiate(gcores, w.d, w.dtheta, w.mode_boxes(), th, X, Y)
        assert np.abs(U.cpu().numpy() - Uo).max() <= 1e-13 * np.abs(Uo).max()
        assert np.abs(M.cpu().numpy() - Mo).max() <= 1e-13 * np.abs(Mo).max()
        assert np.abs(V.cpu().numpy() - Vo).max() <= 1e-13 * np.abs(Vo).max()
        # end to end against the oracle's own TT
        Uo, Mo, Vo = o.instantiate(cores, w.d, w.dtheta, w.mode_boxes(), th, X, Y)
        assert o.rel_fro(Uo @ Mo @ Vo.T, Kg) <= 1e-12


@pytest.mark.parametrize("name", ["c1", "c2"])
def test_instantiate_fp32_within_target(P, torch_cuda, name):
    torch = torch_cuda
    w = W.WORKLOADS[name]
    cores, ranks, C = oracle_build(w)
    tt = _gpu_tt(P, w)
    X, Y = W.sources(w, 700), W.targets(w, 650)
    Xf = torch.tensor(X, device="cuda", dtype=torch.float32)
    Yf = torch.tensor(Y, device="cuda", dtype=torch.float32)
    X32, Y32 = Xf.double().cpu().numpy(), Yf.double().cpu().numpy()
    for th in W.thetas(w, 3):
        U, M, V = P.instantiate(tt, th, Xf, Yf, "fp32")
        assert U.dtype == torch.float32
        Kg = (U.double() @ M.double() @ V.double().T).cpu().numpy()
        Uo, Mo, Vo = o.instantiate(cores, w.d, w.dtheta, w.mode_boxes(), th, X32, Y32)
        assert o.rel_fro(Uo @ Mo @ Vo.T, Kg) <= 1e-5


def test_ragged_and_empty_point_sets(P, torch_cuda):
    torch = torch_cuda
    w = W.C2
    tt = _gpu_tt(P, w)
    gcores = tt.cores()
    th = W.thetas(w, 1)[0]
    for ns, nt in ((1, 1), (63, 65), (64, 0), (0, 129), (0, 0)):
        X, Y = W.sources(w, max(ns, 1))[:ns], W.targets(w, max(nt, 1))[:nt]
        Xd = torch.tensor(X, device="cuda").reshape(ns, w.d)
        Yd = torch.tensor(Y, device="cuda").reshape(nt, w.d)
        U, M, V = P.instantiate(tt, th, Xd, Yd, "fp64")
        assert U.shape[0] == ns and V.shape[0] == nt
        Uo, Mo, Vo = o.instantiate(gcores, w.d, w.dtheta, w.mode_boxes(), th,
                                   X.reshape(ns, w.d), Y.reshape(nt, w.d))
        if ns:
            assert np.allclose(U.cpu().numpy(), Uo, rtol=0, atol=1e-13 * max(1, np.abs(Uo).max()))
        if nt:
            assert np.allclose(V.cpu().numpy(), Vo, rtol=0, atol=1e-13 * max(1, np.abs(Vo).max()))


def test_points_on_box_faces_and_theta_on_edges(P, torch_cuda):
    torch = torch_cuda
    w = W.C2
    tt = _gpu_tt(P, w)
    gcores = tt.cores()
    X = np.array([[0.0, 0.0], [1.0, 1.0], [0.0, 1.0], [1.0, 0.0], [0.5, 0.5]])
    Y = np.array([[2.0, 0.0], [3.0, 1.0], [2.5, 0.0], [3.0, 0.5]])
    for th in ((0.2,), (2.0,)):
        U, M, V = P.instantiate(tt, th, torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda"), "fp64")
        Uo, Mo, Vo = o.instantiate(gcores, w.d, w.dtheta, w.mode_boxes(), th, X, Y)
        assert o.rel_fro(Uo @ Mo @ Vo.T, (U @ M @ V.T).cpu().numpy()) < 1e-13
        K = o.kernel_matrix(w.kernel, X, Y, th)
        assert o.rel_fro(K, Uo @ Mo @ Vo.T) < 1e-3


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16x3"])
def test_points_outside_box_record_a_domain_error(P, torch_cuda, prec):
    """Section 1 states the problem for X in B_s and Y in B_t: a point on a face is valid, a
    point beyond it by more than the 1e-12 relative slack records PTTK_EDOMAIN in the status
    word (pttk_tt_check), single and batched."""
    torch = torch_cuda
    w = W.C2
    tt = _gpu_tt(P, w)
    dt = torch.float64 if prec == "fp64" else torch.float32
    th = W.thetas(w, 1)[0]
    Xin = np.array([[0.0, 0.0], [1.0, 1.0], [0.5, 0.25]])
    Yin = np.array([[2.0, 0.0], [3.0, 1.0], [2.5, 0.5]])
    eps_out = 1e-9 if prec == "fp64" else 1e-6
    cases = [(Xin, Yin, P.OK)]
    for side, j, v in ((0, 0, 1.0 + eps_out), (0, 1, -eps_out), (1, 0, 2.0 - 2 * eps_out), (1, 1, 1.0 + eps_out)):
        X, Y = Xin.copy(), Yin.copy()
        (X if side == 0 else Y)[1, j] = v
        cases.append((X, Y, P.EDOMAIN))
    for X, Y, want in cases:
        Xd, Yd = torch.tensor(X, device="cuda", dtype=dt), torch.tensor(Y, device="cuda", dtype=dt)
        P.instantiate(tt, th, Xd, Yd, prec)
        st = P.load().pttk_tt_check(tt.handle, None)
        assert st == want, (X, Y, prec)
        b = P.Batch(tt, [0, 3], [0, 3], prec)
        thetas = torch.tensor([th], device="cuda", dtype=torch.float64)
        b.instantiate(thetas, Xd, Yd)
        st = P.load().pttk_tt_check(tt.handle, None)
        assert st == want, ("batched", X, Y, prec)
        b.free()
    # the status word is cleared by the check: a valid call afterwards reports OK
    P.instantiate(tt, th, torch.tensor(Xin, device="cuda", dtype=dt), torch.tensor(Yin, device="cuda", dtype=dt),
                  prec)
    assert P.load().pttk_tt_check(tt.handle, None) == P.OK


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_domain_check_on_large_point_sets(P, torch_cuda, prec):
    """The check strides over N x d coordinates with the coordinate index carried from step to
    step: d = 3 boxes whose first interval ([3, 4] on the target side) differs from the others,
    N = 400,001 points (several grid strides), one bad coordinate at a time near the start,
    the middle and the ragged end. A bad value is chosen inside another coordinate's
    interval, so a wrong coordinate index would miss it; NaN of either sign and -inf fail,
    and -0.0 on a face at 0 passes."""
    torch = torch_cuda
    w = dataclasses.replace(W.C3, n=6)
    tt = _gpu_tt(P, w, tol=1e-4)
    dt = torch.float64 if prec == "fp64" else torch.float32
    th = W.thetas(w, 1)[0]
    N = 400_001
    X0, Y0 = W.sources(w, N), W.targets(w, N)
    Xd, Yd = torch.tensor(X0, device="cuda", dtype=dt), torch.tensor(Y0, device="cuda", dtype=dt)
    P.instantiate(tt, th, Xd, Yd, prec)
    assert P.load().pttk_tt_check(tt.handle, None) == P.OK
    for side, i, j, v in ((1, N - 1, 1, 3.5), (1, N - 1, 2, 3.5), (1, 200_000, 0, 0.5), (1, 7, 2, 3.0),
                          (0, N - 1, 2, 1.5), (0, 155_649, 1, -0.25), (0, 0, 0, 2.0),
                          (0, 12_345, 1, math.nan), (1, N - 2, 0, -math.inf), (1, 3, 2, -math.nan)):
        Xb, Yb = Xd.clone(), Yd.clone()
        (Xb if side == 0 else Yb)[i, j] = v
        P.instantiate(tt, th, Xb, Yb, prec)
        assert P.load().pttk_tt_check(tt.handle, None) == P.EDOMAIN, (side, i, j, v)
    Xz = Xd.clone()
    Xz[N - 1, 0] = -0.0
    Xz[0, 2] = 0.0
    P.instantiate(tt, th, Xz, Yd, prec)
    assert P.load().pttk_tt_check(tt.handle, None) == P.OK


def test_theta_outside_box_is_a_domain_error(P, torch_cuda):
    w = W.C1
    tt = _gpu_tt(P, w)
    X = torch_cuda.zeros(4, 1, dtype=torch_cuda.float64, device="cuda")
    with pytest.raises(P.PttkError) as e:
        P.instantiate(tt, (2.5,), X, X + 2, "fp64")
    assert e.value.status == P.EDOMAIN
    with pytest.raises(P.PttkError) as e:
        P.theta_core(tt, (0.4,), "fp64")
    assert e.value.status == P.EDOMAIN


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_apply_matches_oracle(P, torch_cuda, prec):
    torch = torch_cuda
    w = W.C2
    tt = _gpu_tt(P, w)
    dt = torch.float64 if prec == "fp64" else torch.float32
    X, Y = W.sources(w, 3000), W.targets(w, 2777)
    wv, _ = W.weights(2777)
    Xd, Yd = torch.tensor(X, device="cuda", dtype=dt), torch.tensor(Y, device="cuda", dtype=dt)
    U, M, V = P.instantiate(tt, W.thetas(w, 1)[0], Xd, Yd, prec)
    out = P.apply(U, M, V, torch.tensor(wv, device="cuda", dtype=dt))
    ref = o.apply(U.double().cpu().numpy(), M.double().cpu().numpy(), V.double().cpu().numpy(), wv)
    tol = 1e-13 if prec == "fp64" else 1e-5
    assert np.linalg.norm(out.double().cpu().numpy() - ref) <= tol * np.linalg.norm(ref)


@pytest.mark.parametrize("rs,rt", [(7000, 8000), (3, 13000)])
def test_apply_large_ranks_matches_oracle(P, torch_cuda, rs, rt):
    """Ranks whose vectors exceed what one CTA could hold in 48 KB of shared memory (6144 FP64
    values): the reduction and both products must still run and agree with the oracle."""
    torch = torch_cuda
    rng = np.random.default_rng(11)
    Ns, Nt = 700, 900
    U, M, V = rng.standard_normal((Ns, rs)), rng.standard_normal((rs, rt)), rng.standard_normal((Nt, rt))
    wv = rng.standard_normal(Nt)
    dev = [torch.tensor(a, device="cuda") for a in (U, M, V, wv)]
    out = P.apply(*dev)
    ref = o.apply(U, M, V, wv)
    assert np.linalg.norm(out.cpu().numpy() - ref) <= 1e-13 * np.linalg.norm(ref)


def test_apply_rejects_mismatched_buffers(P, torch_cuda):
    torch = torch_cuda
    U = torch.zeros(5, 3, dtype=torch.float64, device="cuda")
    M = torch.zeros(3, 4, dtype=torch.float64, device="cuda")
    V = torch.zeros(6, 4, dtype=torch.float64, device="cuda")
    w = torch.zeros(6, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        P.apply(U, M.float(), V, w)
    with pytest.raises(ValueError):
        P.apply(U, M[:2], V, w)
    with pytest.raises(ValueError):
        P.apply(U, M, V, w[:5])
    with pytest.raises(ValueError):
        P.apply(U, M, V, w, out=torch.zeros(4, dtype=torch.float64, device="cuda"))


def test_save_load_roundtrip(P, torch_cuda, tmp_path):
    w = W.C1
    tt = _gpu_tt(P, w)
    path = str(tmp_path / "c1.tt")
    tt.save(path)
    tt2 = P.TT.load(path)
    assert tt2.ranks == tt.ranks and tt2.dims == tt.dims
    for a, b in zip(tt.cores(), tt2.cores()):
        assert np.array_equal(a, b)
    X = torch_cuda.tensor(W.sources(w, 100), device="cuda")
    Y = torch_cuda.tensor(W.targets(w, 90), device="cuda")
    r1 = [t.cpu() for t in P.instantiate(tt, (1.1,), X, Y, "fp64")]
    r2 = [t.cpu() for t in P.instantiate(tt2, (1.1,), X, Y, "fp64")]
    for a, b in zip(r1, r2):
        assert torch_cuda.equal(a, b)


def test_from_cores_with_oracle_cores(P, torch_cuda):
    """A handle made from the oracle's own TT cores: the GPU online stage on them equals the
    oracle's online stage (no GPU TT-SVD involved), and the cores come back unchanged."""
    w = W.C2
    cores, ranks, _ = o.build_offline(w.kernel, w.d, w.dtheta, w.mode_boxes(), 8, 1e-10)
    tt = P.TT.from_cores(w.kernel, w.d, w.src_box, w.tgt_box, w.dtheta, w.theta_box, 8, cores)
    assert tt.ranks == ranks
    for a, b in zip(cores, tt.cores()):
        assert np.array_equal(a, b)
    X = W.sources(w, 777)
    Y = W.targets(w, 555)
    th = W.thetas(w, 1)[0]
    U, M, V = P.instantiate(tt, th, torch_cuda.tensor(X, device="cuda"), torch_cuda.tensor(Y, device="cuda"), "fp64")
    tt.check()
    Uo, Mo, Vo = o.instantiate(cores, w.d, w.dtheta, w.mode_boxes(), th, X, Y)
    Ko = Uo @ Mo @ Vo.T
    assert o.rel_fro(Ko, U.cpu().numpy() @ M.cpu().numpy() @ V.cpu().numpy().T) <= 1e-12
    tt.free()


# --- full-size workloads (sampled checks) ---------------------------------------------

def test_c3_full_size_fp64(P, torch_cuda):
    """C3 at full size (12^8 grid, N = 1M): coefficients checked by the nodal property at
    sampled nodes, ranks equal to the oracle's (tests/golden), the factors of the FP32 SIMT form
    and of the split tensor-core forms (the bench's fast form 3xFP16 among them) checked on
    sampled rows against the oracle's chain on the same cores, and K~ against dense K."""
    torch = torch_cuda
    w = W.C3
    s, t, p = _boxes(w)
    C = P.grid_coeffs(w.kernel, w.d, s, t, w.dtheta, p, w.n, "fp64")
    Ch = C.cpu().numpy().reshape((w.n,) * w.D, order="F")
    # the interpolant reproduces the kernel at the nodes: sum_k C[k] prod_j T_{k_j}(zeta_{i_j}) = m_i
    zeta = o.cheb_nodes(w.n)
    Tz = o.cheb_vector(zeta, w.n)                      # [i, k]
    eta = o.node_vectors(w.mode_boxes(), w.n)
    rng = np.random.default_rng(12)
    f = o.kernel_f(w.kernel)
    for _ in range(4):
        i = rng.integers(0, w.n, size=w.D)
        v = Ch
        for j in range(w.D):
            v = np.tensordot(Tz[i[j]], v, axes=([0], [0]))
        coords = [np.array(eta[j][i[j]]) for j in range(w.D)]
        ref = f(coords[:w.d], coords[w.d:w.d + w.dtheta], coords[w.d + w.dtheta:])
        assert abs(float(v) - float(ref)) <= 1e-12
    tt = P.TT.from_coeffs(w.kernel, w.d, s, t, w.dtheta, p, w.n, w.tol, C)
    del C
    golden = json.load(open(GOLDEN))["c3"]["ranks"]
    assert tt.ranks == golden
    # factors at full N, checked on sampled rows
    N = w.n_points
    Xd = torch.tensor(W.sources(w), device="cuda", dtype=torch.float32)
    Yd = torch.tensor(W.targets(w), device="cuda", dtype=torch.float32)
    th = W.thetas(w, 1)[0]
    U, M, V = P.instantiate(tt, th, Xd, Yd, "fp32")
    rows = np.sort(rng.choice(N, size=300, replace=False))
    rows[-1] = N - 1
    Xs, Ys = Xd[rows].double().cpu().numpy(), Yd[rows].double().cpu().numpy()
    gcores = tt.cores()
    Uo, Mo, Vo = o.instantiate(gcores, w.d, w.dtheta, w.mode_boxes(), th, Xs, Ys)
    Ug, Mg, Vg = U[rows].double().cpu().numpy(), M.double().cpu().numpy(), V[rows].double().cpu().numpy()
    assert o.rel_fro(Uo @ Mo @ Vo.T, Ug @ Mg @ Vg.T) <= 1e-5
    K = o.kernel_matrix(w.kernel, Xs, Ys, th)
    floor = json.load(open(GOLDEN))["c3"]["rel_err_vs_dense_first4_theta"][0]
    assert o.rel_fro(K, Ug @ Mg @ Vg.T) <= 2 * floor + 1e-5
    Ko = Uo @ Mo @ Vo.T
    for form, tol in (("fp16x3", 1e-5), ("tf32x3", 1e-5), ("bf16x3", 3e-5)):
        U, M, V = P.instantiate(tt, th, Xd, Yd, form, U=U, M=M, V=V)
        tt.check()
        Kg = U[rows].double().cpu().numpy() @ M.double().cpu().numpy() @ V[rows].double().cpu().numpy().T
        assert o.rel_fro(Ko, Kg) <= tol, form

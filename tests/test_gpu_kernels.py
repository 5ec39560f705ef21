"""The other kernels of Table kern-table on the GPU: Exponential, Matern-5/2, Multiquadric and
thin-plate spline (theta = (l)), and the parameter-free Bi-harmonic, Laplace-3D, Laplace-2D
and thin-plate kernels (d_theta = 0, the TTK variant, on boxes apart from each other).

Grid coefficients against the oracle's grid and transform; the whole pipeline (grid, TT-SVD,
H, factor chains) against the oracle's chain on the GPU's cores and against dense K.
"""
import numpy as np
import pytest

import oracle.pttk_oracle as o
from paper_2406_06344_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PARAMETRIC = [W.EXPONENTIAL, W.MATERN52, W.MULTIQUADRIC, W.THIN_PLATE_SPLINE]
PLAIN = [W.BIHARMONIC, W.LAPLACE3D, W.LAPLACE2D, W.THIN_PLATE]


def _workload(kernel, n):
    if kernel in PARAMETRIC:
        return W.Workload(W.KERNEL_NAMES[kernel], kernel, 2, 1, n, ((0.0, 1.0), (0.0, 1.0)),
                          ((2.0, 3.0), (0.0, 1.0)), ((0.5, 2.0),), 3000, 4)
    return W.Workload(W.KERNEL_NAMES[kernel], kernel, 2, 0, n, ((0.0, 1.0), (0.0, 1.0)),
                      ((2.0, 3.0), (0.0, 1.0)), (), 3000, 1)


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_06344_gb300 import pttk as P
    P.load()
    return torch, P


@pytest.mark.parametrize("kernel", PARAMETRIC + PLAIN)
def test_grid_coefficients(env, kernel):
    torch, P = env
    w = _workload(kernel, 7)
    M = o.grid_tensor(o.kernel_f(w.kernel), w.d, w.dtheta, w.mode_boxes(), w.n)
    C = o.coefficient_tensor(M, w.n).ravel(order="F")
    for prec, tol in (("fp64", 1e-13), ("fp32", 2e-6)):
        Cg = P.grid_coeffs(w.kernel, w.d, w.src_box, w.tgt_box, w.dtheta, w.theta_box, w.n, prec)
        Cg = Cg.double().cpu().numpy()
        assert np.abs(Cg - C).max() <= tol * np.abs(C).max(), prec


@pytest.mark.parametrize("kernel", PARAMETRIC + PLAIN)
def test_pipeline_against_oracle_and_dense(env, kernel):
    torch, P = env
    w = _workload(kernel, 14)
    tt = P.TT.build_offline(w.kernel, w.d, w.src_box, w.tgt_box, w.dtheta, w.theta_box, w.n, w.tol, "fp64")
    X, Y = W.sources(w, 400), W.targets(w, 300)
    th = tuple(W.thetas(w, 1)[0]) if w.dtheta else ()
    cores = tt.cores()
    Uo, Mo, Vo = o.instantiate(cores, w.d, w.dtheta, w.mode_boxes(), th, X, Y)
    Ko = Uo @ Mo @ Vo.T
    U, M, V = P.instantiate(tt, th, torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda"), "fp64")
    tt.check()
    Kg = U.cpu().numpy() @ M.cpu().numpy() @ V.cpu().numpy().T
    assert o.rel_fro(Ko, Kg) <= 1e-12
    X32 = torch.tensor(X, device="cuda", dtype=torch.float32)
    Y32 = torch.tensor(Y, device="cuda", dtype=torch.float32)
    U, M, V = P.instantiate(tt, th, X32, Y32, "fp16x3")
    tt.check()
    Uo, Mo, Vo = o.instantiate(cores, w.d, w.dtheta, w.mode_boxes(), th, X32.double().cpu().numpy(),
                               Y32.double().cpu().numpy())
    Kg = U.double().cpu().numpy() @ M.double().cpu().numpy() @ V.double().cpu().numpy().T
    assert o.rel_fro(Uo @ Mo @ Vo.T, Kg) <= 1e-5
    # against the kernel itself: with 14 nodes per mode on these boxes the interpolation floor
    # is 1e-11 (Laplace) to 4.5e-6 (thin-plate spline at l = 0.63), by the oracle
    K = o.kernel_matrix(w.kernel, X, Y, th)
    assert o.rel_fro(K, Ko) <= 1e-5
    tt.free()


def test_batched_without_parameter(env):
    torch, P = env
    w = _workload(W.LAPLACE3D, 10)
    tt = P.TT.build_offline(w.kernel, w.d, w.src_box, w.tgt_box, w.dtheta, w.theta_box, w.n, w.tol, "fp64")
    sizes_s, sizes_t = [200, 0, 57], [31, 90, 1]
    X = torch.tensor(W.sources(w, sum(sizes_s)), device="cuda", dtype=torch.float32)
    Y = torch.tensor(W.targets(w, sum(sizes_t)), device="cuda", dtype=torch.float32)
    xoff = np.concatenate([[0], np.cumsum(sizes_s)]).astype(np.int64)
    yoff = np.concatenate([[0], np.cumsum(sizes_t)]).astype(np.int64)
    batch = P.Batch(tt, xoff, yoff, "fp16x3")
    U, M, V = batch.instantiate(torch.empty(len(sizes_s), 0, device="cuda", dtype=torch.float64), X, Y)
    tt.check()
    Mh = M.double().cpu().numpy()
    for b in range(len(sizes_s)):
        assert np.array_equal(Mh[b], np.eye(Mh.shape[1]))
    U1, M1, V1 = P.instantiate(tt, (), X, Y, "fp16x3")
    assert torch.equal(U, U1) and torch.equal(V, V1)
    batch.free()
    tt.free()

"""Batched instantiation (pttk_batch_create / pttk_instantiate_batched) against the oracle.

Every instance b has its own theta_b and point sets (concatenated, offsets xoff/yoff); its
K~_b = U[rows_b] M_b V[rows_b]^T is compared with the oracle's chain on the same TT cores.
Tolerances are those of the single-instance tests for each form.
"""
import numpy as np
import pytest

import oracle.pttk_oracle as o
from paper_2406_06344_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5, "tf32x3": 1e-5, "fp16x3": 1e-5, "bf16x3": 3e-5, "tf32": 2e-3, "fp16": 2e-3,
       "bf16": 2e-2}


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_06344_gb300 import pttk as P
    P.load()
    w = W.C2
    tt = P.TT.build_offline(w.kernel, w.d, w.src_box, w.tgt_box, w.dtheta, w.theta_box, w.n, w.tol, "fp64")
    return torch, P, w, tt, tt.cores()


def _instances(w, sizes_s, sizes_t, seed=0):
    rng = np.random.default_rng(seed)
    X = np.concatenate([W.points_in_box(w.src_box, n, 100 + seed * 1000 + b) for b, n in enumerate(sizes_s)])
    Y = np.concatenate([W.points_in_box(w.tgt_box, n, 200 + seed * 1000 + b) for b, n in enumerate(sizes_t)])
    th = W.points_in_box(w.theta_box, len(sizes_s), 300 + seed)
    xoff = np.concatenate([[0], np.cumsum(sizes_s)]).astype(np.int64)
    yoff = np.concatenate([[0], np.cumsum(sizes_t)]).astype(np.int64)
    return X.reshape(-1, w.d), Y.reshape(-1, w.d), th, xoff, yoff


@pytest.mark.parametrize("form", ["fp64", "fp32", "tf32x3", "fp16x3", "bf16x3", "tf32", "fp16", "bf16"])
def test_batched_matches_oracle_per_instance(env, form):
    torch, P, w, tt, gc = env
    sizes_s = [300, 1, 0, 129, 777, 64, 2000, 5]
    sizes_t = [250, 17, 333, 0, 128, 900, 1, 66]
    X, Y, th, xoff, yoff = _instances(w, sizes_s, sizes_t)
    dt = torch.float64 if form == "fp64" else torch.float32
    Xd = torch.tensor(X, device="cuda", dtype=dt)
    Yd = torch.tensor(Y, device="cuda", dtype=dt)
    thd = torch.tensor(th, device="cuda", dtype=torch.float64)
    batch = P.Batch(tt, xoff, yoff, form)
    U, M, V = batch.instantiate(thd, Xd, Yd)
    tt.check()
    Uh, Mh, Vh = U.double().cpu().numpy(), M.double().cpu().numpy(), V.double().cpu().numpy()
    Xr, Yr = Xd.double().cpu().numpy(), Yd.double().cpu().numpy()
    for b in range(len(sizes_s)):
        xs, ys = slice(xoff[b], xoff[b + 1]), slice(yoff[b], yoff[b + 1])
        Mo = o.core_matrix_H(gc, w.d, w.dtheta, th[b], w.theta_box)
        mtol = 1e-13 if form == "fp64" else 1e-6
        assert np.abs(Mh[b] - Mo).max() <= mtol * np.abs(Mo).max()
        if sizes_s[b] == 0 or sizes_t[b] == 0:
            continue
        Uo, _, Vo = o.instantiate(gc, w.d, w.dtheta, w.mode_boxes(), th[b], Xr[xs], Yr[ys])
        assert o.rel_fro(Uo @ Mo @ Vo.T, Uh[xs] @ Mh[b] @ Vh[ys].T) <= TOL[form]


def test_batched_theta_outside_box_is_reported(env):
    torch, P, w, tt, gc = env
    X, Y, th, xoff, yoff = _instances(w, [10, 10], [10, 10], seed=1)
    th[1, 0] = 2.5   # the length-scale box is [0.2, 2]
    batch = P.Batch(tt, xoff, yoff, "fp32")
    batch.instantiate(torch.tensor(th, device="cuda"), torch.tensor(X, device="cuda", dtype=torch.float32),
                      torch.tensor(Y, device="cuda", dtype=torch.float32))
    with pytest.raises(P.PttkError) as e:
        tt.check()
    assert e.value.status == P.EDOMAIN
    tt.check()  # the status word is cleared once reported


@pytest.mark.parametrize("form", ["tf32x3", "fp16x3"])
def test_batched_under_cuda_graph_and_autotune(env, form):
    """tf32x3 runs the shared-memory-A kernels (its tensor-memory configurations fall back);
    fp16x3 also runs the tensor-memory-A kernel in clusters of 1, 2 and 4."""
    torch, P, w, tt, gc = env
    rng = np.random.default_rng(3)
    sizes_s = list(rng.integers(1, 3000, 40))
    sizes_t = list(rng.integers(1, 3000, 40))
    X, Y, th, xoff, yoff = _instances(w, sizes_s, sizes_t, seed=2)
    Xd = torch.tensor(X, device="cuda", dtype=torch.float32)
    Yd = torch.tensor(Y, device="cuda", dtype=torch.float32)
    thd = torch.tensor(th, device="cuda", dtype=torch.float64)
    batch = P.Batch(tt, xoff, yoff, form)
    U0, M0, V0 = batch.instantiate(thd, Xd, Yd)
    ms = batch.autotune(Xd, Yd, U0, V0)
    assert len(ms) == batch.config[1] and all(m > 0 for m in ms)
    U1, M1, V1 = batch.instantiate(thd, Xd, Yd)   # eager reference with the tuned config
    U, M, V = torch.empty_like(U1), torch.empty_like(M1), torch.empty_like(V1)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        batch.instantiate(thd, Xd, Yd, U=U, M=M, V=V)  # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        batch.instantiate(thd, Xd, Yd, U=U, M=M, V=V)
    U.zero_(); M.zero_(); V.zero_()
    g.replay()
    torch.cuda.synchronize()
    tt.check()
    assert torch.equal(U, U1) and torch.equal(M, M1) and torch.equal(V, V1)
    # every configuration gives the same factors up to the form's rounding
    for c in range(batch.config[1]):
        batch.set_config(c)
        Uc, Mc, Vc = batch.instantiate(thd, Xd, Yd)
        assert (Uc - U1).norm() <= 1e-5 * U1.norm()


@pytest.mark.parametrize("form", ["fp16x3", "tf32x3"])
def test_batched_full_size_1024_instances(env, form):
    """1024 instances, per-side sizes floor(exp(U(ln 1e3, ln 1e5))) (about 22M points per side),
    checked on sampled instances and rows; 3xFP16 is the form the bench times."""
    torch, P, w, tt, gc = env
    ns, nt = W.batched_sizes()
    xoff = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
    yoff = np.concatenate([[0], np.cumsum(nt)]).astype(np.int64)
    Xd = torch.tensor(W.points_in_box(w.src_box, int(xoff[-1]), 61), device="cuda", dtype=torch.float32)
    Yd = torch.tensor(W.points_in_box(w.tgt_box, int(yoff[-1]), 62), device="cuda", dtype=torch.float32)
    th = W.points_in_box(w.theta_box, len(ns), 63)
    batch = P.Batch(tt, xoff, yoff, form)
    U, M, V = batch.instantiate(torch.tensor(th, device="cuda"), Xd, Yd)
    tt.check()
    rng = np.random.default_rng(64)
    for b in list(rng.choice(len(ns), 6, replace=False)) + [len(ns) - 1]:
        rows_x = np.sort(rng.choice(np.arange(xoff[b], xoff[b + 1]), 100, replace=False))
        rows_y = np.sort(rng.choice(np.arange(yoff[b], yoff[b + 1]), 100, replace=False))
        rows_x[-1], rows_y[-1] = xoff[b + 1] - 1, yoff[b + 1] - 1
        Xs, Ys = Xd[rows_x].double().cpu().numpy(), Yd[rows_y].double().cpu().numpy()
        Uo, Mo, Vo = o.instantiate(gc, w.d, w.dtheta, w.mode_boxes(), th[b], Xs, Ys)
        Kg = U[rows_x].double().cpu().numpy() @ M[b].double().cpu().numpy() @ V[rows_y].double().cpu().numpy().T
        assert o.rel_fro(Uo @ Mo @ Vo.T, Kg) <= 1e-5

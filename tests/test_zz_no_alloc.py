"""pttk_apply_noalloc, the allocation-free variant of pttk_apply for callers that cannot
allocate device memory once running (device memory held by another allocator, or a loop
where cudaMalloc/cudaFree could stall or fail). It is called through the C ABI and must agree
with pttk_apply on two calls in a row (its fixed scratch keeps the previous call's contents).
This file is collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_06344_gb300 import pttk as P
    from paper_2406_06344_gb300 import workloads as W
    P.load()
    return torch, P, W


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 1e-5)])
def test_noalloc_apply_matches_apply_on_two_calls(env, prec, tol):
    torch, P, W = env
    lib = P.load()
    w = W.C2
    tt = P.TT.build_offline(w.kernel, w.d, w.src_box, w.tgt_box, w.dtheta, w.theta_box, w.n, w.tol, "fp64")
    dt = torch.float64 if prec == "fp64" else torch.float32
    X = torch.tensor(W.sources(w, 5000), device="cuda", dtype=dt)
    Y = torch.tensor(W.targets(w, 4321), device="cuda", dtype=dt)
    U, M, V = P.instantiate(tt, W.thetas(w, 1)[0], X, Y, prec)
    stream = torch.cuda.current_stream().cuda_stream
    for seed in (5, 6):
        wv = torch.tensor(np.random.default_rng(seed).standard_normal(Y.shape[0]), device="cuda", dtype=dt)
        ref = P.apply(U, M, V, wv)
        out = torch.full_like(ref, float("nan"))
        st = lib.pttk_apply_noalloc(U.data_ptr(), M.data_ptr(), V.data_ptr(), U.shape[0], V.shape[0],
                                    U.shape[1], V.shape[1], P.PREC_NAMES[prec], wv.data_ptr(),
                                    out.data_ptr(), stream)
        assert st == P.OK, lib.pttk_last_error().decode()
        torch.cuda.synchronize()
        err = (out.double() - ref.double()).norm() / ref.double().norm()
        assert err.item() <= tol


@pytest.mark.parametrize("rs,rt,Nt", [(10, 2000, 200_000), (7000, 8000, 900)])
def test_noalloc_apply_matches_apply_with_fewer_blocks_and_large_ranks(env, rs, rt, Nt):
    """(10, 2000, 200k): the fixed scratch holds (131072 - rs) / rt = 65 partial sums of
    V^T w, fewer than the 608 blocks pttk_apply uses at this N_t, so the call runs with fewer
    blocks. (7000, 8000, 900): ranks beyond what 48 KB of shared memory could stage. Two calls
    in a row against pttk_apply, in FP64."""
    torch, P, W = env
    lib = P.load()
    g = torch.Generator(device="cuda").manual_seed(rs + rt)
    Ns = 1500
    U = torch.randn(Ns, rs, generator=g, device="cuda", dtype=torch.float64)
    M = torch.randn(rs, rt, generator=g, device="cuda", dtype=torch.float64)
    V = torch.randn(Nt, rt, generator=g, device="cuda", dtype=torch.float64)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        wv = torch.randn(Nt, generator=g, device="cuda", dtype=torch.float64)
        ref = P.apply(U, M, V, wv)
        out = torch.full_like(ref, float("nan"))
        st = lib.pttk_apply_noalloc(U.data_ptr(), M.data_ptr(), V.data_ptr(), Ns, Nt, rs, rt, P.FP64,
                                    wv.data_ptr(), out.data_ptr(), stream)
        assert st == P.OK, lib.pttk_last_error().decode()
        torch.cuda.synchronize()
        err = (out - ref).norm() / ref.norm()
        assert err.item() <= 1e-13


def test_noalloc_apply_rejects_ranks_beyond_its_scratch(env):
    torch, P, W = env
    lib = P.load()
    rs, rt = 140000, 1            # rs + rt > 131072 FP64 elements (1 MiB)
    U = torch.zeros(1, rs, dtype=torch.float64, device="cuda")
    M = torch.zeros(rs, rt, dtype=torch.float64, device="cuda")
    V = torch.zeros(1, rt, dtype=torch.float64, device="cuda")
    wv = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = lib.pttk_apply_noalloc(U.data_ptr(), M.data_ptr(), V.data_ptr(), 1, 1, rs, rt, P.FP64,
                                wv.data_ptr(), out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == P.EINVAL
    assert "exceeds its fixed scratch" in lib.pttk_last_error().decode()

"""Failure detection without a GPU fault.

Every wait inside the library's kernels is bounded: once it gives up, the kernel records
PTTK_ETIMEOUT and returns, and the CUDA context stays usable. The self-test entry point runs
one such wait on a barrier that nothing ever completes; afterwards an ordinary instantiation
on the same context must still agree with the oracle.
"""
import numpy as np
import pytest

import oracle.pttk_oracle as o
from paper_2406_06344_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_context_survives():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_06344_gb300 import pttk as P
    P.load()
    assert P.selftest_wait_timeout() == P.ETIMEOUT
    assert "gave up" in P.load().pttk_last_error().decode()
    # the context still works: a tensor-core build on it matches the oracle
    w = W.C1
    tt = P.TT.build_offline(w.kernel, w.d, w.src_box, w.tgt_box, w.dtheta, w.theta_box, w.n, w.tol, "fp64")
    X = torch.tensor(W.sources(w, 500), device="cuda", dtype=torch.float32)
    Y = torch.tensor(W.targets(w, 400), device="cuda", dtype=torch.float32)
    th = W.thetas(w, 1)[0]
    U, M, V = P.instantiate(tt, th, X, Y, "fp16x3")
    tt.check()
    Uo, Mo, Vo = o.instantiate(tt.cores(), w.d, w.dtheta, w.mode_boxes(), th, X.double().cpu().numpy(),
                               Y.double().cpu().numpy())
    Kg = U.double().cpu().numpy() @ M.double().cpu().numpy() @ V.double().cpu().numpy().T
    assert o.rel_fro(Uo @ Mo @ Vo.T, Kg) <= 1e-5
    tt.free()

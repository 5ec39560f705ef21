"""Tensor-core (tcgen05) factor chain against the FP64 oracle's chain on the same cores.

Tolerances (relative Frobenius error of U, V and of K~ = U M V^T):
  TF32X3 / FP16X3 / BF16X3  1e-5, 1e-5 and 3e-5: the split forms carry ~22 / ~22 / ~16
                            mantissa bits per operand, and the 1e-5 FP32 target is claimed
                            for TF32X3 and FP16X3;
  TF32 / FP16 / BF16        2e-3 / 2e-3 / 2e-2: single-product forms, 10 / 10 / 7 mantissa
                            bits per operand.
"""
import dataclasses

import numpy as np
import pytest

import oracle.pttk_oracle as o
from paper_2406_06344_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"tf32x3": 1e-5, "fp16x3": 1e-5, "bf16x3": 3e-5, "tf32": 2e-3, "fp16": 2e-3, "bf16": 2e-2}


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_06344_gb300 import pttk as P
    P.load()
    return torch, P


_tts = {}


def tt_for(P, w):
    key = (w.name, w.n)
    if key not in _tts:
        _tts[key] = P.TT.build_offline(w.kernel, w.d, w.src_box, w.tgt_box, w.dtheta, w.theta_box, w.n,
                                       w.tol, "fp64")
    return _tts[key]


def _case(name, n=None):
    w = W.WORKLOADS[name]
    return dataclasses.replace(w, n=n) if n else w


def _run(env, w, form, ns, nt, th_index=0):
    torch, P = env
    tt = tt_for(P, w)
    X = torch.tensor(W.sources(w, max(ns, 1))[:ns], device="cuda", dtype=torch.float32).reshape(ns, w.d)
    Y = torch.tensor(W.targets(w, max(nt, 1))[:nt], device="cuda", dtype=torch.float32).reshape(nt, w.d)
    th = W.thetas(w, th_index + 1)[th_index]
    U, M, V = P.instantiate(tt, th, X, Y, form)
    tt.check()
    gc = tt.cores()
    Uo, Mo, Vo = o.instantiate(gc, w.d, w.dtheta, w.mode_boxes(), th, X.double().cpu().numpy(),
                               Y.double().cpu().numpy())
    return U.double().cpu().numpy(), M.double().cpu().numpy(), V.double().cpu().numpy(), Uo, Mo, Vo


@pytest.mark.parametrize("form", ["tf32", "tf32x3", "bf16", "bf16x3", "fp16", "fp16x3"])
@pytest.mark.parametrize("name,n", [("c1", None), ("c2", None), ("c3", 6)])
def test_tensor_core_chain_matches_oracle(env, form, name, n):
    w = _case(name, n)
    U, M, V, Uo, Mo, Vo = _run(env, w, form, 1000, 777)
    tol = TOL[form]
    assert o.rel_fro(Uo, U) <= tol
    assert o.rel_fro(Vo, V) <= tol
    assert o.rel_fro(Uo @ Mo @ Vo.T, U @ M @ V.T) <= tol


@pytest.mark.parametrize("ns,nt", [(1, 1), (127, 129), (128, 256), (0, 300), (300, 0)])
def test_tensor_core_ragged_tiles(env, ns, nt):
    w = _case("c2")
    U, M, V, Uo, Mo, Vo = _run(env, w, "tf32x3", ns, nt)
    if ns:
        assert o.rel_fro(Uo, U) <= TOL["tf32x3"]
    if nt:
        assert o.rel_fro(Vo, V) <= TOL["tf32x3"]


def test_tensor_core_repeated_calls_are_identical(env):
    torch, P = env
    w = _case("c2")
    tt = tt_for(P, w)
    X = torch.tensor(W.sources(w, 5000), device="cuda", dtype=torch.float32)
    Y = torch.tensor(W.targets(w, 3000), device="cuda", dtype=torch.float32)
    r1 = [t.clone() for t in P.instantiate(tt, (1.0,), X, Y, "tf32x3")]
    r2 = P.instantiate(tt, (1.0,), X, Y, "tf32x3")
    tt.check()
    for a, b in zip(r1, r2):
        assert torch.equal(a, b)


@pytest.mark.parametrize("form", ["fp16", "fp16x3"])
@pytest.mark.parametrize("scales", [(1e6, 1.0), (1.0, 1e-7), (1e-5, 1e5)])
def test_fp16_forms_keep_range_by_scaling(env, form, scales):
    """FP16 overflows at 65504 and loses precision below 6e-5: cores scaled far outside that
    range (source chain by scales[0], target chain by scales[1]) must give the same relative
    accuracy, because the FP16 forms scale operands by powers of two."""
    torch, P = env
    w = _case("c2")
    base = tt_for(P, w).cores()
    cores = [G.copy() for G in base]
    cores[0] *= scales[0]             # first core: the source chain and H
    cores[-1] *= scales[1]            # last core: the target chain
    tt = P.TT.from_cores(w.kernel, w.d, w.src_box, w.tgt_box, w.dtheta, w.theta_box, w.n, cores)
    X = torch.tensor(W.sources(w, 2000), device="cuda", dtype=torch.float32)
    Y = torch.tensor(W.targets(w, 1500), device="cuda", dtype=torch.float32)
    th = W.thetas(w, 1)[0]
    U, M, V = P.instantiate(tt, th, X, Y, form)
    tt.check()
    Uo, Mo, Vo = o.instantiate(cores, w.d, w.dtheta, w.mode_boxes(), th, X.double().cpu().numpy(),
                               Y.double().cpu().numpy())
    Uh, Vh = U.double().cpu().numpy(), V.double().cpu().numpy()
    assert np.isfinite(Uh).all() and np.isfinite(Vh).all()
    assert o.rel_fro(Uo, Uh) <= TOL[form]
    assert o.rel_fro(Vo, Vh) <= TOL[form]
    tt.free()

"""TT greedy-cross (Algorithms 5-7) on the GPU (pttk_cross_build) against the oracle's
greedy-cross (oracle/pttk_cross.py) with the same SplitMix64 key.

Both sides draw the same random numbers in the same order and take each argmin/argmax as the
first index within a relative 1e-12 of the extremum, so they choose the same pivots: the
ranks, the sweep count and the tensor the cores represent agree (the cores up to rounding:
the interpolation formula over the same index sets, 1e-10 relative). A case whose grid the
device could not hold (n = 27, D = 8: 2.8e11 entries, 2.2 TB in FP64) is checked against the
oracle's kernel entries at random multi-indices.
"""
import dataclasses

import numpy as np
import pytest

import oracle.pttk_cross as xo
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


def _nodal(cores, n):
    """Cores of the nodal tensor from coefficient-form cores: G[a, i, b] = sum_k T_k(zeta_i) C[a, k, b]."""
    Tz = o.cheb_vector(o.cheb_nodes(n), n)          # [i, k]
    return [np.einsum("ik,akb->aib", Tz, G) for G in cores]


@pytest.mark.parametrize("name,n,eps,key", [("c1", 16, 1e-10, 7), ("c2", 8, 1e-6, 7), ("c2", 8, 1e-9, 123)])
def test_cross_matches_oracle_pivots(env, name, n, eps, key):
    torch, P = env
    w = dataclasses.replace(W.WORKLOADS[name], n=n)
    oc, oranks, osweeps = xo.build_offline_cross(w.kernel, w.d, w.dtheta, w.mode_boxes(), w.n, eps, key)
    tt, sweeps, evals = P.TT.cross(w.kernel, w.d, w.src_box, w.tgt_box, w.dtheta, w.theta_box, w.n, eps, key)
    assert tt.ranks == oranks
    assert sweeps == osweeps
    full_o = o.tt_full(oc)
    full_g = o.tt_full(tt.cores())
    assert np.linalg.norm(full_g - full_o) <= 1e-10 * np.linalg.norm(full_o)
    assert evals > 0


def test_cross_on_a_grid_the_device_cannot_hold(env):
    """d = 3 general-nu Matern, d_theta = 2, n = 27 (D = 8): the TT's nodal entries at 400
    random multi-indices against the oracle's kernel values there."""
    torch, P = env
    w = dataclasses.replace(W.C3, n=27)
    eps = 1e-4
    tt, sweeps, evals = P.TT.cross(w.kernel, w.d, w.src_box, w.tgt_box, w.dtheta, w.theta_box, w.n, eps, 2024,
                                   max_sweeps=30, n_check=500)
    assert evals < 27 ** 8 / 1000                 # a vanishing share of the grid was evaluated
    nodal = _nodal(tt.cores(), w.n)
    rng = np.random.default_rng(9)
    idx = rng.integers(0, w.n, size=(400, w.D))
    phi = xo.kernel_phi(w.kernel, w.d, w.dtheta, w.mode_boxes(), w.n)
    x = phi(idx)
    xh = xo.tt_entries(nodal, idx)
    assert np.abs(x - xh).max() <= 50 * eps * np.abs(x).max()


def test_cross_rejects_bad_arguments(env):
    torch, P = env
    w = W.C1
    for kw in ({"eps": 0.0}, {"eps": 1e-6, "n_check": 0}, {"eps": 1e-6, "init_it": 0}):
        eps = kw.pop("eps")
        with pytest.raises(P.PttkError) as e:
            P.TT.cross(w.kernel, w.d, w.src_box, w.tgt_box, w.dtheta, w.theta_box, w.n, eps, 1, **kw)
        assert e.value.status == P.EINVAL

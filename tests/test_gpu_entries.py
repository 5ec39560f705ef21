"""Grid-tensor entries at given multi-indices (pttk_grid_entries), the entry access of the TT
greedy-cross, against the oracle's entries (oracle.pttk_cross.kernel_phi)."""
import numpy as np
import pytest

import oracle.pttk_cross as x
import oracle.pttk_oracle as o

pytestmark = pytest.mark.gpu

CASES = [  # kernel, d, d_theta, boxes (x, theta, y), n
    (o.GAUSS, 2, 1, [(0.0, 1.0), (0.0, 1.0), (0.5, 2.0), (2.0, 3.0), (0.0, 1.0)], 20),
    (o.MATERN_NU, 3, 2, [(0.0, 1.0)] * 3 + [(0.5, 2.0), (0.5, 2.5)] + [(3.0, 4.0), (0.0, 1.0), (0.0, 1.0)], 12),
    (o.LAPLACE3D, 3, 0, [(0.0, 1.0)] * 3 + [(3.0, 4.0), (0.0, 1.0), (0.0, 1.0)], 16),
    (o.MULTIQUADRIC, 2, 1, [(0.0, 1.0), (0.0, 1.0), (0.5, 2.0), (0.0, 1.0), (0.0, 1.0)], 27),
]


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_06344_gb300 import pttk as P
    P.load()
    return torch, P


@pytest.mark.parametrize("case", range(len(CASES)))
def test_entries_match_the_oracle(env, case):
    torch, P = env
    kind, d, dth, boxes, n = CASES[case]
    D = 2 * d + dth
    idx = np.random.default_rng(70 + case).integers(0, n, (10001, D)).astype(np.int32)
    ref = x.kernel_phi(kind, d, dth, boxes, n)(idx.astype(np.int64))
    it = torch.tensor(idx, device="cuda")
    for prec, tol in (("fp64", 1e-12), ("fp32", 2e-6)):
        got = P.grid_entries(kind, d, boxes[:d], boxes[d + dth:], dth, boxes[d:d + dth], n, it, prec)
        got = got.double().cpu().numpy()
        assert np.abs(got - ref).max() <= tol * np.abs(ref).max(), prec


def test_entries_beyond_the_whole_grid_limit(env):
    # d = 3, d_theta = 2, n = 32: n^D = 1.1e12 entries, far beyond any grid in memory
    torch, P = env
    kind, d, dth = o.MATERN_NU, 3, 2
    boxes = [(0.0, 1.0)] * 3 + [(0.5, 2.0), (0.5, 2.5)] + [(3.0, 4.0), (0.0, 1.0), (0.0, 1.0)]
    idx = np.random.default_rng(80).integers(0, 32, (4096, 8)).astype(np.int32)
    ref = x.kernel_phi(kind, d, dth, boxes, 32)(idx.astype(np.int64))
    got = P.grid_entries(kind, d, boxes[:3], boxes[5:], dth, boxes[3:5], 32, torch.tensor(idx, device="cuda"))
    assert np.abs(got.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()


def test_an_index_outside_the_grid_is_rejected(env):
    torch, P = env
    kind, d, dth, boxes, n = CASES[0]
    idx = np.random.default_rng(81).integers(0, n, (100, 5)).astype(np.int32)
    idx[37, 2] = n
    idx[38, 0] = -1
    out = torch.zeros(100, dtype=torch.float64, device="cuda")
    with pytest.raises(P.PttkError) as ei:
        P.grid_entries(kind, d, boxes[:d], boxes[d + dth:], dth, boxes[d:d + dth], n,
                       torch.tensor(idx, device="cuda"), out=out)
    assert ei.value.status == P.EINVAL
    o_ = out.cpu().numpy()
    assert np.isnan(o_[37]) and np.isnan(o_[38])
    good = np.ones(100, bool)
    good[[37, 38]] = False
    ref = x.kernel_phi(kind, d, dth, boxes, n)(idx[good].astype(np.int64))
    assert np.abs(o_[good] - ref).max() <= 1e-12 * np.abs(ref).max()

"""The C-ABI library: loads, exports every declared entry point, and rejects bad
arguments on the host (no GPU work is issued by these calls)."""
import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pttk.h")


@pytest.fixture(scope="module")
def so():
    from paper_2406_06344_gb300 import _build, pttk
    if not os.path.exists(pttk.LIB_PATH):
        _build.build()
    return pttk.load()


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pttk_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("pttk_grid_coeffs", "pttk_tt_from_coeffs", "pttk_build_offline", "pttk_tt_ranks",
                 "pttk_tt_save", "pttk_tt_load", "pttk_tt_free", "pttk_theta_core", "pttk_instantiate",
                 "pttk_apply", "pttk_last_error"):
        assert must in names


def test_every_declared_symbol_is_exported(so):
    for name in declared_symbols():
        assert hasattr(so, name), name


def test_binding_covers_every_symbol():
    from paper_2406_06344_gb300 import pttk
    bound = {name for name, _, _ in pttk.SIGNATURES}
    assert set(declared_symbols()) <= bound


def test_version(so):
    assert so.pttk_version() >= 100


def _boxes():
    from paper_2406_06344_gb300 import pttk
    dbl = pttk._dbl
    return dbl([0, 1]), dbl([2, 3]), dbl([0.5, 2.0])


@pytest.mark.parametrize("kernel,d,dth,n,expect", [
    (11, 1, 1, 16, "unknown kernel"),
    (7, 1, 1, 16, "d_theta = 0"),
    (3, 1, 0, 16, "d_theta = 1"),
    (0, 0, 1, 16, "d must be"),
    (0, 4, 1, 16, "d must be"),
    (0, 1, 2, 16, "d_theta = 1"),
    (2, 1, 1, 16, "d_theta = 2"),
    (0, 1, 1, 1, "n must be"),
    (0, 1, 1, 33, "n must be"),
])
def test_invalid_problem_is_rejected(so, kernel, d, dth, n, expect):
    from paper_2406_06344_gb300 import pttk
    s, t, p = _boxes()
    if dth == 2:
        p = pttk._dbl([0.5, 2.0, 0.5, 2.5])
    h = ctypes.c_void_p()
    st = so.pttk_build_offline(kernel, d, s, t, dth, p, n, 1e-10, 0, None, ctypes.byref(h))
    assert st == pttk.EINVAL
    assert expect in so.pttk_last_error().decode()
    assert not h.value


def test_bad_box_and_tol_are_rejected(so):
    from paper_2406_06344_gb300 import pttk
    h = ctypes.c_void_p()
    st = so.pttk_build_offline(0, 1, pttk._dbl([1, 0]), pttk._dbl([2, 3]), 1, pttk._dbl([0.5, 2]), 8,
                               1e-10, 0, None, ctypes.byref(h))
    assert st == pttk.EINVAL and "lo >= hi" in so.pttk_last_error().decode()
    for sb, tb, pb in (([-math.inf, 1], [2, 3], [0.5, 2]), ([0, 1], [2, math.inf], [0.5, 2]),
                       ([0, 1], [2, 3], [0.5, math.inf])):
        st = so.pttk_build_offline(0, 1, pttk._dbl(sb), pttk._dbl(tb), 1, pttk._dbl(pb), 8, 1e-10, 0, None,
                                   ctypes.byref(h))
        assert st == pttk.EINVAL and "finite" in so.pttk_last_error().decode()
    s, t, p = _boxes()
    st = so.pttk_build_offline(0, 1, s, t, 1, p, 8, 0.0, 0, None, ctypes.byref(h))
    assert st == pttk.EINVAL and "tol" in so.pttk_last_error().decode()
    st = so.pttk_build_offline(0, 1, s, t, 1, p, 8, 1e-10, 4, None, ctypes.byref(h))
    assert st == pttk.EINVAL and "precision" in so.pttk_last_error().decode()
    st = so.pttk_grid_coeffs(0, 1, s, t, 1, p, 8, 0, None, None)
    assert st == pttk.EINVAL and "NULL" in so.pttk_last_error().decode()


def test_null_handles_are_rejected(so):
    from paper_2406_06344_gb300 import pttk
    ranks = (ctypes.c_int * 4)()
    assert so.pttk_tt_ranks(None, ranks) == pttk.EINVAL
    assert so.pttk_instantiate(None, None, None, 0, None, 0, 0, None, None, None, None) == pttk.EINVAL
    assert so.pttk_apply(None, None, None, 1, 1, 1, 1, 0, None, None, None) == pttk.EINVAL
    so.pttk_tt_free(None)  # no-op


def test_load_rejects_garbage(so, tmp_path):
    from paper_2406_06344_gb300 import pttk
    p = tmp_path / "bad.tt"
    p.write_bytes(b"not a tensor train")
    h = ctypes.c_void_p()
    assert so.pttk_tt_load(str(p).encode(), ctypes.byref(h)) == pttk.EINVAL
    assert so.pttk_tt_load(str(tmp_path / "missing.tt").encode(), ctypes.byref(h)) == pttk.EINVAL


def test_from_cores_rejects_bad_ranks_without_touching_the_device(so):
    from paper_2406_06344_gb300 import pttk
    s, t, p = _boxes()
    h = ctypes.c_void_p()
    cores = pttk._dbl([0.0] * 64)
    bad_first = (ctypes.c_int * 4)(2, 3, 3, 1)
    assert so.pttk_tt_from_cores(0, 1, s, t, 1, p, 8, bad_first, cores, ctypes.byref(h)) == pttk.EINVAL
    assert "ranks[0]" in so.pttk_last_error().decode()
    bad_mid = (ctypes.c_int * 4)(1, 0, 3, 1)
    assert so.pttk_tt_from_cores(0, 1, s, t, 1, p, 8, bad_mid, cores, ctypes.byref(h)) == pttk.EINVAL
    assert so.pttk_tt_from_cores(0, 1, s, t, 1, p, 8, None, cores, ctypes.byref(h)) == pttk.EINVAL
    assert so.pttk_tt_from_cores(2, 1, s, t, 1, p, 8, bad_first, cores, ctypes.byref(h)) == pttk.EINVAL
    assert not h.value


def test_kernels_without_parameter_need_boxes_apart(so):
    from paper_2406_06344_gb300 import pttk
    h = ctypes.c_void_p()
    touching = so.pttk_build_offline(pttk.LAPLACE3D, 1, pttk._dbl([0, 1]), pttk._dbl([1, 2]), 0, None, 8,
                                     1e-10, 0, None, ctypes.byref(h))
    assert touching == pttk.EINVAL and "apart" in so.pttk_last_error().decode()
    assert not h.value


def test_round_rejects_bad_arguments(so):
    from paper_2406_06344_gb300 import pttk
    h = ctypes.c_void_p()
    assert so.pttk_tt_round(None, 1e-6, None, ctypes.byref(h)) == pttk.EINVAL
    assert not h.value


def test_global_rejects_bad_arguments_without_touching_the_device(so):
    from paper_2406_06344_gb300 import pttk
    h = ctypes.c_void_p()
    assert so.pttk_global_create(None, None, 10, None, ctypes.byref(h)) == pttk.EINVAL
    assert not h.value
    N, k = ctypes.c_int64(), ctypes.c_int()
    assert so.pttk_global_dims(None, ctypes.byref(N), ctypes.byref(k), None, None) == pttk.EINVAL
    assert so.pttk_global_get_q(None, None, None) == pttk.EINVAL
    assert so.pttk_global_get_r(None, None) == pttk.EINVAL
    r = ctypes.c_int()
    assert so.pttk_global_instantiate(None, None, 0.0, 0, 1, None, None, ctypes.byref(r), None) == pttk.EINVAL
    so.pttk_global_free(None)  # no-op


def test_splitmix64_is_the_published_generator_and_the_oracles(so):
    # host-only entry point: the library's stream equals the reference outputs and the
    # oracle's generator, so both sides of the TT greedy-cross draw the same numbers
    import json
    import numpy as np
    from oracle import pttk_cross as x
    from paper_2406_06344_gb300 import pttk
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "splitmix64.json")))["outputs"]
    for seed, outs in g.items():
        for c, v in enumerate(outs):
            assert pttk.splitmix64(int(seed), c) == int(v, 0)
    rng = np.random.default_rng(60)
    for key, c in zip(rng.integers(0, 2**63, 50, dtype=np.int64), rng.integers(0, 2**40, 50, dtype=np.int64)):
        assert pttk.splitmix64(int(key), int(c)) == x.splitmix64(int(key), int(c))


def test_grid_entries_rejects_bad_arguments_without_touching_the_device(so):
    from paper_2406_06344_gb300 import pttk
    box = (ctypes.c_double * 2)(0.0, 1.0)
    tbox = (ctypes.c_double * 2)(2.0, 3.0)
    lbox = (ctypes.c_double * 2)(0.5, 2.0)
    # M > 0 with NULL buffers, a negative count, a bad precision
    assert so.pttk_grid_entries(0, 1, box, tbox, 1, lbox, 8, None, 5, 0, None, None) == pttk.EINVAL
    assert so.pttk_grid_entries(0, 1, box, tbox, 1, lbox, 8, None, -1, 0, None, None) == pttk.EINVAL
    assert so.pttk_grid_entries(0, 1, box, tbox, 1, lbox, 8, None, 0, 2, None, None) == pttk.EINVAL
    # M = 0 is a no-op, also for an n^D far above the whole-grid limit (no grid is formed)
    assert so.pttk_grid_entries(0, 1, box, tbox, 1, lbox, 8, None, 0, 0, None, None) == pttk.OK
    b3 = (ctypes.c_double * 6)(0.0, 1.0, 0.0, 1.0, 0.0, 1.0)
    t3 = (ctypes.c_double * 6)(3.0, 4.0, 0.0, 1.0, 0.0, 1.0)
    p2 = (ctypes.c_double * 4)(0.5, 2.0, 0.5, 2.5)
    assert so.pttk_grid_entries(2, 3, b3, t3, 2, p2, 32, None, 0, 0, None, None) == pttk.OK

"""Writes the FP64 oracle's full Chebyshev coefficient tensor C of a workload (column-major,
i_1 fastest, as a flat .npy) for the element-wise full-size parity test.

Calls only oracle/ and the workload definitions: the grid of Eq. mdc slab by slab of the last
mode, exactly as oracle.pttk_oracle.grid_tensor evaluates it (node vectors, kernel_f on the
broadcast node coordinates), with the slabs spread over worker processes (spawned, so that no
CUDA context is inherited), then oracle.pttk_oracle.coefficient_tensor. The d = 3 general-nu
Matern workload (12^8 entries) takes about a minute on 12 cores and about 25 GB of host memory.
Usage: python tests/golden/make_oracle_coeffs.py c3 OUT.npy
"""
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _slab(args):
    name, last = args
    import oracle.pttk_oracle as o
    from paper_2406_06344_gb300 import workloads as W
    w = W.WORKLOADS[name]
    D = w.D
    eta = o.node_vectors(w.mode_boxes(), w.n)
    grids = np.ix_(*eta[:-1])
    coords = list(grids) + [np.full((1,) * (D - 1), eta[-1][last])]
    f = o.kernel_f(w.kernel)
    return last, np.ascontiguousarray(
        np.broadcast_to(f(coords[:w.d], coords[w.d:w.d + w.dtheta], coords[w.d + w.dtheta:]), (w.n,) * (D - 1)))


def oracle_coeffs(name: str, workers: int = 0) -> np.ndarray:
    """The oracle's C for workload `name`, flattened column-major."""
    import oracle.pttk_oracle as o
    from paper_2406_06344_gb300 import workloads as W
    w = W.WORKLOADS[name]
    M = np.empty((w.n,) * w.D, dtype=np.float64)
    workers = workers or min(w.n, os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        for last, slab in pool.imap_unordered(_slab, [(name, i) for i in range(w.n)]):
            M[..., last] = slab
    C = o.coefficient_tensor(M, w.n)
    del M
    return C.ravel(order="F")


def cached(name: str, path: str) -> np.ndarray:
    """Loads the tensor from `path`, writing it there first when it is missing."""
    if not os.path.exists(path):
        C = oracle_coeffs(name)
        tmp = path + ".tmp.npy"
        np.save(tmp, C)
        os.replace(tmp, path)
        return C
    return np.load(path, mmap_mode="r")


if __name__ == "__main__":
    np.save(sys.argv[2], oracle_coeffs(sys.argv[1]))

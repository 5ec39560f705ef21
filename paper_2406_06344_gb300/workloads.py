"""Seeded synthetic workloads shaped like the paper's experiments.

This module holds configuration constants and random-input generators only; it
contains none of the method's arithmetic, so both the CUDA path's tests and the
CPU oracle's tests draw identical inputs from it.

The paper's workloads are uniform random points in axis-aligned boxes and
uniform random parameters in a parameter box (Section 4.2, Section 4.1,
Appendix C). The five workloads below follow that recipe at the sizes this
library is measured on:

  c1  d=1, dtheta=1, n=16, Gaussian exp(-(r/l)^2), l in [0.5, 2],
      source [0,1], target [2,3], N_s = N_t = 2000, 10 theta, tol 1e-10.
  c2  d=2, dtheta=1, n=20, Matern nu=3/2, l in [0.2, 2],
      source [0,1]^2, target [2,3]x[0,1], N_s = N_t = 200k, 1000 theta.
  c3  d=3, dtheta=2, n=12, Matern general nu, (l, nu) in [0.5,2]x[0.5,2.5],
      source [0,1]^3, target [3,4]x[0,1]^2, N_s = N_t = 1M, 256 theta.
  cb  the c2 tensor train, 1024 instances, per-instance N_s, N_t drawn
      log-uniform in [1e3, 1e5].
  ca  the c3 tensor train, N_s = N_t = 500k, w, z ~ N(0, 1) (adjoint).

Seeds: X = 1, Y = 2, theta = 3, subsample = 4, w/z = 5, batched sizes = 6.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

GAUSS, MATERN32, MATERN_NU = 0, 1, 2
EXPONENTIAL, MATERN52, MULTIQUADRIC, THIN_PLATE_SPLINE = 3, 4, 5, 6
BIHARMONIC, LAPLACE3D, LAPLACE2D, THIN_PLATE = 7, 8, 9, 10      # no parameter (d_theta = 0)
KERNEL_NAMES = {GAUSS: "gaussian", MATERN32: "matern32", MATERN_NU: "matern_nu", EXPONENTIAL: "exponential",
                MATERN52: "matern52", MULTIQUADRIC: "multiquadric", THIN_PLATE_SPLINE: "thin_plate_spline",
                BIHARMONIC: "biharmonic", LAPLACE3D: "laplace3d", LAPLACE2D: "laplace2d", THIN_PLATE: "thin_plate"}

SEED_X, SEED_Y, SEED_THETA, SEED_SUB, SEED_WZ, SEED_SIZES = 1, 2, 3, 4, 5, 6


@dataclass(frozen=True)
class Workload:
    name: str
    kernel: int
    d: int
    dtheta: int
    n: int
    src_box: tuple          # ((lo, hi), ...) length d
    tgt_box: tuple          # ((lo, hi), ...) length d
    theta_box: tuple        # ((lo, hi), ...) length dtheta
    n_points: int
    n_theta: int
    tol: float = 1e-10

    @property
    def D(self) -> int:
        return 2 * self.d + self.dtheta

    def mode_boxes(self) -> np.ndarray:
        """(D, 2) array of (alpha_j, beta_j) in the variable order (x, theta, y)."""
        return np.array(list(self.src_box) + list(self.theta_box) + list(self.tgt_box), dtype=np.float64)


C1 = Workload("c1", GAUSS, 1, 1, 16, ((0.0, 1.0),), ((2.0, 3.0),), ((0.5, 2.0),), 2000, 10)
C2 = Workload("c2", MATERN32, 2, 1, 20, ((0.0, 1.0), (0.0, 1.0)), ((2.0, 3.0), (0.0, 1.0)),
              ((0.2, 2.0),), 200_000, 1000)
C3 = Workload("c3", MATERN_NU, 3, 2, 12, ((0.0, 1.0),) * 3, ((3.0, 4.0), (0.0, 1.0), (0.0, 1.0)),
              ((0.5, 2.0), (0.5, 2.5)), 1_000_000, 256)
WORKLOADS = {w.name: w for w in (C1, C2, C3)}

CB_INSTANCES = 1024
CB_SIZE_RANGE = (1e3, 1e5)
CA_POINTS = 500_000


def points_in_box(box, count: int, seed: int) -> np.ndarray:
    """count x d row-major FP64 points, i.i.d. uniform per coordinate."""
    rng = np.random.default_rng(seed)
    lo = np.array([b[0] for b in box])
    hi = np.array([b[1] for b in box])
    return lo + (hi - lo) * rng.random((count, len(box)))


def sources(w: Workload, count: int | None = None, seed: int = SEED_X) -> np.ndarray:
    return points_in_box(w.src_box, w.n_points if count is None else count, seed)


def targets(w: Workload, count: int | None = None, seed: int = SEED_Y) -> np.ndarray:
    return points_in_box(w.tgt_box, w.n_points if count is None else count, seed)


def thetas(w: Workload, count: int | None = None, seed: int = SEED_THETA) -> np.ndarray:
    return points_in_box(w.theta_box, w.n_theta if count is None else count, seed)


def subsample(n_total: int, count: int, seed: int = SEED_SUB) -> np.ndarray:
    """Sorted indices of a uniform subsample without replacement (error metric, Section 4)."""
    rng = np.random.default_rng(seed)
    if count >= n_total:
        return np.arange(n_total)
    return np.sort(rng.choice(n_total, size=count, replace=False))


def weights(count: int, seed: int = SEED_WZ) -> tuple[np.ndarray, np.ndarray]:
    """w, z ~ N(0, 1) for the scalar loss w^T K z."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(count), rng.standard_normal(count)


def batched_sizes(instances: int = CB_INSTANCES, seed: int = SEED_SIZES) -> tuple[np.ndarray, np.ndarray]:
    """Per-instance (N_s, N_t), each floor(exp(U(ln 1e3, ln 1e5)))."""
    rng = np.random.default_rng(seed)
    lo, hi = np.log(CB_SIZE_RANGE[0]), np.log(CB_SIZE_RANGE[1])
    ns = np.floor(np.exp(rng.uniform(lo, hi, instances))).astype(np.int64)
    nt = np.floor(np.exp(rng.uniform(lo, hi, instances))).astype(np.int64)
    return ns, nt

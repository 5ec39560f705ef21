"""Numerical readings the GPU path rests on, checked on the CPU against SciPy (no GPU, no
library code): the grid's general-nu Matern tabulates G(z) = z^nu e^z K_nu(z) per nu as
piecewise Chebyshev series on geometric pieces [a, 1.5 a] of degree 16. G's one singularity
is a branch point at z = 0, which every such piece sees at the same relative distance
(Bernstein ellipse rho ~ 9.9), so the series' truncation error stays near 1e-17 on every piece."""
import numpy as np
import pytest

special = pytest.importorskip("scipy.special")

Q, DEG = 1.5, 16


def _G(nu, z):
    return np.power(z, nu) * special.kve(nu, z)


def _table(nu, zlo, P):
    k = np.arange(DEG + 1)
    zeta = np.cos((2 * k + 1) * np.pi / (2 * (DEG + 1)))
    Tm = np.cos(np.outer(np.arange(DEG + 1), (2 * k + 1) * np.pi / (2 * (DEG + 1))))
    tabs = []
    for p in range(P):
        a = zlo * Q ** p
        b = a * Q
        vals = _G(nu, 0.5 * (a + b) + 0.5 * (b - a) * zeta)
        c = 2.0 / (DEG + 1) * Tm @ vals
        c[0] *= 0.5
        tabs.append((0.5 * (a + b), 2.0 / (b - a), c))
    return tabs


def _eval(tabs, zlo, z):
    p = min(max(int(np.log2(z / zlo) / np.log2(Q)), 0), len(tabs) - 1)
    mid, ih, c = tabs[p]
    t = (z - mid) * ih
    b1 = b2 = 0.0
    for ck in c[:0:-1]:
        b1, b2 = 2 * t * b1 - b2 + ck, b1
    return t * b1 - b2 + c[0]


@pytest.mark.parametrize("nu", [0.5, 1.0, 1.7, 2.5, 4.0])
def test_piecewise_chebyshev_table_of_k_nu(nu):
    zlo, zhi = 1e-3, 60.0
    P = int(np.ceil(np.log(zhi / zlo) / np.log(Q)))
    tabs = _table(nu, zlo, P)
    rng = np.random.default_rng(7)
    z = np.exp(rng.uniform(np.log(zlo), np.log(zhi), 300))
    approx = np.array([_eval(tabs, zlo, zz) for zz in z])
    ref = _G(nu, z)
    assert np.max(np.abs(approx - ref) / ref) <= 1e-13


@pytest.mark.parametrize("nu", [1.0, 1.7])
def test_degree_eight_is_not_enough(nu):
    """The degree is not slack: on the same pieces degree 8 leaves 1e-12 or more (measured
    4e-12 at nu = 1.7, 2e-11 at nu = 1.0), degree 12 reaches the rounding level. (For
    half-integer nu, G is a polynomial, z^2 + 3z + 3 times a constant at nu = 5/2, and any
    degree from its own is exact.)"""
    global DEG
    old = DEG
    try:
        DEG = 8
        zlo = 1e-3
        P = int(np.ceil(np.log(60.0 / zlo) / np.log(Q)))
        tabs = _table(nu, zlo, P)
        z = np.exp(np.linspace(np.log(0.0011), np.log(59.0), 300))
        err = max(abs(_eval(tabs, zlo, zz) - _G(nu, zz)) / _G(nu, zz) for zz in z)
        assert err > 1e-12
    finally:
        DEG = old

"""Plain FP64 CPU oracle for the TT greedy-cross of arXiv 2406.06344 (Appendix "TT-cross
Approximation" and "TT greedy-cross initialization": Algorithms 5, 6 and 7).

TEST INFRASTRUCTURE ONLY. The GPU library never imports or calls this module and shares no
code with it. Only the tests, ``__graft_entry__.smoke()`` and the CPU baseline leg of
``bench.py`` may use it.

The method draws random numbers (the initial index vectors, the sample sets of each cross
update, the row-or-column bit, the check points of the stopping test). They come from one
counter-based generator, SplitMix64, written from its published definition, so that another
implementation can draw the same numbers.

Readings of the paper taken here:
  X1  Algorithm 5 prints its residual as A(:, I) A(I, J)^{-1} A(J, :) - A, with I and J
      swapped. The reading is the skeleton A(:, J) A(I, J)^{-1} A(I, :) - A, I the row and J
      the column indices.
  X2  "If applicable" in Algorithm 6: a pivot is added only when its residual exceeds
      1e-14 times the largest |entry| the update evaluated; otherwise the index sets stay.
  X3  The TT-cross interpolation formula prints the inverse with indices (s_k, t_k). The
      reading is the standard cross interpolation X^ = T_1 P_1^{-1} T_2 ... P_{N-1}^{-1} T_N,
      T_k = X(I<=k-1, :, I>k), P_k = X(I<=k, I>k): the cores C_k = T_k x_3 P_k^{-T} as
      C_k^{2} = T_k^{2} P_k^{-1}, C_N = T_N.
  X4  The stopping test: the largest |x - x^| over n_check random entries, drawn anew each
      sweep, divided by the largest |x| among them, is <= eps. The sweep count is capped, and
      a sweep that adds no pivot ends the iteration.
  X5  Algorithm 7: the random index vectors q1, q2 hold one index per mode 2..N, uniform in
      that mode. Ties in the condition-number minimum go to the first pair in the order
      (j1, j2) = (0, 0), (0, 1), ...; ties between recorded candidates to the earliest. Every
      argmin and argmax of the method (this minimum, the largest sampled residual and the
      largest residual of the chosen row or column in Algorithm 5) takes the first index whose
      value lies within a relative 1e-12 of the extremum: kernels on symmetric boxes produce
      exactly equal candidates, and an implementation with another rounding order must make
      the same choice among them.
  X6  Sampling without replacement in Algorithm 5: positions drawn uniformly, repeats
      skipped, until max(rows, cols) distinct ones are drawn (all positions when that is
      every one).
"""
from __future__ import annotations

import numpy as np

from oracle import pttk_oracle as po

_MASK64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


def splitmix64(key: int, counter: int) -> int:
    """Output number `counter` (0-based) of SplitMix64 seeded with `key` (Steele, Lea and
    Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): the state after
    counter + 1 increments by the golden gamma, passed through the variant-13 mix."""
    z = (key + (counter + 1) * _GOLDEN) & _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


class CounterRNG:
    """Draws 0, 1, 2, ... of the SplitMix64 stream of `key`."""

    def __init__(self, key: int):
        self.key = key & _MASK64
        self.counter = 0

    def u64(self) -> int:
        v = splitmix64(self.key, self.counter)
        self.counter += 1
        return v

    def below(self, m: int) -> int:
        """An integer in [0, m): the draw modulo m (bias below m / 2^64)."""
        return self.u64() % m

    def bit(self) -> int:
        return self.u64() >> 63


# --- Algorithm 7: initial index sets of cardinality two ------------------------------------

def _cond2(M: np.ndarray) -> float:
    return float(np.linalg.cond(M, 2))


TIE_RTOL = 1e-12


def first_argmax(v: np.ndarray) -> int:
    """The first index i with v[i] >= (1 - TIE_RTOL) max(v) (reading X5)."""
    v = np.asarray(v, dtype=np.float64)
    return int(np.flatnonzero(v >= (1.0 - TIE_RTOL) * v.max())[0])


def first_argmin(v) -> int:
    """The first index i with v[i] <= (1 + TIE_RTOL) min(v) (reading X5)."""
    v = np.asarray(v, dtype=np.float64)
    return int(np.flatnonzero(v <= (1.0 + TIE_RTOL) * v.min())[0])


def greedy_init(phi, dims, rng: CounterRNG, max_it: int = 10):
    """Index sets I<=k, I>k (k = 1..N-1) of cardinality two (Algorithm 7).

    phi maps an (M, N) integer array of multi-indices (0-based) to the M entries. Returns
    (left, right): left[k] and right[k] are lists of two tuples for k = 1..N-1 (index 0 and N
    hold the empty border sets [()])."""
    N = len(dims)
    q1 = [None] + [rng.below(dims[j]) for j in range(1, N)]
    q2 = [None] + [rng.below(dims[j]) for j in range(1, N)]
    left = [[()]] + [None] * (N - 1) + [[()]]
    right = [[()]] + [[tuple(q1[k:]), tuple(q2[k:])] for k in range(1, N)] + [[()]]
    # right[k] holds I>k: indices of modes k+1..N, i.e. 0-based positions k..N-1
    cands = []

    def entries(rows):
        return phi(np.array(rows, dtype=np.int64))

    for _ in range(max_it):
        cs = []
        for k in range(1, N):                       # left-to-right: mode k (1-based)
            p, pp = (left[k - 1] * 2)[:2] if k == 1 else left[k - 1]
            a, b = right[k]
            pairs, conds = [], []
            for j1 in range(dims[k - 1]):
                for j2 in range(dims[k - 1]):
                    if k == 1 and j1 == j2:
                        continue
                    v = entries([p + (j1,) + a, p + (j1,) + b, pp + (j2,) + a, pp + (j2,) + b])
                    pairs.append((j1, j2))
                    conds.append(_cond2(v.reshape(2, 2)))
            q = first_argmin(conds)
            bj, best = pairs[q], conds[q]
            left[k] = [p + (bj[0],), pp + (bj[1],)]
            cs.append(best)
        cands.append(([list(x) for x in left], [list(x) for x in right], max(cs)))
        cs = []
        for k in range(N, 1, -1):                   # right-to-left: mode k (1-based)
            p, pp = left[k - 1]
            a, b = (right[k] * 2)[:2] if k == N else right[k]
            pairs, conds = [], []
            for j1 in range(dims[k - 1]):
                for j2 in range(dims[k - 1]):
                    if k == N and j1 == j2:
                        continue
                    v = entries([p + (j1,) + a, p + (j2,) + b, pp + (j1,) + a, pp + (j2,) + b])
                    pairs.append((j1, j2))
                    conds.append(_cond2(v.reshape(2, 2)))
            q = first_argmin(conds)
            bj, best = pairs[q], conds[q]
            right[k - 1] = [(bj[0],) + a, (bj[1],) + b]
            cs.append(best)
        cands.append(([list(x) for x in left], [list(x) for x in right], max(cs)))
    i = first_argmin([c[2] for c in cands])
    return cands[i][0], cands[i][1]


# --- Algorithm 5: one update of a matrix cross ---------------------------------------------

def update_cross(entry, rows: int, cols: int, I: list, J: list, rng: CounterRNG):
    """One step of Algorithm 5 on the matrix A (rows x cols) whose entries entry(i, j) returns
    for integer arrays i, j. I, J: current row and column indices (same length). Returns the
    new pivot (l, t), or None when its residual is negligible (reading X2)."""
    total = rows * cols
    want = max(rows, cols)
    if want >= total:
        S = np.arange(total, dtype=np.int64)
    else:
        seen, S = set(), []
        while len(S) < want:
            e = rng.below(total)
            if e not in seen:
                seen.add(e)
                S.append(e)
        S = np.array(S, dtype=np.int64)
    si, sj = S % rows, S // rows
    I_ = np.array(I, dtype=np.int64)
    J_ = np.array(J, dtype=np.int64)
    P = entry(np.repeat(I_, len(J_)), np.tile(J_, len(I_))).reshape(len(I_), len(J_))

    def resid(ri, cj):
        """R = A(:, J) A(I, J)^{-1} A(I, :) - A at positions (ri, cj)."""
        left = entry(np.repeat(ri, len(J_)), np.tile(J_, len(ri))).reshape(len(ri), len(J_))
        right = entry(np.repeat(I_, len(cj)), np.tile(cj, len(I_))).reshape(len(I_), len(cj))
        a = entry(ri, cj)
        skel = np.einsum("pj,pj->p", left, np.linalg.solve(P, right).T) if len(I_) else 0.0
        return skel - a, np.abs(a).max() if len(a) else 0.0

    R, amax = resid(si, sj)
    q = first_argmax(np.abs(R))
    l, t = int(si[q]), int(sj[q])
    if rng.bit() == 1:
        Rr, am = resid(np.full(cols, l, dtype=np.int64), np.arange(cols, dtype=np.int64))
        t = first_argmax(np.abs(Rr))
        val = Rr[t]
    else:
        Rc, am = resid(np.arange(rows, dtype=np.int64), np.full(rows, t, dtype=np.int64))
        l = first_argmax(np.abs(Rc))
        val = Rc[l]
    amax = max(amax, am)
    if not abs(val) > 1e-14 * amax or l in I or t in J:
        return None
    return l, t


# --- Algorithm 6 and the interpolation formula ----------------------------------------------

def cross_cores(phi, dims, left, right):
    """Cores of the TT-cross interpolation (reading X3): C_k^{2} = T_k^{2} P_k^{-1} for
    k < N, C_N = T_N, T_k = X(I<=k-1, :, I>k), P_k = X(I<=k, I>k)."""
    N = len(dims)
    cores = []
    for k in range(1, N + 1):
        L, Rt = left[k - 1], right[k]
        idx = [l + (i,) + r for r in Rt for i in range(dims[k - 1]) for l in L]   # column-major
        T = phi(np.array(idx, dtype=np.int64)).reshape(len(L), dims[k - 1], len(Rt), order="F")
        if k < N:
            Pk = phi(np.array([l + r for r in right[k] for l in left[k]], dtype=np.int64))
            Pk = Pk.reshape(len(left[k]), len(right[k]), order="F")
            T2 = po.unfold2(T)
            C2 = np.linalg.solve(Pk.T, T2.T).T
            T = C2.reshape(T.shape, order="F")
        cores.append(T)
    return cores


def tt_entries(cores, idx: np.ndarray) -> np.ndarray:
    """x^_{i_1..i_N} = G_1[:, i_1, :] ... G_N[:, i_N, :] for each row of idx."""
    out = np.ones((idx.shape[0], 1))
    for k, G in enumerate(cores):
        out = np.einsum("pa,apb->pb", out, G[:, idx[:, k], :])
    return out[:, 0]


def tt_greedy_cross(phi, dims, eps: float, rng: CounterRNG, max_sweeps: int = 60, n_check: int = 1000,
                    init_it: int = 10):
    """TT greedy-cross (Algorithm 6): Algorithm 7's index sets, then left-to-right sweeps of
    Algorithm 5 on the unfolded super-cores [X(I<=k-1, :, :, I>k+1)]^{2} (rows s + r_{k-1} i_k,
    columns i_{k+1} + n_{k+1} t) until the sampled Chebyshev-norm error is <= eps (reading X4).
    Returns (cores, ranks, left, right, sweeps)."""
    N = len(dims)
    left, right = greedy_init(phi, dims, rng, init_it)
    sweeps = 0
    while True:
        cores = cross_cores(phi, dims, left, right)
        idx = np.array([[rng.below(n) for n in dims] for _ in range(n_check)], dtype=np.int64)
        x = phi(idx)
        err = np.abs(x - tt_entries(cores, idx)).max() / np.abs(x).max()
        if err <= eps or sweeps >= max_sweeps:
            break
        sweeps += 1
        added = 0
        for k in range(1, N):
            L, Rn = left[k - 1], right[k + 1]
            nk, nk1 = dims[k - 1], dims[k]
            rows, cols = len(L) * nk, nk1 * len(Rn)

            def entry(i, j, L=L, Rn=Rn, nk1=nk1):
                s, ik = i % len(L), i // len(L)
                jk, t = j % nk1, j // nk1
                return phi(np.array([L[a] + (b, c) + Rn[e] for a, b, c, e in zip(s, ik, jk, t)],
                                    dtype=np.int64).reshape(len(i), N))

            I = [L.index(l[:-1]) + len(L) * l[-1] for l in left[k]]
            J = [r[0] + nk1 * Rn.index(r[1:]) for r in right[k]]
            piv = update_cross(entry, rows, cols, I, J, rng)
            if piv is None:
                continue
            l, t = piv
            left[k] = left[k] + [L[l % len(L)] + (l // len(L),)]
            right[k] = right[k] + [(t % nk1,) + Rn[t // nk1]]
            added += 1
        if added == 0:
            break
    return cores, [1] + [len(left[k]) for k in range(1, N)] + [1], left, right, sweeps


def kernel_phi(kind: int, d: int, dtheta: int, mode_boxes, n: int):
    """Entries of the grid tensor M (Eq. mdc) by multi-index: m_{i_1..i_D} =
    f_kappa(eta^{(1)}_{i_1}, ..., eta^{(D)}_{i_D})."""
    eta = po.node_vectors(mode_boxes, n)
    f = po.kernel_f(kind)

    def phi(idx):
        idx = np.atleast_2d(idx)
        coords = [eta[j][idx[:, j]] for j in range(idx.shape[1])]
        return np.asarray(f(coords[:d], coords[d:d + dtheta], coords[d + dtheta:]), dtype=np.float64)
    return phi


def build_offline_cross(kind: int, d: int, dtheta: int, mode_boxes, n: int, eps: float, key: int,
                        **kw):
    """Phases 1-2 of Algorithm 2 with TT greedy-cross on the grid tensor M, then each core
    transformed to Chebyshev coefficients (G_k <- G_k x_2 A, reading R3: the TT of
    C = M x_1 A ... x_D A). Returns (cores, ranks, sweeps)."""
    D = 2 * d + dtheta
    phi = kernel_phi(kind, d, dtheta, mode_boxes, n)
    cores, ranks, _, _, sweeps = tt_greedy_cross(phi, (n,) * D, eps, CounterRNG(key), **kw)
    A = po.cheb_transform_matrix(n)
    return [po.mode_product(G, A, 1) for G in cores], ranks, sweeps

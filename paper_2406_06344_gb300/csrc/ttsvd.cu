// Offline stage, Phase 2 with TT-SVD (Section 2.3; Oseledets 2011, Algorithm 1) in place
// of TT greedy-cross, entirely in FP64 on the device.
//
// Step k (k = 1..D-1) works on the unfolding X (m x c, column-major, m = r_{k-1} n):
//   wide  (c >= m): W = X^T; R = qr_r(W) (Householder); one-sided Jacobi on R gives
//                   R V = U_R Sigma, so the left singular vectors of X are V. The core is
//                   G_k = V[:, top r] and the remainder X <- G_k^T X.
//   tall  (c <  m): R = qr_r(X); Jacobi on R gives Sigma and the right singular vectors V;
//                   Y = X V[:, top r] spans the top-r left singular subspace; a second
//                   Jacobi pass orthogonalises Y's columns (they are nearly orthogonal
//                   already) and G_k is Y with unit columns; X <- G_k^T X.
// In both cases G_k has orthonormal columns to working precision, so G_k G_k^T X is the
// orthogonal projection of X and the discarded part has norm sqrt(sum_{i>r} sigma_i^2).
// r_k is the smallest r >= 1 with that tail <= delta = tol / sqrt(D-1) ||C||_F (the
// threshold of Algorithm 1, TT-Round). QR first keeps singular values down to
// ~1e-16 ||X|| meaningful (a Gram-matrix route would lose everything below ~1e-8 ||X||).
//
// Every kernel is launched as a sequence of independent grids; no kernel waits on another
// CTA, so nothing here can spin.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <chrono>
#include <numeric>
#include <vector>

#include "pttk_internal.cuh"

namespace pttk {
namespace {

constexpr int RC = 1024;  // Householder rows per chunk
constexpr int HU = 8;     // rows per lane per load batch in the Householder passes
constexpr int CG = 32;    // Householder columns per group

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int THREADS>
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (l < THREADS / 32) ? red[l] : 0.0;
    v = warp_sum(v);
  }
  __syncthreads();
  return v;  // valid in warp 0
}

// partial[b] = sum of squares of x over the block's grid-stride share
__global__ void __launch_bounds__(256) sumsq_kernel(const double* __restrict__ x, int64_t n,
                                                    double* __restrict__ partial) {
  __shared__ double red[8];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    acc = fma(x[i], x[i], acc);
  acc = block_sum<256>(acc, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

__global__ void sum_kernel(const double* __restrict__ partial, int np, double* __restrict__ out) {
  __shared__ double red[8];
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc += partial[i];
  acc = block_sum<256>(acc, red);
  if (threadIdx.x == 0) *out = acc;
}

// W (c x m, column-major) = (P X)^T for X m x c column-major, where row i of P X is row
// rowperm[i] of X (rowperm may be null: identity)
__global__ void transpose_kernel(const double* __restrict__ X, int64_t m, int64_t c,
                                 const int* __restrict__ rowperm, double* __restrict__ W) {
  __shared__ double t[32][33];
  const int64_t c0 = (int64_t)blockIdx.x * 32, m0 = (int64_t)blockIdx.y * 32;
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int64_t row = m0 + threadIdx.x, col = c0 + yy;
    if (row < m && col < c) t[yy][threadIdx.x] = X[(rowperm ? rowperm[row] : row) + col * m];
  }
  __syncthreads();
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int64_t row = c0 + threadIdx.x, col = m0 + yy;  // W[row, col] = X[col, row]
    if (row < c && col < m) W[row + col * c] = t[threadIdx.x][yy];
  }
}

// ---------------- Householder QR with column pivoting, truncated --------------------------
// A: M x N column-major (M >= N), overwritten. Step j picks, among the columns not yet
// factored, the one with the largest norm in rows j..M-1 (ties: lowest position), moves it to
// position j, and reflects it: x = A[j:M, p], beta = -sign(x_0) ||x||,
// v = [1; x_{1:}/(x_0 - beta)], tau = (beta - x_0) / beta, H_j = I - tau v v^T,
// H_j x = beta e_1 (LAPACK convention). The factorisation stops before step j as soon as
// the remaining block A[j:M, j:N] (the R22 of A P = Q [R11 R12; 0 R22]) has Frobenius norm
// <= `stop`: then A P = Q [R11 R12] + (a term of norm ||R22||_F), which is what the
// truncated SVD downstream needs, and k = j rows of R are kept.
//
// Columns are never moved: perm[l] is the physical column at position l, the reflector data
// of step j stays in physical column perm[j], and R is stored by physical column,
// Rp[i + N * perm[l]] = R[i, l]. The norm of every remaining column below the next diagonal
// row comes exactly from the update of the previous step (per 1024-row chunk, summed in a
// fixed order), so pivots and the stopping test use exact norms, not downdated ones.
struct HHState {
  double beta, scale, tau;
  double tail2;  // ||R22||_F^2 at the stop (0 if every column was factored)
  int done, k;
};

// part[c * N + p] = sum of A[i, p]^2 over rows i >= 1 of chunk c, for every column p
__global__ void __launch_bounds__(256) hh_init_norms_kernel(const double* __restrict__ A, int64_t M,
                                                            int64_t N, double* __restrict__ part) {
  const int64_t c = blockIdx.x;
  const int64_t r_begin = std::max<int64_t>(c * RC, 1), r_end = std::min<int64_t>((c + 1) * RC, M);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t p = (int64_t)blockIdx.y * CG + warp; p < std::min<int64_t>(N, ((int64_t)blockIdx.y + 1) * CG); p += 8) {
    const double* col = A + p * M;
    double acc = 0.0;
    for (int64_t i = r_begin + lane; i < r_end; i += 32) acc = fma(col[i], col[i], acc);
    acc = warp_sum(acc);
    if (lane == 0) part[c * N + p] = acc;
  }
}

// below[perm[l]] = sum over chunks of part (rows > j), for positions l >= j; one warp per column
__global__ void __launch_bounds__(256) hh_below_kernel(const double* __restrict__ part, int64_t N,
                                                       int64_t j, int64_t nchunks,
                                                       const int* __restrict__ perm,
                                                       const HHState* __restrict__ st,
                                                       double* __restrict__ below) {
  if (st->done) return;
  const int64_t l = j + ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  if (l >= N) return;
  const int p = perm[l];
  double acc = 0.0;
  for (int64_t c = j / RC + lane; c < nchunks; c += 32) acc += part[c * N + p];
  acc = warp_sum(acc);
  if (lane == 0) below[p] = acc;
}

// Pivot choice, stopping test and reflector of step j (one block).
__global__ void __launch_bounds__(1024) hh_pivot_kernel(const double* __restrict__ A, int64_t M,
                                                        int64_t N, int64_t j,
                                                        const double* __restrict__ below,
                                                        int* __restrict__ perm, double stop2,
                                                        HHState* __restrict__ st,
                                                        double* __restrict__ Rp) {
  __shared__ double s_tot[32], s_max[32];
  __shared__ int64_t s_arg[32];
  if (st->done) return;
  double tot = 0.0, best = -1.0;
  int64_t arg = N;
  for (int64_t l = j + threadIdx.x; l < N; l += blockDim.x) {
    const int p = perm[l];
    const double x = A[j + (int64_t)p * M];
    const double t = fma(x, x, below[p]);
    tot += t;
    if (t > best) {  // strictly greater: the lowest position wins ties within a thread
      best = t;
      arg = l;
    }
  }
  // fixed-order block reductions: sum, and max with the lowest position on ties
  for (int o = 16; o; o >>= 1) {
    tot += __shfl_xor_sync(0xffffffffu, tot, o);
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int64_t oa = __shfl_xor_sync(0xffffffffu, arg, o);
    if (ob > best || (ob == best && oa < arg)) {
      best = ob;
      arg = oa;
    }
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    s_tot[w] = tot;
    s_max[w] = best;
    s_arg[w] = arg;
  }
  __syncthreads();
  if (w != 0) return;
  const int nw = blockDim.x >> 5;
  tot = lane < nw ? s_tot[lane] : 0.0;
  best = lane < nw ? s_max[lane] : -1.0;
  arg = lane < nw ? s_arg[lane] : N;
  for (int o = 16; o; o >>= 1) {
    tot += __shfl_xor_sync(0xffffffffu, tot, o);
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int64_t oa = __shfl_xor_sync(0xffffffffu, arg, o);
    if (ob > best || (ob == best && oa < arg)) {
      best = ob;
      arg = oa;
    }
  }
  if (lane != 0) return;
  if (j > 0 && tot <= stop2) {
    st->done = 1;
    st->k = (int)j;
    st->tail2 = tot;
    return;
  }
  if (arg >= N) arg = j;
  const int pj = perm[arg];
  perm[arg] = perm[j];
  perm[j] = pj;
  const double x0 = A[j + (int64_t)pj * M];
  const double acc = below[pj];  // sum of squares strictly below the diagonal
  HHState h = *st;
  if (!(acc > 0.0)) {  // nothing below the diagonal: no reflection
    h.beta = x0;
    h.scale = 0.0;
    h.tau = 0.0;
  } else {
    const double nrm = hypot(x0, sqrt(acc));
    h.beta = (x0 >= 0.0) ? -nrm : nrm;
    h.scale = 1.0 / (x0 - h.beta);
    h.tau = (h.beta - x0) / h.beta;
  }
  h.k = (int)(j + 1);
  *st = h;
  Rp[j + (int64_t)pj * N] = h.beta;
}

// w_part[c * N + l] = sum_{i in chunk c, i >= j} v_i A[i, perm[l]], l in (j, N)
__global__ void __launch_bounds__(256) hh_w_kernel(const double* __restrict__ A, int64_t M,
                                                   int64_t N, int64_t j,
                                                   const int* __restrict__ perm,
                                                   const HHState* __restrict__ st,
                                                   double* __restrict__ w_part) {
  __shared__ double v[RC];
  if (st->done) return;
  const int64_t c = blockIdx.x + j / RC;
  const int64_t r_begin = std::max<int64_t>(c * RC, j), r_end = std::min<int64_t>((c + 1) * RC, M);
  const double scale = st->scale;
  const double* vj = A + (int64_t)perm[j] * M;
  for (int64_t i = r_begin + threadIdx.x; i < r_end; i += blockDim.x)
    v[i - c * RC] = (i == j) ? 1.0 : vj[i] * scale;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t l0 = j + 1 + (int64_t)blockIdx.y * CG;
  for (int q = warp; q < CG; q += 8) {
    const int64_t l = l0 + q;
    if (l >= N) break;
    const double* col = A + (int64_t)perm[l] * M;
    double acc = 0.0;
    for (int64_t i0 = r_begin + lane; i0 < r_end; i0 += 32 * HU) {
      double x[HU];  // HU loads in flight before the arithmetic
#pragma unroll
      for (int u = 0; u < HU; ++u) x[u] = i0 + 32 * u < r_end ? col[i0 + 32 * u] : 0.0;
#pragma unroll
      for (int u = 0; u < HU; ++u)
        if (i0 + 32 * u < r_end) acc = fma(v[i0 + 32 * u - c * RC], x[u], acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) w_part[c * N + l] = acc;
  }
}

// w[l] = tau * sum_c w_part[c * N + l]
__global__ void hh_wsum_kernel(const double* __restrict__ w_part, int64_t N, int64_t j,
                               int64_t nchunks, const HHState* __restrict__ st,
                               double* __restrict__ w) {
  __shared__ double red[8];
  if (st->done) return;
  const int64_t l = j + 1 + blockIdx.x;
  double acc = 0.0;
  for (int64_t c = j / RC + threadIdx.x; c < nchunks; c += blockDim.x) acc += w_part[c * N + l];
  acc = block_sum<256>(acc, red);
  if (threadIdx.x == 0) w[l] = st->tau * acc;
}

// A[i, perm[l]] -= v_i w[l] for rows i >= j; row j of the result is row j of R; the squares
// of rows i >= j+2 (below the next diagonal) go to part[c * N + perm[l]]. One warp per column.
__global__ void __launch_bounds__(256) hh_update_kernel(double* __restrict__ A, int64_t M,
                                                        int64_t N, int64_t j,
                                                        const int* __restrict__ perm,
                                                        const HHState* __restrict__ st,
                                                        const double* __restrict__ w,
                                                        double* __restrict__ Rp,
                                                        double* __restrict__ part) {
  __shared__ double v[RC];
  if (st->done) return;
  const int64_t c = blockIdx.x + j / RC;
  const int64_t r_begin = std::max<int64_t>(c * RC, j), r_end = std::min<int64_t>((c + 1) * RC, M);
  const double scale = st->scale;
  const double* vj = A + (int64_t)perm[j] * M;
  for (int64_t i = r_begin + threadIdx.x; i < r_end; i += blockDim.x)
    v[i - c * RC] = (i == j) ? 1.0 : vj[i] * scale;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t l0 = j + 1 + (int64_t)blockIdx.y * CG;
  for (int q = warp; q < CG; q += 8) {
    const int64_t l = l0 + q;
    if (l >= N) break;
    const int p = perm[l];
    const double wl = w[l];
    double* col = A + (int64_t)p * M;
    double nacc = 0.0;
    for (int64_t i0 = r_begin + lane; i0 < r_end; i0 += 32 * HU) {
      double x[HU];  // HU loads in flight before the arithmetic
#pragma unroll
      for (int u = 0; u < HU; ++u) x[u] = i0 + 32 * u < r_end ? col[i0 + 32 * u] : 0.0;
#pragma unroll
      for (int u = 0; u < HU; ++u) {
        const int64_t i = i0 + 32 * u;
        if (i < r_end) {
          const double a = fma(-v[i - c * RC], wl, x[u]);
          col[i] = a;
          if (i == j) Rp[j + (int64_t)p * N] = a;
          if (i >= j + 2) nacc = fma(a, a, nacc);
        }
      }
    }
    nacc = warp_sum(nacc);
    if (lane == 0) part[c * N + p] = nacc;
  }
}

// At[l + N * i] = R[i, l] = Rp[i + N * perm[l]] for l < N, i < k: the transpose of the kept rows
__global__ void gather_rt_kernel(const double* __restrict__ Rp, int64_t N, int k,
                                 const int* __restrict__ perm, double* __restrict__ At) {
  const int64_t total = N * k;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t l = e % N, i = e / N;
    At[e] = Rp[i + N * (int64_t)perm[l]];
  }
}

// Rd[i + k * l] = R[i, l] = Rp[i + N * perm[l]] for i < k, l < N: the kept rows of R, dense,
// in pivoted column order
__global__ void gather_r_kernel(const double* __restrict__ Rp, int64_t N, int k, const int* __restrict__ perm,
                                double* __restrict__ Rd) {
  const int64_t total = N * k;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % k, l = e / k;
    Rd[e] = Rp[i + N * (int64_t)perm[l]];
  }
}

// V = I (n x n, column-major)
__global__ void eye_kernel(double* __restrict__ V, int64_t n) {
  const int64_t total = n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x)
    V[e] = (e % n == e / n) ? 1.0 : 0.0;
}

__global__ void iota_kernel(int* __restrict__ p, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    p[e] = (int)e;
}

// ---------------- one-sided Jacobi (Hestenes) with round-robin pairing -----------------
// All sweeps of one call run in a single cooperative launch with one block per SM. Round r of
// a sweep pairs the columns (a, b) of the round-robin tournament on p = ncols (+1 if odd)
// players; each warp rotates one pair at a time, and the rounds are separated by a grid
// barrier. Rotation (Rutishauser): zeta = (beta - alpha) / (2 gamma),
// t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1/sqrt(1 + t^2), s = c t,
// [a, b] <- [c a - s b, s a + c b].
// colsq[] holds every column's squared norm (refreshed for the two columns of each
// rotation). A pair whose squared norms are both below `small2` is skipped without being
// read, and a rotation counts toward convergence only if it moves a column of squared norm
// >= `count2` by more than rounding (a rotation of a large column with a far smaller one
// changes only the smaller). The sweeps end when no such rotation is left. With
// small2 = (1e-3 delta)^2 / q and count2 = (1e-2 delta)^2 / q the columns left unsettled carry
// < 1e-4 delta^2 in total, so they change neither the kept subspace nor, except within that
// margin of the threshold, the truncation rank.
// Columns and norms written by other blocks in earlier rounds are read through L2 (ld.cg),
// never from a possibly stale L1 line. A pair's alpha and beta are read from colsq[] (the
// squared norms its last rotation, or the initial pass, summed from the stored columns), so the
// first pass over the pair only forms gamma = a.b. When V is given (vrows x ncols), every
// rotation is applied to V's columns as well, accumulating the right rotation.
constexpr int JB = 256;            // threads per block
constexpr int JU = 8;              // rows per lane per load batch
constexpr int JMAX_SWEEPS = 60;

struct JacobiSync {                // device state of one call (zeroed before the launch)
  alignas(128) unsigned count;     // grid-barrier arrivals
  alignas(128) unsigned gen;       // grid-barrier generation (polled: its own line)
  alignas(128) int err;            // a barrier wait gave up
  int sweeps;                      // sweeps run; JMAX_SWEEPS + 1 if not converged
  unsigned rot[JMAX_SWEEPS];       // counted rotations per sweep
};

// Bounded grid barrier (the launch is cooperative, so every block is resident): gives up
// after ~2 s (2^32 SM clocks) or once another block has given up; returns false then.
__device__ bool grid_barrier(JacobiSync* js, unsigned nblocks) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &js->gen;
    volatile int* verr = &js->err;
    const unsigned gen = *vgen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(&js->count, 1u) == nblocks - 1) {
      atomicExch(&js->count, 0u);
      __threadfence();
      atomicAdd(&js->gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == gen) {
        __nanosleep(32);
        if (*verr) {
          ok = 0;
          break;
        }
        if (clock64() - t0 > (4ll << 30)) {
          atomicExch(&js->err, 1);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    s_ok = ok && !*verr;
  }
  __syncthreads();
  return s_ok != 0;
}

__global__ void __launch_bounds__(JB) jacobi_kernel(double* __restrict__ A, int64_t rows, int ncols,
                                                    int p, double tol, double small2, double count2,
                                                    double* __restrict__ colsq,
                                                    JacobiSync* __restrict__ js, double* __restrict__ V,
                                                    int64_t vrows) {
  const unsigned nb = gridDim.x;
  const int npairs = p / 2;
  const int lane = threadIdx.x & 31;
  // pairs are dealt to blocks first (pair pr goes to block pr mod nb), so that a round's FP64
  // work spreads over every SM even when there are fewer pairs than warps
  const int gw0 = (int)(blockIdx.x + nb * (threadIdx.x >> 5));
  const int nwarps = (int)(nb * (JB / 32));
  for (int sweep = 0; sweep < JMAX_SWEEPS; ++sweep) {
    for (int r = 0; r < p - 1; ++r) {
      for (int pr = gw0; pr < npairs; pr += nwarps) {
        int a, b;
        if (pr == 0) {
          a = p - 1;
          b = r;
        } else {
          a = (r + pr) % (p - 1);
          b = (r - pr + (p - 1)) % (p - 1);
        }
        if (a > b) {
          const int t = a;
          a = b;
          b = t;
        }
        if (b >= ncols) continue;  // dummy player when ncols is odd
        const double al = __ldcg(colsq + a), be = __ldcg(colsq + b);
        if (al < small2 && be < small2) continue;
        double* ca = A + (int64_t)a * rows;
        double* cb = A + (int64_t)b * rows;
        // JU rows per lane per iteration, all loads issued before the arithmetic, so that the
        // L2 latency is paid once per JU rows
        double ga = 0.0;
        for (int64_t i0 = lane; i0 < rows; i0 += 32 * JU) {
          double x[JU], y[JU];
#pragma unroll
          for (int u = 0; u < JU; ++u) {
            const int64_t i = i0 + 32 * u;
            x[u] = i < rows ? __ldcg(ca + i) : 0.0;
            y[u] = i < rows ? __ldcg(cb + i) : 0.0;
          }
#pragma unroll
          for (int u = 0; u < JU; ++u) ga = fma(x[u], y[u], ga);
        }
        ga = warp_sum(ga);
        if (!(al > 0.0) || !(be > 0.0) || !(fabs(ga) > tol * sqrt(al) * sqrt(be))) continue;
        const double zeta = (be - al) / (2.0 * ga);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
        double na = 0.0, nbb = 0.0;
        for (int64_t i0 = lane; i0 < rows; i0 += 32 * JU) {
          double x[JU], y[JU];
#pragma unroll
          for (int u = 0; u < JU; ++u) {
            const int64_t i = i0 + 32 * u;
            x[u] = i < rows ? __ldcg(ca + i) : 0.0;
            y[u] = i < rows ? __ldcg(cb + i) : 0.0;
          }
#pragma unroll
          for (int u = 0; u < JU; ++u) {
            const int64_t i = i0 + 32 * u;
            const double xa = cs * x[u] - sn * y[u], yb = sn * x[u] + cs * y[u];
            if (i < rows) {
              ca[i] = xa;
              cb[i] = yb;
            }
            na = fma(xa, xa, na);
            nbb = fma(yb, yb, nbb);
          }
        }
        if (V) {
          double* va = V + (int64_t)a * vrows;
          double* vb = V + (int64_t)b * vrows;
          for (int64_t i0 = lane; i0 < vrows; i0 += 32 * JU) {
            double x[JU], y[JU];
#pragma unroll
            for (int u = 0; u < JU; ++u) {
              const int64_t i = i0 + 32 * u;
              x[u] = i < vrows ? __ldcg(va + i) : 0.0;
              y[u] = i < vrows ? __ldcg(vb + i) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < JU; ++u) {
              const int64_t i = i0 + 32 * u;
              if (i < vrows) {
                va[i] = cs * x[u] - sn * y[u];
                vb[i] = sn * x[u] + cs * y[u];
              }
            }
          }
        }
        na = warp_sum(na);
        nbb = warp_sum(nbb);
        if (lane == 0) {
          colsq[a] = na;
          colsq[b] = nbb;
          // the rotation counts toward convergence if it moved a column of squared norm
          // >= count2 by more than rounding: column a changes by ~|t| ||b||, column b by ~|t| ||a||
          const double move_a = al >= count2 ? fabs(t) * sqrt(be / al) : 0.0;
          const double move_b = be >= count2 ? fabs(t) * sqrt(al / be) : 0.0;
          if (fmax(move_a, move_b) > 4.0 * 2.220446049250313e-16) atomicAdd(&js->rot[sweep], 1u);
        }
      }
      if (!grid_barrier(js, nb)) return;
    }
    // after the sweep's last barrier every block reads the same final count
    if (*(volatile unsigned*)&js->rot[sweep] == 0) {
      if (blockIdx.x == 0 && threadIdx.x == 0) js->sweeps = sweep + 1;
      return;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) js->sweeps = JMAX_SWEEPS + 1;
}

__global__ void colsq_init_kernel(const double* __restrict__ A, int64_t rows, int ncols,
                                  double* __restrict__ colsq) {
  const int gw = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (gw >= ncols) return;
  const double* col = A + (int64_t)gw * rows;
  double acc = 0.0;
  for (int64_t i = lane; i < rows; i += 32) acc = fma(col[i], col[i], acc);
  acc = warp_sum(acc);
  if (lane == 0) colsq[gw] = acc;
}


// norms[c] = ||A[:, c]||_2, one warp per column
__global__ void colnorm_kernel(const double* __restrict__ A, int64_t rows, int ncols,
                               double* __restrict__ norms) {
  const int gw = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (gw >= ncols) return;
  const double* col = A + (int64_t)gw * rows;
  double acc = 0.0;
  for (int64_t i = lane; i < rows; i += 32) acc = fma(col[i], col[i], acc);
  acc = warp_sum(acc);
  if (lane == 0) norms[gw] = sqrt(acc);
}

// out[:, q] = in[:, perm[q]] * (scale ? 1/norms[perm[q]] : 1), q < r
__global__ void gather_cols_kernel(const double* __restrict__ in, int64_t rows,
                                   const int* __restrict__ perm, int r,
                                   const double* __restrict__ norms, double* __restrict__ out) {
  const int64_t total = rows * r;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % rows;
    const int q = (int)(e / rows);
    const int src = perm[q];
    double val = in[i + (int64_t)src * rows];
    if (norms) {
      const double nr = norms[src];
      val = nr > 0.0 ? val / nr : 0.0;
    }
    out[e] = val;
  }
}

// out[perm[i] + rows q] = in[i + rows q] (rows x ncols, column-major)
__global__ void scatter_rows_kernel(const double* __restrict__ in, int64_t rows, int ncols,
                                    const int* __restrict__ perm, double* __restrict__ out) {
  const int64_t total = rows * ncols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % rows, q = e / rows;
    out[perm[i] + q * rows] = in[e];
  }
}

__global__ void cast_f32_kernel(const double* __restrict__ in, int64_t n, float* __restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (float)in[e];
}

__global__ void widen_f32_kernel(const float* __restrict__ in, int64_t n, double* __restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (double)in[e];
}

// ---------------- FP64 SIMT GEMM (column-major) -------------------------------------
template <int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    dgemm_kernel(bool tA, bool tB, int64_t M, int64_t N, int64_t K, double alpha,
                 const double* __restrict__ A, int64_t lda, const double* __restrict__ B,
                 int64_t ldb, double beta, double* __restrict__ C, int64_t ldc) {
  constexpr int NT = (BM / TM) * (BN / TN);
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int tx = threadIdx.x % (BN / TN), ty = threadIdx.x / (BN / TN);
  const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
  double acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;
  for (int64_t k0 = 0; k0 < K; k0 += BK) {
    for (int e = threadIdx.x; e < BM * BK; e += NT) {
      int mm, kk;
      if (tA) { kk = e % BK; mm = e / BK; } else { mm = e % BM; kk = e / BM; }
      const int64_t gm = m0 + mm, gk = k0 + kk;
      double val = 0.0;
      if (gm < M && gk < K) val = tA ? A[gk + gm * lda] : A[gm + gk * lda];
      As[kk][mm] = val;
    }
    for (int e = threadIdx.x; e < BN * BK; e += NT) {
      int nn, kk;
      if (tB) { nn = e % BN; kk = e / BN; } else { kk = e % BK; nn = e / BK; }
      const int64_t gn = n0 + nn, gk = k0 + kk;
      double val = 0.0;
      if (gn < N && gk < K) val = tB ? B[gn + gk * ldb] : B[gk + gn * ldb];
      Bs[kk][nn] = val;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int64_t gm = m0 + ty * TM + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int64_t gn = n0 + tx * TN + j;
      if (gn >= N) continue;
      double* cp = C + gm + gn * ldc;
      *cp = alpha * acc[i][j] + (beta == 0.0 ? 0.0 : beta * *cp);
    }
  }
}

struct Buf {
  double* p = nullptr;
  ~Buf() {
    if (p) cudaFree(p);
  }
  pttk_status alloc(size_t elems) {
    if (p) cudaFree(p);
    p = nullptr;
    if (elems == 0) elems = 1;
    const cudaError_t e = cudaMalloc(&p, elems * sizeof(double));
    if (e != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      return set_error(PTTK_ENOMEM, "device allocation failed in TT-SVD");
    }
    return PTTK_OK;
  }
};

unsigned grid1d(int64_t work, int threads, int cap_per_sm = 8) {
  const int64_t b = (work + threads - 1) / threads;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)sm_count() * cap_per_sm));
}

// Pivoted Householder QR of A (M x N, M >= N, overwritten), stopped once ||R22||_F^2 <= stop2
// (at least one step is taken). On return perm[0..N) holds the column order, Rp the rows
// 0..k-1 of R by physical column (Rp must be N x N and is zeroed here), *k_out the number of
// rows kept and *tail2_out ||R22||_F^2 at the stop. Synchronises `s` every 16 steps to read the
// stop flag; steps enqueued after the stop return at once.
pttk_status householder_qrcp(double* A, int64_t M, int64_t N, double stop2, double* Rp, int* perm,
                             double* part, double* below, double* w_part, double* w, HHState* st,
                             int* k_out, double* tail2_out, cudaStream_t s) {
  const int64_t nchunks = (M + RC - 1) / RC;
  PTTK_PROF("householder", s);
  PTTK_CUDA(cudaMemsetAsync(Rp, 0, sizeof(double) * N * N, s));
  PTTK_CUDA(cudaMemsetAsync(st, 0, sizeof(HHState), s));
  iota_kernel<<<grid1d(N, 256), 256, 0, s>>>(perm, N); pttk::count_launch();
  hh_init_norms_kernel<<<dim3((unsigned)nchunks, (unsigned)((N + CG - 1) / CG)), 256, 0, s>>>(A, M, N, part); pttk::count_launch();
  HHState h{};
  for (int64_t j = 0; j < N; ++j) {
    hh_below_kernel<<<(unsigned)((N - j + 7) / 8), 256, 0, s>>>(part, N, j, nchunks, perm, st, below); pttk::count_launch();
    hh_pivot_kernel<<<1, 1024, 0, s>>>(A, M, N, j, below, perm, stop2, st, Rp); pttk::count_launch();
    const int64_t trailing = N - j - 1;
    if (trailing > 0) {
      const unsigned gx = (unsigned)(nchunks - j / RC);
      const unsigned gy = (unsigned)((trailing + CG - 1) / CG);
      hh_w_kernel<<<dim3(gx, gy), 256, 0, s>>>(A, M, N, j, perm, st, w_part); pttk::count_launch();
      hh_wsum_kernel<<<(unsigned)trailing, 256, 0, s>>>(w_part, N, j, nchunks, st, w); pttk::count_launch();
      hh_update_kernel<<<dim3(gx, gy), 256, 0, s>>>(A, M, N, j, perm, st, w, Rp, part); pttk::count_launch();
    }
    if ((j & 15) == 15 || j == N - 1) {
      PTTK_CUDA(cudaGetLastError());
      PTTK_CUDA(cudaMemcpyAsync(&h, st, sizeof(HHState), cudaMemcpyDeviceToHost, s));
      PTTK_CUDA(cudaStreamSynchronize(s));
      if (h.done) break;
    }
  }
  PTTK_CUDA(cudaGetLastError());
  *k_out = h.done ? h.k : (int)N;
  *tail2_out = h.done ? h.tail2 : 0.0;
  return PTTK_OK;
}

static pttk_status launch_jacobi(double* A, int64_t rows, int ncols, int p, double tol, double small2,
                                 double count2, double* colsq, JacobiSync* js, double* V, int64_t vrows,
                                 cudaStream_t s) {
  int per_sm = 0;
  PTTK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_kernel, JB, 0));
  if (per_sm < 1) return set_error(PTTK_ECUDA, "Jacobi kernel cannot be resident");
  // one block per SM (fewer when there are fewer pairs); each block takes up to 8 pairs of a
  // round at a time, pairs dealt round-robin over the blocks
  const int want = p / 2;
  const unsigned grid = (unsigned)std::max(1, std::min(want, sm_count()));
  void* args[] = {&A, &rows, &ncols, &p, &tol, &small2, &count2, &colsq, &js, &V, &vrows};
  PTTK_CUDA(cudaLaunchCooperativeKernel((const void*)jacobi_kernel, dim3(grid), dim3(JB), args, 0, s));
  pttk::count_launch();
  return PTTK_OK;
}

// One-sided Jacobi on the columns of A (rows x ncols), all sweeps in one cooperative launch;
// synchronises `s` once to read the outcome. With V (vrows x ncols), every rotation is also
// applied to V's columns.
pttk_status jacobi(double* A, int64_t rows, int ncols, cudaStream_t s, double small = 0.0, double* V = nullptr,
                   int64_t vrows = 0) {
  if (ncols < 2) return PTTK_OK;
  Buf colsq, state;
  PTTK_TRY(colsq.alloc(ncols));
  PTTK_TRY(state.alloc((sizeof(JacobiSync) + sizeof(double) - 1) / sizeof(double)));
  static_assert(alignof(JacobiSync) <= 256, "cudaMalloc alignment");
  JacobiSync* js = reinterpret_cast<JacobiSync*>(state.p);
  PTTK_CUDA(cudaMemsetAsync(js, 0, sizeof(JacobiSync), s));
  colsq_init_kernel<<<(unsigned)(((int64_t)ncols * 32 + 255) / 256), 256, 0, s>>>(A, rows, ncols, colsq.p); pttk::count_launch();
  const double small2 = small * small;
  const double count2 = 100.0 * small2;
  const int p = ncols + (ncols & 1);
  // A pair counts as orthogonal once |a.b| <= sqrt(rows) eps ||a|| ||b||: the typical rounding
  // level of a computed dot product. The singular subspaces are then accurate to that level,
  // which the 1e-12 parity of K~ needs (a looser rows * eps stops ~20x earlier in accuracy).
  const double tol = sqrt((double)std::max<int64_t>(rows, 16)) * 2.220446049250313e-16;
  {
    PTTK_PROF("jacobi", s);
    PTTK_TRY(launch_jacobi(A, rows, ncols, p, tol, small2, count2, colsq.p, js, V, vrows, s));
  }
  JacobiSync h{};
  PTTK_CUDA(cudaMemcpyAsync(&h, js, sizeof(JacobiSync), cudaMemcpyDeviceToHost, s));
  PTTK_CUDA(cudaStreamSynchronize(s));
  if (kDebugLog)
    for (int sw = 0; sw < std::min(h.sweeps, JMAX_SWEEPS); ++sw)
      fprintf(stderr, "pttk: jacobi %lld x %d sweep %d rotations %u\n", (long long)rows, ncols, sw, h.rot[sw]);
  if (h.err) return set_error(PTTK_ETIMEOUT, "one-sided Jacobi: a grid barrier timed out");
  if (h.sweeps > JMAX_SWEEPS) return set_error(PTTK_ECUDA, "one-sided Jacobi SVD did not converge in 60 sweeps");
  return PTTK_OK;
}

// Sorted order of sigma (descending) and the truncation rank for threshold delta.
// `extra2` is a squared norm already discarded (the R22 of a truncated QR), counted in every tail.
int truncation(const std::vector<double>& sigma, double delta, std::vector<int>& perm, double extra2 = 0.0) {
  perm.resize(sigma.size());
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int x, int y) { return sigma[x] > sigma[y]; });
  const int m = (int)sigma.size();
  std::vector<double> tail(m + 1, 0.0);  // tail[r] = extra2 + sum_{i >= r} sigma_(i)^2
  tail[m] = extra2;
  for (int i = m - 1; i >= 0; --i) tail[i] = tail[i + 1] + sigma[perm[i]] * sigma[perm[i]];
  for (int r = 1; r <= m; ++r)
    if (sqrt(tail[r]) <= delta) return r;
  return m;
}

}  // namespace

void dgemm(bool tA, bool tB, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
           int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
           cudaStream_t s) {
  if (M <= 0 || N <= 0) return;
  PTTK_PROF("dgemm", s);
  if (M <= 16) {
    dim3 grid((unsigned)((N + 127) / 128), (unsigned)((M + 15) / 16));
    dgemm_kernel<16, 128, 16, 2, 4><<<grid, 256, 0, s>>>(tA, tB, M, N, K, alpha, A, lda, B, ldb,
                                                         beta, C, ldc); pttk::count_launch();
  } else {
    dim3 grid((unsigned)((N + 63) / 64), (unsigned)((M + 63) / 64));
    dgemm_kernel<64, 64, 16, 4, 4><<<grid, 256, 0, s>>>(tA, tB, M, N, K, alpha, A, lda, B, ldb,
                                                        beta, C, ldc); pttk::count_launch();
  }
}

// Wall-clock stage timing of the TT-SVD, printed to stderr in a PTTK_DEBUG build (it
// synchronises the stream at every mark, so release builds compile it out).
struct StageClock {
  bool on;
  cudaStream_t s;
  std::chrono::steady_clock::time_point t0;
  explicit StageClock(cudaStream_t st) : on(kDebugLog), s(st) { reset(); }
  void reset() {
    if (!on) return;
    cudaStreamSynchronize(s);
    t0 = std::chrono::steady_clock::now();
  }
  void mark(int k, const char* what) {
    if (!on) return;
    cudaStreamSynchronize(s);
    const auto t1 = std::chrono::steady_clock::now();
    fprintf(stderr, "pttk: tt-svd step %d %-10s %9.3f ms\n", k + 1, what,
            std::chrono::duration<double, std::milli>(t1 - t0).count());
    t0 = t1;
  }
};

// Working buffers of svd_basis, reused (reallocated) from call to call.
struct StepWork {
  Buf qrin, A, U, Y, Yt, norms, part, wpart, wv, below, R, A0, Rd, V, PV;
  int* d_perm = nullptr;
  int* d_perm2 = nullptr;
  HHState* d_hs = nullptr;
  ~StepWork() {
    if (d_perm) cudaFree(d_perm);
    if (d_perm2) cudaFree(d_perm2);
    if (d_hs) cudaFree(d_hs);
  }
};

// Orthonormal basis (m x r, unit columns in decreasing singular value, column-major, into
// `core`) of the top-r left singular subspace of X (m x c, column-major, not modified), r the
// smallest rank >= 1 whose discarded tail sqrt(sum_{i>r} sigma_i^2) is <= delta; delta = 0
// keeps every direction X has (an orthonormal basis of its range). stop_frac: the pivoted QR
// stops once the discarded block has ||R22||_F <= stop_frac delta (see below).
static pttk_status svd_basis(const double* X, int64_t m, int64_t c, double delta, StepWork& wk, Buf& core,
                             int* r_out, StageClock& clk, int k, cudaStream_t s, double stop_frac = 0.03) {
  if (!wk.d_hs) PTTK_CUDA(cudaMalloc(&wk.d_hs, sizeof(HHState)));
  const bool wide = c >= m;
  // QR input: wide -> W = X^T (c x m), tall -> a copy of X (m x c). The pivoted QR makes
  // the triangular factor graded, so one-sided Jacobi on its transpose converges in a few
  // sweeps, and stops once the remaining block is negligible next to delta.
  const int64_t q = wide ? m : c;        // columns of the QR input
  const int64_t Mqr = wide ? c : m;      // rows of the QR input
  if (clk.on) fprintf(stderr, "pttk: tt-svd step %d m %lld c %lld %s\n", k + 1, (long long)m, (long long)c, wide ? "wide" : "tall");
  clk.reset();
  PTTK_TRY(wk.norms.alloc(std::max<int64_t>(q, 1)));
  if (wk.d_perm) cudaFree(wk.d_perm);
  wk.d_perm = nullptr;
  PTTK_CUDA(cudaMalloc(&wk.d_perm, sizeof(int) * q));
  PTTK_TRY(wk.qrin.alloc(Mqr * q));
  if (wide) {
    dim3 tg((unsigned)((c + 31) / 32), (unsigned)((m + 31) / 32));
    transpose_kernel<<<tg, dim3(32, 8), 0, s>>>(X, m, c, nullptr, wk.qrin.p); pttk::count_launch();
  } else {
    PTTK_CUDA(cudaMemcpyAsync(wk.qrin.p, X, sizeof(double) * m * c, cudaMemcpyDeviceToDevice, s));
  }
  const int64_t nchunks = (Mqr + RC - 1) / RC;
  PTTK_TRY(wk.part.alloc(nchunks * q));
  PTTK_TRY(wk.wpart.alloc(nchunks * q));
  PTTK_TRY(wk.wv.alloc(q));
  PTTK_TRY(wk.below.alloc(q));
  PTTK_TRY(wk.R.alloc(q * q));
  clk.mark(k, "layout");
  // rows of R kept: the QR stops once the discarded block has ||R22||_F <= stop_frac delta
  // (0.03 for the TT-SVD). The tails below count ||R22||^2, so the error bound of the
  // truncation holds as it is; only a tail within stop_frac^2 delta^2 of the threshold could
  // give a rank one higher than the exact singular values would. The discarded block also
  // moves the kept subspace by about stop_frac delta against the exact SVD's
  int kq = 0;
  double tail2 = 0.0;
  const double stop = stop_frac * delta;
  PTTK_TRY(householder_qrcp(wk.qrin.p, Mqr, q, stop * stop, wk.R.p, wk.d_perm, wk.part.p, wk.below.p,
                            wk.wpart.p, wk.wv.p, wk.d_hs, &kq, &tail2, s));
  clk.mark(k, "qr");
  if (clk.on) fprintf(stderr, "pttk: tt-svd step %d kept %d of %lld rows of R, ||R22|| %.3e\n", k + 1, kq, (long long)q, sqrt(tail2));
  // A = R1^T (q x kq), R1 = the kept rows of R in pivoted column order
  PTTK_TRY(wk.A.alloc(q * kq));
  gather_rt_kernel<<<grid1d(q * kq, 256), 256, 0, s>>>(wk.R.p, q, kq, wk.d_perm, wk.A.p); pttk::count_launch();
  // one-sided Jacobi on R1^T: R1^T V = U' Sigma, so R1 = V Sigma U'^T and the right singular
  // vectors of R1 (= of the pivoted QR input, up to the discarded R22) are the normalised
  // columns of the rotated R1^T; columns below (stop_frac / 30) delta / sqrt(kq) together carry
  // < (stop_frac / 30)^2 delta^2, and pairs of them are skipped
  const double jsmall = (stop_frac / 30.0) * delta / sqrt((double)kq);
  if (2 * q >= 5 * (int64_t)kq && kq >= 2) {
    // R1^T has at least 2.5 times as many rows as columns: a second pivoted QR,
    // R1^T P2 = Q2 R2, and the Jacobi on R2 (kq x kq), whose columns have the Gram matrix of
    // R1^T P2's and so take the same rotations, accumulated in V; the rotated R1^T is then
    // R1^T (P2 V), one DGEMM. Each rotation touches 2 kq rows (R2 and V) instead of q. The
    // second QR and the fixed cost of a Jacobi round (L2 round trips, grid barrier) eat the
    // gain below that ratio (c3: 2124 x 751 254 -> 201 ms, 1728 x 256 46 -> 37 ms, but
    // 528 x 236 21 -> 27 ms).
    PTTK_TRY(wk.A0.alloc(q * kq));
    PTTK_CUDA(cudaMemcpyAsync(wk.A0.p, wk.A.p, sizeof(double) * q * kq, cudaMemcpyDeviceToDevice, s));
    if (wk.d_perm2) cudaFree(wk.d_perm2);
    wk.d_perm2 = nullptr;
    PTTK_CUDA(cudaMalloc(&wk.d_perm2, sizeof(int) * kq));
    int k2 = 0;
    double t2 = 0.0;
    // the first QR's work buffers are large enough (its rows >= q, its columns q >= kq), and
    // its R has been consumed into wk.A; stop2 < 0: every column is factored
    PTTK_TRY(householder_qrcp(wk.A.p, q, kq, -1.0, wk.R.p, wk.d_perm2, wk.part.p, wk.below.p, wk.wpart.p, wk.wv.p,
                              wk.d_hs, &k2, &t2, s));
    PTTK_TRY(wk.Rd.alloc((int64_t)k2 * kq));
    gather_r_kernel<<<grid1d((int64_t)k2 * kq, 256), 256, 0, s>>>(wk.R.p, kq, k2, wk.d_perm2, wk.Rd.p); pttk::count_launch();
    PTTK_TRY(wk.V.alloc((int64_t)kq * kq));
    PTTK_TRY(wk.PV.alloc((int64_t)kq * kq));
    eye_kernel<<<grid1d((int64_t)kq * kq, 256), 256, 0, s>>>(wk.V.p, kq); pttk::count_launch();
    PTTK_TRY(jacobi(wk.Rd.p, k2, kq, s, jsmall, wk.V.p, kq));
    // P2 V: row perm2[l] of the result is row l of V
    scatter_rows_kernel<<<grid1d((int64_t)kq * kq, 256), 256, 0, s>>>(wk.V.p, kq, kq, wk.d_perm2, wk.PV.p); pttk::count_launch();
    dgemm(false, false, q, kq, kq, 1.0, wk.A0.p, q, wk.PV.p, kq, 0.0, wk.A.p, q, s);
    PTTK_CUDA(cudaGetLastError());
  } else {
    PTTK_TRY(jacobi(wk.A.p, q, kq, s, jsmall));
  }
  clk.mark(k, "jacobi");
  colnorm_kernel<<<(unsigned)(((int64_t)kq * 32 + 255) / 256), 256, 0, s>>>(wk.A.p, q, kq, wk.norms.p); pttk::count_launch();
  std::vector<double> sigma(kq);
  PTTK_CUDA(cudaMemcpyAsync(sigma.data(), wk.norms.p, sizeof(double) * kq, cudaMemcpyDeviceToHost, s));
  PTTK_CUDA(cudaStreamSynchronize(s));
  std::vector<int> perm;
  const int r = truncation(sigma, delta, perm, tail2);
  int* d_top = nullptr;
  PTTK_CUDA(cudaMalloc(&d_top, sizeof(int) * std::max<int64_t>(kq, 1)));
  struct TopGuard { int* p; ~TopGuard() { if (p) cudaFree(p); } } top_guard{d_top};
  PTTK_CUDA(cudaMemcpyAsync(d_top, perm.data(), sizeof(int) * kq, cudaMemcpyHostToDevice, s));
  // top-r right singular vectors (unit columns), in the pivoted order
  PTTK_TRY(wk.U.alloc(q * r));
  PTTK_TRY(wk.Y.alloc(q * r));
  gather_cols_kernel<<<grid1d(q * r, 256), 256, 0, s>>>(wk.A.p, q, d_top, r, wk.norms.p, wk.Y.p); pttk::count_launch();
  // back to the original order: row perm[l] of the result is row l of Y
  scatter_rows_kernel<<<grid1d(q * r, 256), 256, 0, s>>>(wk.Y.p, q, r, wk.d_perm, wk.U.p); pttk::count_launch();
  double* basis = wk.U.p;  // m x r (wide): left singular vectors of X
  if (!wide) {
    // tall: U holds the top right singular vectors of X (c x r); Y = X U spans the top-r
    // left singular subspace
    PTTK_TRY(wk.Yt.alloc(m * r));
    dgemm(false, false, m, r, c, 1.0, X, m, wk.U.p, c, 0.0, wk.Yt.p, m, s);
    basis = wk.Yt.p;
  }
  // make the m x r basis orthonormal to working precision: its columns are orthogonal up
  // to ~eps ||X|| / sigma_i, so one-sided Jacobi needs one or two sweeps
  clk.mark(k, "basis");
  PTTK_TRY(jacobi(basis, m, r, s));
  clk.mark(k, "reorth");
  Buf bn;
  PTTK_TRY(bn.alloc(r));
  colnorm_kernel<<<(unsigned)(((int64_t)r * 32 + 255) / 256), 256, 0, s>>>(basis, m, r, bn.p); pttk::count_launch();
  std::vector<double> bnh(r);
  PTTK_CUDA(cudaMemcpyAsync(bnh.data(), bn.p, sizeof(double) * r, cudaMemcpyDeviceToHost, s));
  PTTK_CUDA(cudaStreamSynchronize(s));
  std::vector<int> bperm;
  truncation(bnh, 0.0, bperm);
  PTTK_CUDA(cudaMemcpyAsync(d_top, bperm.data(), sizeof(int) * r, cudaMemcpyHostToDevice, s));
  PTTK_TRY(core.alloc(m * r));
  gather_cols_kernel<<<grid1d(m * r, 256), 256, 0, s>>>(basis, m, d_top, r, bn.p, core.p); pttk::count_launch();
  PTTK_CUDA(cudaStreamSynchronize(s));
  *r_out = r;
  return PTTK_OK;
}

// Packs device cores (core k: ranks[k] x n x ranks[k+1], column-major) into the handle.
static pttk_status pack_cores(pttk_tt* tt, std::vector<Buf>& cores, cudaStream_t s) {
  size_t off = 0;
  for (int k = 0; k < tt->D; ++k) {
    tt->core_off[k] = off;
    off += tt->core_elems(k);
  }
  tt->core_total = off;
  PTTK_CUDA(cudaMalloc(&tt->cores64, sizeof(double) * off));
  PTTK_CUDA(cudaMalloc(&tt->cores32, sizeof(float) * off));
  for (int k = 0; k < tt->D; ++k)
    PTTK_CUDA(cudaMemcpyAsync(tt->cores64 + tt->core_off[k], cores[k].p,
                              sizeof(double) * tt->core_elems(k), cudaMemcpyDeviceToDevice, s));
  cast_f32_kernel<<<grid1d((int64_t)off, 256), 256, 0, s>>>(tt->cores64, (int64_t)off, tt->cores32); pttk::count_launch();
  PTTK_CUDA(cudaGetLastError());
  PTTK_CUDA(cudaStreamSynchronize(s));
  return PTTK_OK;
}

// squared Frobenius norm of x (n doubles), synchronous
static pttk_status sumsq_host(const double* x, int64_t n, double* out, cudaStream_t s) {
  Buf part, scal;
  const unsigned nb = grid1d(n, 256, 4);
  PTTK_TRY(part.alloc(nb));
  PTTK_TRY(scal.alloc(1));
  sumsq_kernel<<<nb, 256, 0, s>>>(x, n, part.p); pttk::count_launch();
  sum_kernel<<<1, 256, 0, s>>>(part.p, (int)nb, scal.p); pttk::count_launch();
  PTTK_CUDA(cudaGetLastError());
  PTTK_CUDA(cudaMemcpyAsync(out, scal.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  PTTK_CUDA(cudaStreamSynchronize(s));
  return PTTK_OK;
}

pttk_status tt_svd_run(pttk_tt* tt, double* X, double tol, cudaStream_t s) {
  const int D = tt->D, n = tt->n;
  StageClock clk(s);
  int64_t total = 1;
  for (int k = 0; k < D; ++k) total *= n;

  // ||C||_F
  double sumsq = 0.0;
  PTTK_TRY(sumsq_host(X, total, &sumsq, s));
  const double delta = tol / sqrt((double)(D - 1)) * sqrt(sumsq);

  Buf Xn;
  PTTK_TRY(Xn.alloc(total));
  StepWork wk;
  std::vector<Buf> cores(D);
  tt->ranks[0] = 1;
  int64_t r_prev = 1;
  double* cur = X;
  double* nxt = Xn.p;
  int64_t cur_elems = total;
  for (int k = 0; k < D - 1; ++k) {
    PTTK_CUDA(cudaStreamSynchronize(s));  // buffers are reallocated per step
    const int64_t m = r_prev * n;
    const int64_t c = cur_elems / m;
    int r = 0;
    PTTK_TRY(svd_basis(cur, m, c, delta, wk, cores[k], &r, clk, k, s));
    // X <- G_k^T X  (r x c)
    dgemm(true, false, r, c, m, 1.0, cores[k].p, m, cur, m, 0.0, nxt, r, s);
    PTTK_CUDA(cudaGetLastError());
    clk.mark(k, "project");
    if (clk.on) fprintf(stderr, "pttk: tt-svd step %d rank %d\n", k + 1, r);
    tt->ranks[k + 1] = r;
    std::swap(cur, nxt);
    cur_elems = (int64_t)r * c;
    r_prev = r;
  }
  tt->ranks[D] = 1;
  // last core: the remainder (r_{D-1} x n)
  PTTK_TRY(cores[D - 1].alloc(r_prev * n));
  PTTK_CUDA(cudaMemcpyAsync(cores[D - 1].p, cur, sizeof(double) * r_prev * n,
                            cudaMemcpyDeviceToDevice, s));
  return pack_cores(tt, cores, s);
}

// TT-Round (Algorithm 1): right-to-left orthogonalisation, then a left-to-right sweep of
// truncated SVDs with delta = tol / sqrt(D-1) ||X||_F. Each factorisation is svd_basis: with
// delta = 0 for the orthogonalisation (an orthonormal basis of the whole range, in place of the
// thin QR; any orthonormal factor serves), with delta for the truncation. Works on device cores
// G[k] (r[k] x nm[k] x r[k+1], column-major) of any mode sizes nm[k]; on return G and r hold the
// rounded TT.
// TT-Round's QR stops at 1e-4 delta (the TT-SVD's at 0.03 delta): its unfoldings are small
// (r_{i-1} n x r_i), so the later stop costs little, and the kept subspaces then agree with
// an exact SVD's to about 1e-4 delta.
constexpr double kRoundStopFrac = 1e-4;

pttk_status tt_round_cores(std::vector<Buf>& G, std::vector<int64_t>& r, const std::vector<int64_t>& nm, double tol,
                           cudaStream_t s) {
  const int D = (int)G.size();
  StageClock clk(s);
  std::vector<Buf> nb(D);
  StepWork wk;
  Buf A, W, T;
  // right to left: (G_i^{1})^T = U W, G_i <- U^T, G_{i-1} <- G_{i-1} x_3 W^T
  for (int i = D - 1; i >= 1; --i) {
    const int64_t m = nm[i] * r[i + 1], c = r[i];
    PTTK_TRY(A.alloc(m * c));
    dim3 tg((unsigned)((m + 31) / 32), (unsigned)((c + 31) / 32));
    transpose_kernel<<<tg, dim3(32, 8), 0, s>>>(G[i].p, c, m, nullptr, A.p); pttk::count_launch();
    int k = 0;
    PTTK_TRY(svd_basis(A.p, m, c, 0.0, wk, nb[i], &k, clk, i, s));
    PTTK_TRY(W.alloc((int64_t)k * c));
    dgemm(true, false, k, c, m, 1.0, nb[i].p, m, A.p, m, 0.0, W.p, k, s);   // W = U^T A (k x c)
    PTTK_TRY(G[i].alloc((int64_t)k * m));
    dim3 tg2((unsigned)((k + 31) / 32), (unsigned)((m + 31) / 32));
    transpose_kernel<<<tg2, dim3(32, 8), 0, s>>>(nb[i].p, m, k, nullptr, G[i].p); pttk::count_launch();
    const int64_t mp = r[i - 1] * nm[i - 1];                               // G_{i-1}^{2}: mp x c
    PTTK_TRY(T.alloc(mp * k));
    dgemm(false, true, mp, k, c, 1.0, G[i - 1].p, mp, W.p, k, 0.0, T.p, mp, s);
    std::swap(G[i - 1].p, T.p);
    r[i] = k;
  }
  double sumsq = 0.0;
  PTTK_TRY(sumsq_host(G[0].p, r[0] * nm[0] * r[1], &sumsq, s));
  const double delta = D > 1 ? tol / sqrt((double)(D - 1)) * sqrt(sumsq) : 0.0;
  // left to right: G_i^{2} = U W (truncated), G_i <- U, G_{i+1} <- W x_1 G_{i+1}
  for (int i = 0; i < D - 1; ++i) {
    const int64_t m = r[i] * nm[i], c = r[i + 1];
    int k = 0;
    PTTK_TRY(svd_basis(G[i].p, m, c, delta, wk, nb[i], &k, clk, i, s, kRoundStopFrac));
    PTTK_TRY(W.alloc((int64_t)k * c));
    dgemm(true, false, k, c, m, 1.0, nb[i].p, m, G[i].p, m, 0.0, W.p, k, s);
    std::swap(G[i].p, nb[i].p);
    const int64_t cn = nm[i + 1] * r[i + 2];                               // G_{i+1}^{1}: c x cn
    PTTK_TRY(T.alloc((int64_t)k * cn));
    dgemm(false, false, k, cn, c, 1.0, W.p, k, G[i + 1].p, c, 0.0, T.p, k, s);
    std::swap(G[i + 1].p, T.p);
    r[i + 1] = k;
  }
  PTTK_CUDA(cudaStreamSynchronize(s));
  return PTTK_OK;
}

pttk_status tt_round_run(const pttk_tt* in, double tol, pttk_tt* out, cudaStream_t s) {
  const int D = in->D;
  std::vector<Buf> G(D);
  std::vector<int64_t> r(D + 1), nm(D, in->n);
  for (int k = 0; k <= D; ++k) r[k] = in->ranks[k];
  for (int k = 0; k < D; ++k) {
    PTTK_TRY(G[k].alloc(in->core_elems(k)));
    PTTK_CUDA(cudaMemcpyAsync(G[k].p, in->cores64 + in->core_off[k], sizeof(double) * in->core_elems(k),
                              cudaMemcpyDeviceToDevice, s));
  }
  PTTK_TRY(tt_round_cores(G, r, nm, tol, s));
  for (int k = 0; k <= D; ++k) out->ranks[k] = (int)r[k];
  return pack_cores(out, G, s);
}

// Phase 4 of Algorithm 2: TT-Round of [T^(1)(S), G_{d+1}, .., G_{d+d_theta}, T^(3)(T^T)]
// (Eq. twist). Scol: N_s x r_s column-major (the first core 1 x N_s x r_s); theta cores
// ranks[j] x n x ranks[j+1], j < d_theta (ranks[0] = r_s, ranks[d_theta] = r_t); Tt: r_t x N_t
// column-major (the last core r_t x N_t x 1, i.e. T row-major). Inputs are not modified. On
// return out[0] (N_s x r_s' column-major), out[1 .. d_theta] (the rounded theta cores) and
// out[d_theta + 1] (r_t' x N_t column-major) are cudaMalloc'd arrays the caller frees, and
// new_ranks[0 .. d_theta] their ranks. Synchronises `s`.
pttk_status phase4_round(const double* Scol, int64_t Ns, const double* const* theta_cores, const int* ranks, int n,
                         int dtheta, const double* Tt, int64_t Nt, double tol, double** out, int* new_ranks,
                         cudaStream_t s) {
  const int D = dtheta + 2;
  std::vector<Buf> G(D);
  std::vector<int64_t> r(D + 1), nm(D, n);
  r[0] = 1;
  for (int j = 0; j <= dtheta; ++j) r[j + 1] = ranks[j];
  r[D] = 1;
  nm[0] = Ns;
  nm[D - 1] = Nt;
  for (int k = 0; k < D; ++k) {
    const int64_t e = r[k] * nm[k] * r[k + 1];
    PTTK_TRY(G[k].alloc(e));
    const double* src = k == 0 ? Scol : k == D - 1 ? Tt : theta_cores[k - 1];
    PTTK_CUDA(cudaMemcpyAsync(G[k].p, src, sizeof(double) * e, cudaMemcpyDeviceToDevice, s));
  }
  PTTK_TRY(tt_round_cores(G, r, nm, tol, s));
  for (int k = 0; k < D; ++k) {
    out[k] = G[k].p;
    G[k].p = nullptr;
  }
  for (int j = 0; j <= dtheta; ++j) new_ranks[j] = (int)r[j + 1];
  return PTTK_OK;
}

// Orthonormal basis of the range of X (m x c, column-major, not modified): svd_basis with
// delta = 0. *basis is allocated here (cudaMalloc, m x r column-major, r <= min(m, c)); the
// caller frees it with cudaFree. Synchronises `s`.
pttk_status range_basis(const double* X, int64_t m, int64_t c, double** basis, int* r, cudaStream_t s) {
  StageClock clk(s);
  StepWork wk;
  Buf core;
  PTTK_TRY(svd_basis(X, m, c, 0.0, wk, core, r, clk, 0, s));
  *basis = core.p;
  core.p = nullptr;
  return PTTK_OK;
}

// One-sided Jacobi on the columns of A (rows x ncols, column-major), in place: on return the
// columns are orthogonal, A V = U Sigma. Synchronises `s`.
pttk_status jacobi_columns(double* A, int64_t rows, int ncols, cudaStream_t s) {
  return jacobi(A, rows, ncols, s, 0.0);
}

// FP32 tensor -> FP64 work buffer
pttk_status widen_to_f64(const float* in, int64_t n, double* out, cudaStream_t s) {
  widen_f32_kernel<<<grid1d(n, 256), 256, 0, s>>>(in, n, out); pttk::count_launch();
  PTTK_CUDA(cudaGetLastError());
  return PTTK_OK;
}

}  // namespace pttk

// Symmetric eigendecomposition of a batch of small dense matrices in FP64, for the online
// stage of PTTK-Global (Algorithm 4: the eigenpairs of R H^ R^T, one k x k matrix per theta).
// The paper leaves this step to a library; it is built here from the classical steps:
//   1. Householder reduction to tridiagonal form T = H^T A H, H = H_0 .. H_{k-3}, with the
//      reflector of LAPACK's dlarfg (beta = -sign(alpha) ||x||, tau = (beta - alpha) / beta,
//      v = [1; x_{1:} / (alpha - beta)]) and the two-sided update of dsytd2
//      (p = tau A22 v, w = p - (tau/2)(p^T v) v, A22 <- A22 - v w^T - w v^T);
//   2. every eigenvalue of T by bisection on Sturm counts (the number of negative pivots of
//      T - x I), one thread per eigenvalue;
//   3. the eigenvectors of T for the selected eigenvalues by inverse iteration (Gaussian
//      elimination with partial pivoting on T - lambda I), re-orthogonalised by modified
//      Gram-Schmidt against the earlier vectors of their cluster (eigenvalues closer than
//      1e-3 of the weight the caller gives them, see sym_eig_vectors);
//   4. the eigenvectors of A = H times those of T (the reflectors applied in reverse order).
// The matrices of a batch are independent; every launch covers the whole batch (grid z or a
// block per matrix), so a batch costs the launches of one matrix. No kernel waits on another
// CTA.
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "pttk_internal.cuh"

namespace pttk {
namespace {

constexpr int EB = 256;        // threads per block
constexpr int CHUNK = 64;      // columns per partial sum of the symmetric product
constexpr int SB = 64;         // rows per block of the symmetric product

// 1/x by Newton-Raphson from the hardware approximation (rcp.approx.ftz.f64, good to about
// 20 bits): each step r <- r + r (1 - x r) squares the relative error, so two steps reach
// the rounding level (within an ulp or two of the IEEE quotient). Arguments below 1e-290 in magnitude (where the approximation
// flushes) take the IEEE division.
__device__ __forceinline__ double rcp_nr(double x) {
  if (fabs(x) < 1e-290) return 1.0 / x;
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double h = fma(-x, r, 1.0);
  r = fma(r, h, r);
  h = fma(-x, r, 1.0);
  return fma(r, h, r);
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (int)(blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) sh[0] = t;
  }
  __syncthreads();
  return sh[0];
}

// Step j of the tridiagonalisation, first half, for matrix blockIdx.z. Every block forms the
// reflector of x = A[j+1:k, j] itself (beta = -sign(alpha) ||x||, tau = (beta - alpha) / beta,
// v = [1; x_{1:} / (alpha - beta)]) and then the partial products
//   part[(z * nch + c) * k + i] = sum over the columns l of chunk c (l > j) of A[i, l] v_l
// for its rows i > j. Block (0, 0) also writes v to vbuf, tau[j], the diagonal d[j] = A[j, j]
// and the off-diagonal e[j] = beta. Column j keeps x until the second half, which runs after
// every block of this one has read it.
__global__ void __launch_bounds__(SB * 4) reflect_symv_kernel(const double* __restrict__ A, int k, int j, int nch,
                                                              double* __restrict__ part, double* __restrict__ vbuf,
                                                              double* __restrict__ tau, double* __restrict__ d,
                                                              double* __restrict__ e, unsigned* __restrict__ done,
                                                              double* __restrict__ w) {
  __shared__ double sh[32];
  __shared__ double vs[CHUNK];
  __shared__ double red[4][SB];
  const int z = blockIdx.z;
  const double* a = A + (size_t)z * k * k;
  const double* col = a + (size_t)j * k;
  double s = 0.0;
  for (int i = j + 2 + threadIdx.x; i < k; i += blockDim.x) s += col[i] * col[i];
  const double xn2 = block_sum(s, sh);
  const double alpha = col[j + 1];
  double t = 0.0, beta = alpha, scale = 0.0;
  if (xn2 > 0.0) {
    beta = -copysign(sqrt(alpha * alpha + xn2), alpha);
    t = (beta - alpha) / beta;
    scale = 1.0 / (alpha - beta);
  }
  const int l0 = j + 1 + blockIdx.y * CHUNK, l1 = min(k, l0 + CHUNK);
  for (int l = l0 + threadIdx.x; l < l0 + CHUNK; l += blockDim.x)
    vs[l - l0] = l >= l1 ? 0.0 : (l == j + 1 ? 1.0 : (xn2 > 0.0 ? col[l] * scale : 0.0));
  __syncthreads();
  // four column groups of CHUNK / 4: the 16 loads of a thread are independent, so they are all
  // in flight together; the groups' sums meet in shared memory
  const int rr = threadIdx.x % SB, grp = threadIdx.x / SB;
  const int i = j + 1 + blockIdx.x * SB + rr;
  const int ir = i < k ? i : k - 1;
  double acc = 0.0;
#pragma unroll
  for (int q = 0; q < CHUNK / 4; ++q) {
    const int l = l0 + grp * (CHUNK / 4) + q;
    const double x = l < l1 ? a[(size_t)l * k + ir] : 0.0;
    acc = fma(x, vs[l - l0], acc);
  }
  red[grp][rr] = acc;
  __syncthreads();
  if (grp == 0 && i < k)
    part[((size_t)z * nch + blockIdx.y) * k + i] = (red[0][rr] + red[1][rr]) + (red[2][rr] + red[3][rr]);
  if (blockIdx.x == 0 && blockIdx.y == 0) {
    for (int l = j + 1 + threadIdx.x; l < k; l += blockDim.x)
      vbuf[(size_t)z * k + l] = l == j + 1 ? 1.0 : (xn2 > 0.0 ? col[l] * scale : 0.0);
    if (threadIdx.x == 0) {
      tau[(size_t)z * k + j] = t;
      d[(size_t)z * k + j] = col[j];
      e[(size_t)z * k + j] = beta;
    }
  }
  // The block that finishes last (a counter per matrix and step, no waiting) forms
  // w = p - (tau/2)(p^T v) v with p = tau sum_c part once, for the second half to read.
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&done[(size_t)z * k + j], 1u) == gridDim.x * gridDim.y - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int m = k - j - 1;
  double sp = 0.0;
  for (int q = threadIdx.x; q < m; q += blockDim.x) {
    double p = 0.0;
    for (int c = 0; c < nch; ++c) p += __ldcg(part + ((size_t)z * nch + c) * k + j + 1 + q);
    p *= t;
    const double v = q == 0 ? 1.0 : (xn2 > 0.0 ? col[j + 1 + q] * scale : 0.0);
    w[(size_t)z * k + j + 1 + q] = p;
    sp += p * v;
  }
  const double pv = block_sum(sp, sh);
  for (int q = threadIdx.x; q < m; q += blockDim.x) {
    const double v = q == 0 ? 1.0 : (xn2 > 0.0 ? col[j + 1 + q] * scale : 0.0);
    w[(size_t)z * k + j + 1 + q] -= 0.5 * t * pv * v;
  }
}

// Step j, second half (the two-sided update of dsytd2): every block loads w (formed by the
// first half's last block) and v for the rows i > j into shared memory, applies
// A22 <- A22 - v w^T - w v^T to its columns of A22 = A[j+1:, j+1:] (both triangles), and block
// 0 stores v over x in column j, where the back-transformation reads it. Dynamic shared
// memory: 2 (k - 1) doubles.
__global__ void __launch_bounds__(EB) w_rank2_kernel(double* __restrict__ A, int k, int j,
                                                     const double* __restrict__ wbuf,
                                                     const double* __restrict__ vbuf) {
  extern __shared__ double wv_smem[];
  const int z = blockIdx.z, m = k - j - 1;
  double* ws = wv_smem;
  double* vs = wv_smem + m;
  double* a = A + (size_t)z * k * k;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    ws[i] = wbuf[(size_t)z * k + j + 1 + i];
    vs[i] = vbuf[(size_t)z * k + j + 1 + i];
  }
  __syncthreads();
  for (int l = blockIdx.x; l < m; l += gridDim.x) {
    double* cl = a + (size_t)(j + 1 + l) * k + j + 1;
    const double vl = vs[l], wl = ws[l];
    for (int i = threadIdx.x; i < m; i += blockDim.x) cl[i] -= vs[i] * wl + ws[i] * vl;
  }
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < m; i += blockDim.x) a[(size_t)j * k + j + 1 + i] = vs[i];
}

// the last 2 x 2 block: d[k-2], d[k-1], e[k-2]
__global__ void tail_kernel(const double* __restrict__ A, int k, double* __restrict__ d, double* __restrict__ e) {
  const int z = blockIdx.x;
  const double* a = A + (size_t)z * k * k;
  if (threadIdx.x == 0) {
    if (k >= 2) {
      d[(size_t)z * k + k - 2] = a[(size_t)(k - 2) * k + k - 2];
      e[(size_t)z * k + k - 2] = a[(size_t)(k - 2) * k + k - 1];
    }
    d[(size_t)z * k + k - 1] = a[(size_t)(k - 1) * k + k - 1];
  }
}

// number of eigenvalues of T (d, e) below x: negative pivots of the LDL^T factorisation of
// T - x I; a zero pivot is replaced by -pivmin (LAPACK's dlaebz convention)
__device__ int sturm_count(const double* d, const double* e, int k, double x, double pivmin) {
  int cnt = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0.0) ++cnt;
  for (int i = 1; i < k; ++i) {
    q = (d[i] - x) - e[i - 1] * e[i - 1] * rcp_nr(q);
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

// lam[z * k + i] = the i-th smallest eigenvalue of T_z, by multisection of the Gershgorin
// interval: a group of L lanes (L a power of two up to 32, the lanes of one warp) works on one
// eigenvalue, lane j counting the eigenvalues below the point x_j = lo + (j + 1)(hi - lo)/(L + 1);
// the first point whose count exceeds i becomes hi and the point before it lo (bisection for
// L = 1). Every lane of the group computes the same lo and hi. The matrix's own rounding
// leaves every eigenvalue an absolute uncertainty of order eps ||T||, so the search stops
// at an interval of 4 eps ||T||.
__global__ void __launch_bounds__(32) multisect_kernel(const double* __restrict__ d, const double* __restrict__ e,
                                                       int k, int nb, int L, double* __restrict__ lam) {
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)k * nb;
  const int64_t q = gtid / L;
  const int lane = threadIdx.x & 31, j = lane & (L - 1);
  // the whole group takes the same q: groups past the end work on the last eigenvalue and
  // write nothing, so that every lane of a warp takes part in the ballots
  const int64_t qq = q < total ? q : total - 1;
  const int z = (int)(qq / k), i = (int)(qq % k);
  const double* dz = d + (size_t)z * k;
  const double* ez = e + (size_t)z * k;
  double lo = dz[0], hi = dz[0], emax2 = 0.0;
  for (int r = 0; r < k; ++r) {
    const double rad = (r > 0 ? fabs(ez[r - 1]) : 0.0) + (r < k - 1 ? fabs(ez[r]) : 0.0);
    lo = fmin(lo, dz[r] - rad);
    hi = fmax(hi, dz[r] + rad);
    if (r < k - 1) emax2 = fmax(emax2, ez[r] * ez[r]);
  }
  const double tnorm = fmax(fabs(lo), fabs(hi));
  const double pivmin = fmax(2.2250738585072014e-308 * fmax(emax2, 1.0), 1e-300);
  lo -= 2.0 * 2.2204460492503131e-16 * tnorm + pivmin;
  hi += 2.0 * 2.2204460492503131e-16 * tnorm + pivmin;
  const double tol = 4.0 * 2.2204460492503131e-16 * tnorm + pivmin;
  const unsigned gmask = L == 32 ? 0xffffffffu : (((1u << L) - 1u) << (lane & ~(L - 1)));
  for (int it = 0; it < 200; ++it) {
    if (hi - lo <= tol) break;
    const double step = (hi - lo) / (double)(L + 1);
    const double x0 = lo + step, xl = lo + (double)L * step;
    if (x0 <= lo || xl >= hi) break;
    const double x = lo + (double)(j + 1) * step;
    const bool above = sturm_count(dz, ez, k, x, pivmin) > i;
    unsigned bits = __ballot_sync(gmask, above) & gmask;
    bits >>= (lane & ~(L - 1));
    const int f = bits ? __ffs(bits) - 1 : L;  // first point whose count exceeds i
    const double nlo = f == 0 ? lo : lo + (double)f * step;
    const double nhi = f == L ? hi : lo + (double)(f + 1) * step;
    lo = nlo;
    hi = nhi;
  }
  if (q < total && j == 0) lam[q] = 0.5 * (lo + hi);
}

// Inverse iteration for the selected eigenvalues. One block per cluster: sel[c0 .. c1) of
// (matrix, eigenvalue) entries listed in `job` (start, count) per cluster; the eigenvalues of a
// cluster belong to one matrix and are processed in order. Thread 0 solves (T - lambda I) y = x
// by Gaussian elimination with partial pivoting (a tridiagonal LU, fill-in one super-diagonal,
// the reciprocals of the pivots kept); the block normalises and re-orthogonalises y against the
// cluster's earlier vectors. Vectors go to V[z] columns vcol (k x ncols per matrix,
// column-major). The factors and y (5 k doubles and k pivot flags) sit in dynamic shared memory
// when `in_smem`, else in work (6 k doubles per block).
__global__ void __launch_bounds__(EB) inverse_iteration_kernel(const double* __restrict__ d, const double* __restrict__ e,
                                                               int k, const int* __restrict__ job,
                                                               const int* __restrict__ sel_z,
                                                               const double* __restrict__ sel_lam,
                                                               const int* __restrict__ sel_col, double* V, int ncols,
                                                               double* work, int in_smem) {
  extern __shared__ double ii_smem[];
  __shared__ double sh[32];
  const int c0 = job[2 * blockIdx.x], cn = job[2 * blockIdx.x + 1];
  double* wk = in_smem ? ii_smem : work + (size_t)blockIdx.x * 6 * k;
  double* dl = wk;           // multipliers
  double* rdu = wk + k;      // reciprocals of the upper factor's diagonal
  double* du1 = wk + 2 * k;  // first super-diagonal
  double* du2 = wk + 3 * k;  // second super-diagonal (fill-in)
  double* y = wk + 4 * k;
  unsigned char* piv = reinterpret_cast<unsigned char*>(wk + 5 * k);
  const int z = sel_z[c0];
  const double* dz = d + (size_t)z * k;
  const double* ez = e + (size_t)z * k;
  double tn = 0.0;  // ||T||_1
  for (int r = 0; r < k; ++r) tn = fmax(tn, fabs(dz[r]) + (r > 0 ? fabs(ez[r - 1]) : 0.0) + (r < k - 1 ? fabs(ez[r]) : 0.0));
  const double eps = 2.2204460492503131e-16;
  const double tiny = fmax(eps * tn, 1e-300);
  for (int q = c0; q < c0 + cn; ++q) {
    const double lambda = sel_lam[q];
    double* vz = V + (size_t)z * k * ncols;
    double* vout = vz + (size_t)sel_col[q] * k;
    // LU of T - lambda I with partial pivoting (thread 0)
    if (threadIdx.x == 0) {
      double a = dz[0] - lambda, b = k > 1 ? ez[0] : 0.0;
      for (int r = 0; r < k - 1; ++r) {
        const double c = ez[r], dn = dz[r + 1] - lambda, en = r + 1 < k - 1 ? ez[r + 1] : 0.0;
        if (fabs(a) >= fabs(c)) {
          if (fabs(a) < tiny) a = tiny;
          const double ra = rcp_nr(a), m = c * ra;
          dl[r] = m;
          piv[r] = 0;
          rdu[r] = ra;
          du1[r] = b;
          du2[r] = 0.0;
          a = dn - m * b;
          b = en;
        } else {
          const double rc = rcp_nr(c), m = a * rc;
          dl[r] = m;
          piv[r] = 1;
          rdu[r] = rc;
          du1[r] = dn;
          du2[r] = en;
          a = b - m * dn;
          b = -m * en;
        }
      }
      if (fabs(a) < tiny) a = tiny;
      rdu[k - 1] = rcp_nr(a);
    }
    // start vector: a fixed, non-degenerate one
    for (int r = threadIdx.x; r < k; r += blockDim.x) y[r] = 1.0 + 0.3 * sin(1.7 * (r + 1) + 0.37 * (q - c0 + 1));
    __syncthreads();
    for (int it = 0; it < 3; ++it) {
      if (threadIdx.x == 0) {
        // Both sweeps carry the entries still being updated in registers: every load reads an
        // entry the sweep has not written yet and every store is final, so no entry is read
        // back after a store to it.
        // forward: apply the row interchanges and multipliers; cur is the working row's entry
        double cur = y[0];
        for (int r = 0; r < k - 1; ++r) {
          const double nxt = y[r + 1];
          if (piv[r]) {
            y[r] = nxt;
            cur = cur - dl[r] * nxt;
          } else {
            y[r] = cur;
            cur = nxt - dl[r] * cur;
          }
        }
        // back substitution with the upper factor (diagonal, two super-diagonals); x1, x2 are
        // the solution entries r + 1 and r + 2
        double x1 = cur * rdu[k - 1], x2 = 0.0;
        y[k - 1] = x1;
        for (int r = k - 2; r >= 0; --r) {
          const double x0 = (y[r] - du1[r] * x1 - du2[r] * x2) * rdu[r];
          y[r] = x0;
          x2 = x1;
          x1 = x0;
        }
      }
      __syncthreads();
      // orthogonalise against the earlier vectors of the cluster, then normalise
      for (int p = c0; p < q; ++p) {
        const double* u = vz + (size_t)sel_col[p] * k;
        double s = 0.0;
        for (int r = threadIdx.x; r < k; r += blockDim.x) s += u[r] * y[r];
        const double dot = block_sum(s, sh);
        for (int r = threadIdx.x; r < k; r += blockDim.x) y[r] -= dot * u[r];
        __syncthreads();
      }
      double s = 0.0;
      for (int r = threadIdx.x; r < k; r += blockDim.x) s += y[r] * y[r];
      const double nrm = sqrt(block_sum(s, sh));
      const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
      for (int r = threadIdx.x; r < k; r += blockDim.x) y[r] *= inv;
      __syncthreads();
    }
    for (int r = threadIdx.x; r < k; r += blockDim.x) vout[r] = y[r];
    __syncthreads();
  }
}

// V <- H_0 .. H_{k-3} V for the ncols columns of each matrix (column block per CTA): the
// reflectors applied from the last to the first, y <- y - tau v (v^T y)
__global__ void __launch_bounds__(EB) back_transform_kernel(const double* __restrict__ A, const double* __restrict__ tau,
                                                            int k, double* __restrict__ V, int ncols) {
  __shared__ double sh[32];
  const int z = blockIdx.y, col = blockIdx.x;
  if (col >= ncols) return;
  const double* a = A + (size_t)z * k * k;
  double* y = V + ((size_t)z * ncols + col) * k;
  for (int j = k - 3; j >= 0; --j) {
    const double t = tau[(size_t)z * k + j];
    if (t == 0.0) continue;
    const double* v = a + (size_t)j * k;
    double s = 0.0;
    for (int r = j + 1 + threadIdx.x; r < k; r += blockDim.x) s += v[r] * y[r];
    const double dot = block_sum(s, sh);
    for (int r = j + 1 + threadIdx.x; r < k; r += blockDim.x) y[r] -= t * dot * v[r];
    __syncthreads();
  }
}

}  // namespace

// Tridiagonalises nb symmetric k x k matrices (A: nb x k x k, column-major, overwritten by the
// reflectors) and returns every eigenvalue in ascending order (lam: nb x k), plus the
// tridiagonal (d, e: nb x k) and tau (nb x k) for sym_eig_vectors. Device buffers throughout.
pttk_status sym_eig_values(double* A, int k, int nb, double* d, double* e, double* tau, double* lam, cudaStream_t s) {
  if (k < 1 || nb < 1) return set_error(PTTK_EINVAL, "empty eigenproblem");
  if (k >= 3) {
    const size_t wv_bytes = sizeof(double) * 2 * (size_t)(k - 1);
    if (wv_bytes > 200 * 1024) return set_error(PTTK_ENOTSUP, "eigenproblem larger than 12800 x 12800");
    if (wv_bytes > 48 * 1024)
      PTTK_CUDA(cudaFuncSetAttribute(w_rank2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wv_bytes));
    const int nch_max = (k + CHUNK - 1) / CHUNK;
    double *part = nullptr, *vbuf = nullptr, *wbuf = nullptr;
    unsigned* done = nullptr;
    PTTK_CUDA(cudaMallocAsync(&part, sizeof(double) * (size_t)nb * nch_max * k, s));
    PTTK_CUDA(cudaMallocAsync(&vbuf, sizeof(double) * (size_t)nb * k, s));
    PTTK_CUDA(cudaMallocAsync(&wbuf, sizeof(double) * (size_t)nb * k, s));
    PTTK_CUDA(cudaMallocAsync(&done, sizeof(unsigned) * (size_t)nb * k, s));
    PTTK_CUDA(cudaMemsetAsync(done, 0, sizeof(unsigned) * (size_t)nb * k, s));
    PTTK_PROF("eig_tridiag", s);
    const int gmax = std::max(1, 2 * sm_count() / nb);
    for (int j = 0; j < k - 2; ++j) {
      const int m = k - j - 1, nch = (m + CHUNK - 1) / CHUNK;
      reflect_symv_kernel<<<dim3((unsigned)((m + SB - 1) / SB), (unsigned)nch, (unsigned)nb), SB * 4, 0, s>>>(
          A, k, j, nch, part, vbuf, tau, d, e, done, wbuf);
      pttk::count_launch();
      w_rank2_kernel<<<dim3((unsigned)std::min(m, gmax), 1, (unsigned)nb), EB, sizeof(double) * 2 * (size_t)m, s>>>(
          A, k, j, wbuf, vbuf);
      pttk::count_launch();
    }
    cudaFreeAsync(part, s);
    cudaFreeAsync(vbuf, s);
    cudaFreeAsync(wbuf, s);
    cudaFreeAsync(done, s);
  }
  tail_kernel<<<nb, 32, 0, s>>>(A, k, d, e); pttk::count_launch();
  {
    // lanes per eigenvalue: the most (up to 32) that keep about one warp per SM, the FP64
    // pipe being the limit of the Sturm counts
    const int64_t nt = (int64_t)k * nb;
    int L = 1;
    while (L < 32 && (nt * 2 * L + 31) / 32 <= sm_count()) L *= 2;
    const int64_t threads = nt * L;
    PTTK_PROF("eig_bisect", s);
    multisect_kernel<<<(unsigned)((threads + 31) / 32), 32, 0, s>>>(d, e, k, nb, L, lam); pttk::count_launch();
  }
  PTTK_CUDA(cudaGetLastError());
  return PTTK_OK;
}

// Eigenvectors of the matrices tridiagonalised by sym_eig_values for selected eigenvalues:
// selection q has matrix sel_z[q], eigenvalue sel_lam[q], weight sel_w[q] and output column
// sel_col[q] of V (nb x k x ncols, column-major per matrix). Selections of one matrix must be
// listed in ascending order of eigenvalue. Host arrays; synchronises `s`.
//
// Clusters. Inverse iteration gives each vector as an eigenvector of its own perturbation
// T + E_q, ||E_q|| ~ eps ||T||, so two vectors carry components of about eps ||T|| / gap along
// each other. In a spectral function sum f(lambda_q) u_q u_q^T such a pair is off by about
// |f| eps ||T|| / gap. Re-orthogonalising the pairs whose gap is below 1e-3 max(|f|) (LAPACK's
// dstein uses 1e-3 ||T|| for every pair) keeps that below 1e3 eps ||T|| per pair, while
// eigenvalues that are small against ||T|| (the numerically low-rank tail, dense in absolute
// terms) stay in clusters of their own and run in parallel.
pttk_status sym_eig_vectors(const double* A, const double* d, const double* e, const double* tau, int k, int nb,
                            const std::vector<int>& sel_z, const std::vector<double>& sel_lam,
                            const std::vector<double>& sel_w, const std::vector<int>& sel_col, double* V,
                            int ncols, cudaStream_t s) {
  const int nsel = (int)sel_z.size();
  if (nsel == 0) return PTTK_OK;
  if ((int)sel_lam.size() != nsel || (int)sel_w.size() != nsel || (int)sel_col.size() != nsel)
    return set_error(PTTK_EINVAL, "eigenvector selection arrays of different lengths");
  // clusters: consecutive selections of one matrix closer than 1e-3 of the larger weight
  std::vector<int> job;
  int start = 0;
  for (int q = 1; q <= nsel; ++q) {
    const bool brk = q == nsel || sel_z[q] != sel_z[q - 1] ||
                     std::fabs(sel_lam[q] - sel_lam[q - 1]) > 1e-3 * std::max(sel_w[q], sel_w[q - 1]);
    if (brk) {
      job.push_back(start);
      job.push_back(q - start);
      start = q;
    }
  }
  const int nclus = (int)job.size() / 2;
  int *djob = nullptr, *dz = nullptr, *dcol = nullptr;
  double *dlam = nullptr, *work = nullptr;
  PTTK_CUDA(cudaMallocAsync(&djob, sizeof(int) * job.size(), s));
  PTTK_CUDA(cudaMallocAsync(&dz, sizeof(int) * nsel, s));
  PTTK_CUDA(cudaMallocAsync(&dcol, sizeof(int) * nsel, s));
  PTTK_CUDA(cudaMallocAsync(&dlam, sizeof(double) * nsel, s));
  // factors in shared memory up to k = 4900 (5 k doubles + k flags); beyond, in global memory
  const size_t ii_bytes = sizeof(double) * 5 * (size_t)k + (size_t)k;
  const int in_smem = ii_bytes <= 200 * 1024;
  if (in_smem && ii_bytes > 48 * 1024)
    PTTK_CUDA(cudaFuncSetAttribute(inverse_iteration_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ii_bytes));
  PTTK_CUDA(cudaMallocAsync(&work, in_smem ? sizeof(double) : sizeof(double) * 6 * (size_t)k * nclus, s));
  PTTK_CUDA(cudaMemcpyAsync(djob, job.data(), sizeof(int) * job.size(), cudaMemcpyHostToDevice, s));
  PTTK_CUDA(cudaMemcpyAsync(dz, sel_z.data(), sizeof(int) * nsel, cudaMemcpyHostToDevice, s));
  PTTK_CUDA(cudaMemcpyAsync(dcol, sel_col.data(), sizeof(int) * nsel, cudaMemcpyHostToDevice, s));
  PTTK_CUDA(cudaMemcpyAsync(dlam, sel_lam.data(), sizeof(double) * nsel, cudaMemcpyHostToDevice, s));
  inverse_iteration_kernel<<<nclus, EB, in_smem ? ii_bytes : 0, s>>>(d, e, k, djob, dz, dlam, dcol, V, ncols, work,
                                                                     in_smem);
  pttk::count_launch();
  back_transform_kernel<<<dim3((unsigned)ncols, (unsigned)nb), EB, 0, s>>>(A, tau, k, V, ncols); pttk::count_launch();
  PTTK_CUDA(cudaGetLastError());
  PTTK_CUDA(cudaStreamSynchronize(s));
  cudaFreeAsync(djob, s);
  cudaFreeAsync(dz, s);
  cudaFreeAsync(dcol, s);
  cudaFreeAsync(dlam, s);
  cudaFreeAsync(work, s);
  return PTTK_OK;
}

}  // namespace pttk

// PTTK-Global (Algorithm 4, Section 3 "Global low-rank approximation"): one point set X in
// one box (source box = target box) and a kernel symmetric in its arguments.
//
// Offline: S = U(X), T = V(X) by the FP64 factor chains of Algorithm 2 (Phase 3) on the one
// point set; the thin QR [S T] = Q R. Q is an orthonormal basis of the range of [S T] (the
// TT-SVD's pivoted Householder QR and one-sided Jacobi, delta = 0) and R = Q^T [S T]: any
// factor pair with orthonormal Q and Q R = [S T] gives the same Q R H^ R^T Q^T, which is all
// Algorithm 4 uses.
//
// Online, per theta: H = H(theta) (Algorithm 3); R H^ R^T = sym(C1), C1 = R_s H R_t^T
// (Eq. pttk1: H^ = [[0, H/2], [H^T/2, 0]], R = [R_s R_t]); its eigendecomposition by Householder
// tridiagonalisation, bisection and inverse iteration (eig.cu). Eigenvalues within
// 64 eps max|lambda| of zero are below FP64's resolution for this matrix and give no term.
//
// The Gaussian-process use of Section 1 (pttk_gp_lml): the log marginal likelihood of
// y ~ N(0, K~ + s2 I) and its theta gradient for the low-rank kernel K~ = Q sym(C1) Q^T =
// sym(S H T^T), reduced to k x k algebra on B = sym(C1) (Woodbury and the eigenbasis of B).
//
// Memory: the handle keeps Q (N x k row-major, k <= r_s + r_t), R (k x (r_s + r_t)) and a copy
// of the FP64 cores (for H(theta)); the offline stage holds about five N x (r_s + r_t) FP64
// buffers at its peak.
#include "pttk_internal.cuh"

#include <cmath>
#include <numeric>

struct pttk_global {
  pttk_tt tt;          // metadata of the TT; tt.cores64 is a private copy of its FP64 cores
  int64_t N = 0;
  int rs = 0, rt = 0;  // r_d and r_{d+d_theta}: columns of S and of T
  int k = 0;           // columns of Q
  double* Q = nullptr; // dev, N x k row-major
  double* R = nullptr; // dev, k x (rs + rt) column-major
};

namespace pttk {
namespace {

struct DevBuf {
  double* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  pttk_status alloc(size_t elems) {
    if (p) cudaFree(p);
    p = nullptr;
    const cudaError_t e = cudaMalloc(&p, std::max<size_t>(elems, 1) * sizeof(double));
    if (e != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      return set_error(PTTK_ENOMEM, "device allocation failed in PTTK-Global");
    }
    return PTTK_OK;
  }
};

// A (N x (rs + rt), column-major) = [S T]; S (N x rs) and T (N x rt) row-major. 32 x 32 tiles
// through shared memory, so that both the reads and the writes are coalesced.
__global__ void concat_cols_kernel(const double* __restrict__ S, const double* __restrict__ T,
                                   int64_t N, int rs, int rt, double* __restrict__ A) {
  __shared__ double t[32][33];
  const int kk = rs + rt;
  const int64_t p0 = (int64_t)blockIdx.x * 32;
  const int j0 = (int)blockIdx.y * 32;
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int64_t p = p0 + yy;
    const int j = j0 + (int)threadIdx.x;
    double v = 0.0;
    if (p < N && j < kk) v = j < rs ? S[p * rs + j] : T[p * rt + (j - rs)];
    t[yy][threadIdx.x] = v;
  }
  __syncthreads();
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int j = j0 + yy;
    const int64_t p = p0 + threadIdx.x;
    if (p < N && j < kk) A[p + (int64_t)j * N] = t[threadIdx.x][yy];
  }
}

// Qr (N x k, row-major) = Qc (N x k, column-major)
__global__ void to_rowmajor_kernel(const double* __restrict__ Qc, int64_t N, int k,
                                   double* __restrict__ Qr) {
  __shared__ double t[32][33];
  const int64_t p0 = (int64_t)blockIdx.x * 32;
  const int j0 = (int)blockIdx.y * 32;
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int j = j0 + yy;
    const int64_t p = p0 + threadIdx.x;
    if (p < N && j < k) t[yy][threadIdx.x] = Qc[p + (int64_t)j * N];
  }
  __syncthreads();
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int64_t p = p0 + yy;
    const int j = j0 + (int)threadIdx.x;
    if (p < N && j < k) Qr[p * k + j] = t[threadIdx.x][yy];
  }
}

// B = (C + C^T) / 2 + shift I, k x k column-major
__global__ void sym_shift_kernel(const double* __restrict__ C, int k, double shift,
                                 double* __restrict__ B) {
  const int64_t total = (int64_t)k * k;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % k), j = (int)(e / k);
    B[e] = 0.5 * (C[i + (int64_t)j * k] + C[j + (int64_t)i * k]) + (i == j ? shift : 0.0);
  }
}

// *out = sum of x[i]^2, one block of 1024 threads, summed in a fixed order
__global__ void __launch_bounds__(1024) sumsq_block_kernel(const double* __restrict__ x, int64_t n,
                                                           double* __restrict__ out) {
  __shared__ double part[1024];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += 1024) acc = fma(x[i], x[i], acc);
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = part[0];
}

// *out = ||(C - C^T) / 2||_F^2 (C: k x k, column-major), one block of 1024 threads
__global__ void __launch_bounds__(1024) asym_sumsq_block_kernel(const double* __restrict__ C, int k,
                                                                double* __restrict__ out) {
  __shared__ double part[1024];
  double acc = 0.0;
  const int64_t total = (int64_t)k * k;
  for (int64_t e = threadIdx.x; e < total; e += 1024) {
    const int i = (int)(e % k), j = (int)(e / k);
    const double a = 0.5 * (C[e] - C[j + (int64_t)i * k]);
    acc = fma(a, a, acc);
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = part[0];
}

// out[:, q] = A[:, q] * scale[q], rows x m column-major
__global__ void scale_cols_kernel(const double* __restrict__ A, int64_t rows, const double* __restrict__ scale, int m,
                                  double* __restrict__ out) {
  const int64_t total = rows * m;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = A[e] * scale[e / rows];
}

// W = diag(lam), m x m
__global__ void diag_kernel(const double* __restrict__ lam, int m, double* __restrict__ W) {
  const int64_t total = (int64_t)m * m;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % m), j = (int)(e / m);
    W[e] = i == j ? lam[i] : 0.0;
  }
}

unsigned blocks_for(int64_t work, int threads) {
  const int64_t b = (work + threads - 1) / threads;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)sm_count() * 8));
}

}  // namespace

// Offline stage of Algorithm 4 into g (g->tt already holds the metadata).
static pttk_status global_create_run(const pttk_tt* tt, const double* X, int64_t N, pttk_global* g,
                                     cudaStream_t s) {
  const int d = tt->d, dth = tt->dtheta;
  const int rs = tt->ranks[d], rt = tt->ranks[d + dth], kk = rs + rt;
  g->N = N;
  g->rs = rs;
  g->rt = rt;
  // the FP64 cores, for H(theta) in the online stage
  PTTK_CUDA(cudaMalloc(&g->tt.cores64, sizeof(double) * std::max<size_t>(tt->core_total, 1)));
  PTTK_CUDA(cudaMemcpyAsync(g->tt.cores64, tt->cores64, sizeof(double) * tt->core_total,
                            cudaMemcpyDeviceToDevice, s));
  g->tt.cores32 = nullptr;
  DevBuf S, T, A;
  PTTK_TRY(S.alloc((size_t)N * rs));
  PTTK_TRY(T.alloc((size_t)N * rt));
  {
    PTTK_PROF("global_factors", s);
    PTTK_TRY(factor_build_run(tt, true, X, N, PTTK_FP64, S.p, s));
    PTTK_TRY(factor_build_run(tt, false, X, N, PTTK_FP64, T.p, s));
  }
  PTTK_TRY(A.alloc((size_t)N * kk));
  const dim3 tb(32, 8);
  concat_cols_kernel<<<dim3((unsigned)((N + 31) / 32), (unsigned)((kk + 31) / 32)), tb, 0, s>>>(
      S.p, T.p, N, rs, rt, A.p); pttk::count_launch();
  PTTK_CUDA(cudaGetLastError());
  cudaFree(S.p);
  S.p = nullptr;
  cudaFree(T.p);
  T.p = nullptr;
  // Q: orthonormal basis of range([S T]) (N x k column-major), R = Q^T [S T]
  DevBuf Qc;
  int k = 0;
  PTTK_TRY(range_basis(A.p, N, kk, &Qc.p, &k, s));
  g->k = k;
  PTTK_CUDA(cudaMalloc(&g->R, sizeof(double) * (size_t)k * kk));
  dgemm(true, false, k, kk, N, 1.0, Qc.p, N, A.p, N, 0.0, g->R, k, s);
  PTTK_CUDA(cudaMalloc(&g->Q, sizeof(double) * (size_t)N * k));
  to_rowmajor_kernel<<<dim3((unsigned)((N + 31) / 32), (unsigned)((k + 31) / 32)), tb, 0, s>>>(
      Qc.p, N, k, g->Q); pttk::count_launch();
  PTTK_CUDA(cudaGetLastError());
  PTTK_CUDA(cudaStreamSynchronize(s));
  return PTTK_OK;
}

// Online stage of Algorithm 4 at theta_hat.
static pttk_status global_online_run(const pttk_global* g, const double* th, double eps, bool compress,
                                     bool definite, double* Z, double* W, int* rank, cudaStream_t s) {
  const int k = g->k, rs = g->rs, rt = g->rt;
  const int64_t N = g->N;
  DevBuf H, P, C1, B, t2d;
  PTTK_TRY(H.alloc((size_t)rs * rt));
  PTTK_TRY(P.alloc((size_t)k * rt));
  PTTK_TRY(C1.alloc((size_t)k * k));
  PTTK_TRY(B.alloc((size_t)k * k));
  PTTK_TRY(t2d.alloc(2));
  PTTK_TRY(theta_core_run(&g->tt, th, true, H.p, s));  // H(theta), rs x rt row-major
  // P = R_s H (k x rt); H row-major is H^T column-major with leading dimension rt
  dgemm(false, true, k, rt, rs, 1.0, g->R, k, H.p, rt, 0.0, P.p, k, s);
  // C1 = P R_t^T (k x k) = R E R^T, E = [[0, H], [0, 0]]: Q C1 Q^T = S H T^T
  dgemm(false, true, k, k, rt, 1.0, P.p, k, g->R + (size_t)k * rs, k, 0.0, C1.p, k, s);
  // ||C1||_F^2 and ||(C1 - C1^T)/2||_F^2
  sumsq_block_kernel<<<1, 1024, 0, s>>>(C1.p, (int64_t)k * k, t2d.p); pttk::count_launch();
  asym_sumsq_block_kernel<<<1, 1024, 0, s>>>(C1.p, k, t2d.p + 1); pttk::count_launch();
  PTTK_CUDA(cudaGetLastError());
  double t2a[2] = {0.0, 0.0};
  PTTK_CUDA(cudaMemcpyAsync(t2a, t2d.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  PTTK_CUDA(cudaStreamSynchronize(s));
  const double t2 = t2a[0], a2 = t2a[1];
  if (!(t2 > 0.0)) {
    // S H T^T = 0: W = 0 (Global-1) or no term (Global-2)
    if (!compress) PTTK_CUDA(cudaMemsetAsync(W, 0, sizeof(double) * (size_t)k * k, s));
    *rank = compress ? 0 : k;
    PTTK_CUDA(cudaStreamSynchronize(s));
    return PTTK_OK;
  }
  // B = sym(C1) = (C1 + C1^T)/2: Q B Q^T = Q R H^ R^T Q^T, the matrix of Algorithm 4
  sym_shift_kernel<<<blocks_for((int64_t)k * k, 256), 256, 0, s>>>(C1.p, k, 0.0, B.p); pttk::count_launch();
  PTTK_CUDA(cudaGetLastError());
  DevBuf dd, ee, dtau, dlam_all;
  PTTK_TRY(dd.alloc(k));
  PTTK_TRY(ee.alloc(k));
  PTTK_TRY(dtau.alloc(k));
  PTTK_TRY(dlam_all.alloc(k));
  {
    PTTK_PROF("global_eig", s);
    PTTK_TRY(sym_eig_values(B.p, k, 1, dd.p, ee.p, dtau.p, dlam_all.p, s));
  }
  std::vector<double> lam(k);
  PTTK_CUDA(cudaMemcpyAsync(lam.data(), dlam_all.p, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
  PTTK_CUDA(cudaStreamSynchronize(s));
  // eigenvalues in decreasing |lambda|; a definite kernel drops the negative ones. Eigenvalues
  // within 64 eps max|lambda| of zero are below what FP64 resolves (their computed values carry
  // absolute errors of that order, sign included) and count as zero: no term.
  double lmax = 0.0;
  for (int i = 0; i < k; ++i) lmax = std::max(lmax, std::fabs(lam[i]));
  const double res = 64.0 * 2.2204460492503131e-16 * lmax;
  std::vector<int> order(k);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return std::fabs(lam[a]) > std::fabs(lam[b]); });
  std::vector<int> kept;
  std::vector<char> is_kept(k, 0);
  for (int i : order)
    if ((!definite || lam[i] > 0.0) && std::fabs(lam[i]) > res) {
      kept.push_back(i);
      is_kept[i] = 1;
    }
  int m = (int)kept.size();
  if (compress) {
    // ||Q U_j Lambda_j U_j^T Q^T - S H T^T||_F^2 = ||C1 - U_j Lambda_j U_j^T||_F^2
    //   = ||(C1 - C1^T)/2||_F^2 + (sum of lambda_i^2 over the eigenpairs not kept),
    // the symmetric and antisymmetric parts being orthogonal, summed from the discarded terms
    // themselves (||C1||^2 - sum of the kept lambda^2 would cancel).
    const double bound2 = eps * eps * t2;
    double excl2 = 0.0;  // eigenvalues not eligible: negative ones of a definite kernel, unresolved ones
    for (int i = 0; i < k; ++i)
      if (!is_kept[i]) excl2 += lam[i] * lam[i];
    std::vector<double> tail(kept.size() + 1, 0.0);  // tail[j] = sum over kept[j..] of lambda^2
    for (int q = (int)kept.size() - 1; q >= 0; --q) tail[q] = tail[q + 1] + lam[kept[q]] * lam[kept[q]];
    int j = 0;
    while (j < (int)kept.size() && a2 + excl2 + tail[j] > bound2) ++j;
    m = j;
  }
  *rank = compress ? m : k;
  if (m == 0) {
    if (!compress) PTTK_CUDA(cudaMemsetAsync(W, 0, sizeof(double) * (size_t)k * k, s));
    PTTK_CUDA(cudaStreamSynchronize(s));
    return PTTK_OK;
  }
  // eigenvectors of the m terms (column q of Un for kept[q]), computed in ascending order of
  // eigenvalue as the inverse iteration's clustering needs
  DevBuf Un, Ul, dlam;
  PTTK_TRY(Un.alloc((size_t)k * m));
  {
    std::vector<int> idx(kept.begin(), kept.begin() + m), pos(m);
    std::vector<int> asc(m);
    std::iota(asc.begin(), asc.end(), 0);
    std::stable_sort(asc.begin(), asc.end(), [&](int a, int b) { return lam[idx[a]] < lam[idx[b]]; });
    std::vector<int> sz(m, 0), scol(m);
    std::vector<double> slam(m), sw(m);
    for (int q = 0; q < m; ++q) {
      slam[q] = lam[idx[asc[q]]];
      // Global-1 needs W = sum lambda u u^T (weight |lambda|); Global-2 hands out Z = Q U^,
      // whose columns must be orthonormal to working accuracy (weight max |lambda|, LAPACK's
      // absolute rule, over its m leading pairs only)
      sw[q] = compress ? lmax : std::fabs(slam[q]);
      scol[q] = asc[q];
    }
    PTTK_PROF("global_eigvec", s);
    PTTK_TRY(sym_eig_vectors(B.p, dd.p, ee.p, dtau.p, k, 1, sz, slam, sw, scol, Un.p, m, s));
  }
  std::vector<double> lk(m);
  for (int q = 0; q < m; ++q) lk[q] = lam[kept[q]];
  PTTK_TRY(dlam.alloc(m));
  PTTK_CUDA(cudaMemcpyAsync(dlam.p, lk.data(), sizeof(double) * m, cudaMemcpyHostToDevice, s));
  if (!compress) {
    // W = U Lambda U^T (k x k)
    PTTK_TRY(Ul.alloc((size_t)k * m));
    scale_cols_kernel<<<blocks_for((int64_t)k * m, 256), 256, 0, s>>>(Un.p, k, dlam.p, m, Ul.p); pttk::count_launch();
    PTTK_CUDA(cudaGetLastError());
    dgemm(false, true, k, k, m, 1.0, Ul.p, k, Un.p, k, 0.0, W, k, s);
  } else {
    // Z = Q U^ (N x m row-major): Z^T (m x N column-major) = U^T Q^T, Q^T being Q row-major
    {
      PTTK_PROF("global_z", s);
      dgemm(true, false, m, N, k, 1.0, Un.p, k, g->Q, k, 0.0, Z, m, s);
    }
    diag_kernel<<<blocks_for((int64_t)m * m, 256), 256, 0, s>>>(dlam.p, m, W); pttk::count_launch();
    PTTK_CUDA(cudaGetLastError());
  }
  PTTK_CUDA(cudaStreamSynchronize(s));
  return PTTK_OK;
}

// Online stage of Algorithm 4, uncompressed (PTTK-Global-1), for B parameter values at once:
// the B matrices sym(C1(theta_b)) go through one batched eigensolver call (every launch of the
// tridiagonalisation, the eigenvalues and the eigenvectors covers all of them), then
// W_b = U_b Lambda_b U_b^T with the same selection as the single-theta call.
static pttk_status global_online_batched_run(const pttk_global* g, const double* th_all, int nb, bool definite,
                                             double* W, cudaStream_t s) {
  const int k = g->k, rs = g->rs, rt = g->rt;
  const size_t kk = (size_t)k * k;
  DevBuf H, P, C1, Bb, t2d, dd, ee, dtau, dlam;
  PTTK_TRY(H.alloc((size_t)rs * rt));
  PTTK_TRY(P.alloc((size_t)k * rt));
  PTTK_TRY(C1.alloc(kk));
  PTTK_TRY(Bb.alloc(kk * nb));
  PTTK_TRY(t2d.alloc(nb));
  PTTK_TRY(dd.alloc((size_t)k * nb));
  PTTK_TRY(ee.alloc((size_t)k * nb));
  PTTK_TRY(dtau.alloc((size_t)k * nb));
  PTTK_TRY(dlam.alloc((size_t)k * nb));
  for (int b = 0; b < nb; ++b) {
    PTTK_TRY(theta_core_run(&g->tt, th_all + (size_t)b * PTTK_MAX_D, true, H.p, s));
    dgemm(false, true, k, rt, rs, 1.0, g->R, k, H.p, rt, 0.0, P.p, k, s);
    dgemm(false, true, k, k, rt, 1.0, P.p, k, g->R + (size_t)k * rs, k, 0.0, C1.p, k, s);
    sumsq_block_kernel<<<1, 1024, 0, s>>>(C1.p, (int64_t)kk, t2d.p + b); pttk::count_launch();
    sym_shift_kernel<<<blocks_for((int64_t)kk, 256), 256, 0, s>>>(C1.p, k, 0.0, Bb.p + kk * b); pttk::count_launch();
  }
  PTTK_CUDA(cudaGetLastError());
  {
    PTTK_PROF("global_eig", s);
    PTTK_TRY(sym_eig_values(Bb.p, k, nb, dd.p, ee.p, dtau.p, dlam.p, s));
  }
  std::vector<double> lam((size_t)k * nb), t2(nb);
  PTTK_CUDA(cudaMemcpyAsync(lam.data(), dlam.p, sizeof(double) * lam.size(), cudaMemcpyDeviceToHost, s));
  PTTK_CUDA(cudaMemcpyAsync(t2.data(), t2d.p, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
  PTTK_CUDA(cudaStreamSynchronize(s));
  // per matrix: the resolved eigenvalues (and the positive ones for a definite kernel), listed
  // in ascending order as the inverse iteration needs; column q of matrix b's block of V
  std::vector<int> sz, scol, cnt(nb, 0);
  std::vector<double> slam, sw;
  for (int b = 0; b < nb; ++b) {
    const double* lb = lam.data() + (size_t)k * b;
    if (!(t2[b] > 0.0)) continue;  // S H T^T = 0: W_b = 0
    double lmax = 0.0;
    for (int i = 0; i < k; ++i) lmax = std::max(lmax, std::fabs(lb[i]));
    const double res = 64.0 * 2.2204460492503131e-16 * lmax;
    for (int i = 0; i < k; ++i)
      if ((!definite || lb[i] > 0.0) && std::fabs(lb[i]) > res) {
        sz.push_back(b);
        scol.push_back(cnt[b]++);
        slam.push_back(lb[i]);
        sw.push_back(std::fabs(lb[i]));
      }
  }
  int ncols = 0;
  for (int b = 0; b < nb; ++b) ncols = std::max(ncols, cnt[b]);
  PTTK_CUDA(cudaMemsetAsync(W, 0, sizeof(double) * kk * nb, s));
  if (ncols > 0) {
    DevBuf U, Ul, dl;
    PTTK_TRY(U.alloc((size_t)k * ncols * nb));
    PTTK_TRY(Ul.alloc((size_t)k * ncols));
    PTTK_TRY(dl.alloc((size_t)ncols * nb));
    {
      PTTK_PROF("global_eigvec", s);
      PTTK_TRY(sym_eig_vectors(Bb.p, dd.p, ee.p, dtau.p, k, nb, sz, slam, sw, scol, U.p, ncols, s));
    }
    std::vector<double> lk((size_t)ncols * nb, 0.0);
    for (size_t q = 0; q < sz.size(); ++q) lk[(size_t)sz[q] * ncols + scol[q]] = slam[q];
    PTTK_CUDA(cudaMemcpyAsync(dl.p, lk.data(), sizeof(double) * lk.size(), cudaMemcpyHostToDevice, s));
    for (int b = 0; b < nb; ++b) {
      const int m = cnt[b];
      if (m == 0) continue;
      const double* Ub = U.p + (size_t)k * ncols * b;
      scale_cols_kernel<<<blocks_for((int64_t)k * m, 256), 256, 0, s>>>(Ub, k, dl.p + (size_t)ncols * b, m, Ul.p);
      pttk::count_launch();
      dgemm(false, true, k, k, m, 1.0, Ul.p, k, Ub, k, 0.0, W + kk * b, k, s);
    }
    PTTK_CUDA(cudaGetLastError());
  }
  PTTK_CUDA(cudaStreamSynchronize(s));
  return PTTK_OK;
}

// ---------------- Gaussian-process likelihood on the low-rank kernel --------------------------
namespace {
// out (ra x rb, column-major) = sum_k G[:, k, :] T_k'(th) * scale (derivative of Eq. hmat's
// contraction; T_0' = 0, T_1' = 1, T_{k+1}' = 2 T_k + 2 th T_k' - T_{k-1}')
__global__ void contract_theta_deriv_kernel(const double* __restrict__ G, int ra, int n, int rb, double th,
                                            double scale, double* __restrict__ out) {
  double T[PTTK_MAX_N], dT[PTTK_MAX_N];
  T[0] = 1.0;
  dT[0] = 0.0;
  if (n > 1) {
    T[1] = th;
    dT[1] = 1.0;
  }
  for (int k = 2; k < n; ++k) {
    T[k] = 2.0 * th * T[k - 1] - T[k - 2];
    dT[k] = 2.0 * T[k - 1] + 2.0 * th * dT[k - 1] - dT[k - 2];
  }
  const int64_t total = (int64_t)ra * rb;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = e % ra, b = e / ra;
    const double* g = G + a + (int64_t)ra * n * b;
    double acc = 0.0;
    for (int k = 0; k < n; ++k) acc = fma(g[(int64_t)ra * k], dT[k], acc);
    out[e] = acc * scale;
  }
}
__global__ void contract_theta_cm_kernel(const double* __restrict__ G, int ra, int n, int rb, double th,
                                         double* __restrict__ out) {
  double T[PTTK_MAX_N];
  T[0] = 1.0;
  if (n > 1) T[1] = th;
  for (int k = 2; k < n; ++k) T[k] = 2.0 * th * T[k - 1] - T[k - 2];
  const int64_t total = (int64_t)ra * rb;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = e % ra, b = e / ra;
    const double* g = G + a + (int64_t)ra * n * b;
    double acc = 0.0;
    for (int k = 0; k < n; ++k) acc = fma(g[(int64_t)ra * k], T[k], acc);
    out[e] = acc;
  }
}
// sum_i coef[i] (U[:, i] . Y[:, i]) and the trace of A (k x k) into out[0], out[1]; one block
__global__ void __launch_bounds__(1024) coldot_trace_kernel(const double* __restrict__ U, const double* __restrict__ Y,
                                                            int k, int m, const double* __restrict__ coef,
                                                            const double* __restrict__ A, double* __restrict__ out) {
  __shared__ double sh[2][1024];
  double acc = 0.0, tr = 0.0;
  for (int64_t e = threadIdx.x; e < (int64_t)k * m; e += 1024) acc = fma(U[e] * coef[e / k], Y[e], acc);
  for (int i = threadIdx.x; i < k; i += 1024) tr += A[(int64_t)i * k + i];
  sh[0][threadIdx.x] = acc;
  sh[1][threadIdx.x] = tr;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sh[0][0];
    out[1] = sh[1][0];
  }
}
// a . b (n doubles) into *out, one block in a fixed order
__global__ void __launch_bounds__(1024) dot_block_kernel(const double* __restrict__ a, const double* __restrict__ b,
                                                         int64_t n, double* __restrict__ out) {
  __shared__ double sh[1024];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += 1024) acc = fma(a[i], b[i], acc);
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}
// out[i] = a[i] * b[i] (+ c[i] * t when c is given)
__global__ void mul_add_kernel(const double* __restrict__ a, const double* __restrict__ b, const double* __restrict__ c,
                               double t, int n, double* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = a[i] * b[i] + (c ? c[i] * t : 0.0);
}
__global__ void axpy_kernel(double t, const double* __restrict__ x, int n, double* __restrict__ y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] = fma(t, x[i], y[i]);
}
}  // namespace

// B (k x k) = sym(R_s M R_t^T) for M (rs x rt, column-major)
static pttk_status global_sym_form(const pttk_global* g, const double* M, double* P, double* C, double* B, cudaStream_t s) {
  const int k = g->k, rs = g->rs, rt = g->rt;
  dgemm(false, false, k, rt, rs, 1.0, g->R, k, M, rs, 0.0, P, k, s);
  dgemm(false, true, k, k, rt, 1.0, P, k, g->R + (size_t)k * rs, k, 0.0, C, k, s);
  sym_shift_kernel<<<blocks_for((int64_t)k * k, 256), 256, 0, s>>>(C, k, 0.0, B); pttk::count_launch();
  PTTK_CUDA(cudaGetLastError());
  return PTTK_OK;
}

// H(theta) (which < 0) or dH/dtheta_which (column-major rs x rt) of the handle's theta cores
static pttk_status global_theta_matrix(const pttk_global* g, const double* th, int which, double* out, double* work,
                                       cudaStream_t s) {
  const pttk_tt& tt = g->tt;
  const int d = tt.d, dth = tt.dtheta, n = tt.n;
  double* Hj[2] = {work, work + (size_t)tt.ranks[d] * tt.ranks[d + 1]};
  for (int j = 0; j < dth; ++j) {
    const int ra = tt.ranks[d + j], rb = tt.ranks[d + j + 1];
    double* dst = dth == 1 ? out : Hj[j];
    const unsigned blocks = blocks_for((int64_t)ra * rb, 256);
    if (j == which) {
      const double lo = tt.box[d + j][0], hi = tt.box[d + j][1];
      contract_theta_deriv_kernel<<<blocks, 256, 0, s>>>(tt.cores64 + tt.core_off[d + j], ra, n, rb, th[j],
                                                         2.0 / (lo - hi), dst); pttk::count_launch();
    } else {
      contract_theta_cm_kernel<<<blocks, 256, 0, s>>>(tt.cores64 + tt.core_off[d + j], ra, n, rb, th[j], dst); pttk::count_launch();
    }
  }
  if (dth == 2) dgemm(false, false, g->rs, g->rt, tt.ranks[d + 1], 1.0, Hj[0], g->rs, Hj[1], tt.ranks[d + 1], 0.0, out, g->rs, s);
  PTTK_CUDA(cudaGetLastError());
  return PTTK_OK;
}

static void global_release(pttk_global* g) {
  if (!g) return;
  if (g->Q) cudaFree(g->Q);
  if (g->R) cudaFree(g->R);
  if (g->tt.cores64) cudaFree(g->tt.cores64);
  delete g;
}

}  // namespace pttk

using namespace pttk;

extern "C" {

pttk_status pttk_global_create(const pttk_tt* tt, const double* X, int64_t N, void* stream, pttk_global** out) {
  clear_error();
  if (!tt || !X || !out) return set_error(PTTK_EINVAL, "NULL argument");
  *out = nullptr;
  if (N < 1) return set_error(PTTK_EINVAL, "PTTK-Global needs at least one point");
  const int d = tt->d, dth = tt->dtheta;
  for (int i = 0; i < d; ++i)
    if (tt->box[i][0] != tt->box[d + dth + i][0] || tt->box[i][1] != tt->box[d + dth + i][1])
      return set_error(PTTK_EINVAL, "PTTK-Global needs the source box equal to the target box");
  pttk_global* g = new pttk_global();
  g->tt = *tt;  // metadata; the core pointers are replaced by the handle's own copy
  g->tt.cores64 = nullptr;
  g->tt.cores32 = nullptr;
  const pttk_status st = global_create_run(tt, X, N, g, as_stream(stream));
  if (st != PTTK_OK) {
    global_release(g);
    return st;
  }
  *out = g;
  return PTTK_OK;
}

pttk_status pttk_global_dims(const pttk_global* g, int64_t* N, int* k, int* r_s, int* r_t) {
  clear_error();
  if (!g) return set_error(PTTK_EINVAL, "NULL handle");
  if (N) *N = g->N;
  if (k) *k = g->k;
  if (r_s) *r_s = g->rs;
  if (r_t) *r_t = g->rt;
  return PTTK_OK;
}

pttk_status pttk_global_get_q(const pttk_global* g, double* Q, void* stream) {
  clear_error();
  if (!g || !Q) return set_error(PTTK_EINVAL, "NULL argument");
  PTTK_CUDA(cudaMemcpyAsync(Q, g->Q, sizeof(double) * (size_t)g->N * g->k, cudaMemcpyDeviceToDevice,
                            as_stream(stream)));
  return PTTK_OK;
}

pttk_status pttk_global_get_r(const pttk_global* g, double* R_host) {
  clear_error();
  if (!g || !R_host) return set_error(PTTK_EINVAL, "NULL argument");
  PTTK_CUDA(cudaMemcpy(R_host, g->R, sizeof(double) * (size_t)g->k * (g->rs + g->rt), cudaMemcpyDeviceToHost));
  return PTTK_OK;
}

pttk_status pttk_global_instantiate(const pttk_global* g, const double* theta, double eps, int compress,
                                    int definite, double* Z, double* W, int* rank, void* stream) {
  clear_error();
  if (!g || !W || !rank) return set_error(PTTK_EINVAL, "NULL argument");
  if (compress && !Z) return set_error(PTTK_EINVAL, "PTTK-Global-2 needs the Z buffer");
  if (!(eps >= 0.0) || !(eps < 1.0)) return set_error(PTTK_EINVAL, "eps must be in [0, 1)");
  double th[PTTK_MAX_D];
  PTTK_TRY(theta_hat(&g->tt, theta, th));
  return global_online_run(g, th, eps, compress != 0, definite != 0, Z, W, rank, as_stream(stream));
}

pttk_status pttk_global_instantiate_batched(const pttk_global* g, int B, const double* thetas, int definite,
                                            double* W, void* stream) {
  clear_error();
  if (!g || (B > 0 && (!thetas || !W))) return set_error(PTTK_EINVAL, "NULL argument");
  if (B < 0) return set_error(PTTK_EINVAL, "B must be >= 0");
  if (B == 0) return PTTK_OK;
  const int dth = g->tt.dtheta;
  std::vector<double> th((size_t)B * PTTK_MAX_D, 0.0);
  for (int b = 0; b < B; ++b) PTTK_TRY(theta_hat(&g->tt, thetas + (size_t)b * dth, th.data() + (size_t)b * PTTK_MAX_D));
  return global_online_batched_run(g, th.data(), B, definite != 0, W, as_stream(stream));
}

void pttk_global_free(pttk_global* g) { global_release(g); }

pttk_status pttk_gp_lml(const pttk_global* g, const double* theta, double s2, const double* y, double* lml,
                        double* grad, void* stream) {
  clear_error();
  if (!g || !y || !lml) return set_error(PTTK_EINVAL, "NULL argument");
  if (!(s2 > 0.0)) return set_error(PTTK_EINVAL, "the noise variance s2 must be positive");
  const int dth = g->tt.dtheta;
  if (dth < 1 || dth > 2) return set_error(PTTK_ENOTSUP, "the likelihood needs a kernel with 1 or 2 parameters");
  double th[PTTK_MAX_D];
  PTTK_TRY(theta_hat(&g->tt, theta, th));
  cudaStream_t s = as_stream(stream);
  const int k = g->k, rs = g->rs, rt = g->rt;
  const int64_t N = g->N;
  const pttk_tt& tt = g->tt;
  const size_t hwork = (size_t)tt.ranks[tt.d] * tt.ranks[tt.d + 1] + (size_t)tt.ranks[tt.d + 1] * tt.ranks[tt.d + dth];
  DevBuf c, Mbuf, work, P, C, B, Bw, dB, dd, ee, tau, lamd, sc;
  PTTK_TRY(c.alloc(k));
  PTTK_TRY(Mbuf.alloc((size_t)rs * rt));
  PTTK_TRY(work.alloc(hwork));
  PTTK_TRY(P.alloc((size_t)k * rt));
  PTTK_TRY(C.alloc((size_t)k * k));
  PTTK_TRY(B.alloc((size_t)k * k));
  PTTK_TRY(Bw.alloc((size_t)k * k));
  PTTK_TRY(dB.alloc((size_t)dth * k * k));
  PTTK_TRY(dd.alloc(k));
  PTTK_TRY(ee.alloc(k));
  PTTK_TRY(tau.alloc(k));
  PTTK_TRY(lamd.alloc(k));
  PTTK_TRY(sc.alloc(8));
  // c = Q^T y (Q row-major N x k = column-major k x N), ||y||^2, ||c||^2
  dgemm(false, false, k, 1, N, 1.0, g->Q, k, y, N, 0.0, c.p, k, s);
  dot_block_kernel<<<1, 1024, 0, s>>>(y, y, N, sc.p); pttk::count_launch();
  dot_block_kernel<<<1, 1024, 0, s>>>(c.p, c.p, k, sc.p + 1); pttk::count_launch();
  // B = sym(R_s H R_t^T) and dB_j = sym(R_s dH_j R_t^T)
  PTTK_TRY(global_theta_matrix(g, th, -1, Mbuf.p, work.p, s));
  PTTK_TRY(global_sym_form(g, Mbuf.p, P.p, C.p, B.p, s));
  for (int j = 0; j < dth; ++j) {
    PTTK_TRY(global_theta_matrix(g, th, j, Mbuf.p, work.p, s));
    PTTK_TRY(global_sym_form(g, Mbuf.p, P.p, C.p, dB.p + (size_t)j * k * k, s));
  }
  PTTK_CUDA(cudaMemcpyAsync(Bw.p, B.p, sizeof(double) * (size_t)k * k, cudaMemcpyDeviceToDevice, s));
  {
    PTTK_PROF("global_eig", s);
    PTTK_TRY(sym_eig_values(Bw.p, k, 1, dd.p, ee.p, tau.p, lamd.p, s));
  }
  std::vector<double> lam(k);
  double yy_cc[2];
  PTTK_CUDA(cudaMemcpyAsync(lam.data(), lamd.p, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
  PTTK_CUDA(cudaMemcpyAsync(yy_cc, sc.p, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
  PTTK_CUDA(cudaStreamSynchronize(s));
  double lmax = 0.0, logdet = (double)(N - k) * std::log(s2);
  for (int i = 0; i < k; ++i) {
    lmax = std::max(lmax, std::fabs(lam[i]));
    if (!(lam[i] + s2 > 0.0))
      return set_error(PTTK_EDOMAIN, "the low-rank kernel plus s2 I is not positive definite at this theta");
    logdet += std::log(lam[i] + s2);
  }
  // eigenvectors of the resolved eigenvalues; the others count as zero, their eigenspace
  // entering only through the 1/s2 terms below
  const double res = 64.0 * 2.2204460492503131e-16 * lmax;
  std::vector<int> sz, scol;
  std::vector<double> slam, coef, sw;
  for (int i = 0; i < k; ++i)
    if (std::fabs(lam[i]) > res) {
      sz.push_back(0);
      scol.push_back((int)slam.size());
      slam.push_back(lam[i]);
      coef.push_back(1.0 / (lam[i] + s2) - 1.0 / s2);
      // the spectral function here is coef(lambda) = -lambda / (s2 (lambda + s2)); its weight on
      // the scale of lambda is |coef| s2^2 = |lambda| s2 / (lambda + s2), about min(|lambda|, s2)
      sw.push_back(std::fabs(lam[i]) * s2 / (lam[i] + s2));
    }
  const int m = (int)slam.size();
  DevBuf U, Y, w, alpha, coefd, v;
  PTTK_TRY(U.alloc((size_t)k * std::max(m, 1)));
  PTTK_TRY(Y.alloc((size_t)k * std::max(m, 1)));
  PTTK_TRY(w.alloc(std::max(m, 1)));
  PTTK_TRY(alpha.alloc(k));
  PTTK_TRY(coefd.alloc(std::max(m, 1)));
  PTTK_TRY(v.alloc(k));
  if (m > 0) {
    PTTK_PROF("global_eigvec", s);
    PTTK_TRY(sym_eig_vectors(Bw.p, dd.p, ee.p, tau.p, k, 1, sz, slam, sw, scol, U.p, m, s));
    PTTK_CUDA(cudaMemcpyAsync(coefd.p, coef.data(), sizeof(double) * m, cudaMemcpyHostToDevice, s));
  }
  // alpha~ = (B + s2 I)^{-1} c = U ((1/(lambda + s2) - 1/s2) .* (U^T c)) + c / s2
  PTTK_CUDA(cudaMemsetAsync(v.p, 0, sizeof(double) * k, s));
  if (m > 0) {
    dgemm(true, false, m, 1, k, 1.0, U.p, k, c.p, k, 0.0, w.p, m, s);
    mul_add_kernel<<<(m + 255) / 256, 256, 0, s>>>(w.p, coefd.p, nullptr, 0.0, m, w.p); pttk::count_launch();
    dgemm(false, false, k, 1, m, 1.0, U.p, k, w.p, m, 0.0, v.p, k, s);
  }
  // alpha = v + c / s2
  PTTK_CUDA(cudaMemcpyAsync(alpha.p, v.p, sizeof(double) * k, cudaMemcpyDeviceToDevice, s));
  axpy_kernel<<<(k + 255) / 256, 256, 0, s>>>(1.0 / s2, c.p, k, alpha.p); pttk::count_launch();
  dot_block_kernel<<<1, 1024, 0, s>>>(c.p, alpha.p, k, sc.p + 2); pttk::count_launch();
  // per parameter: alpha~^T dB alpha~ and tr((B + s2 I)^{-1} dB)
  //   = sum_i (u_i^T dB u_i)(1/(lambda_i + s2) - 1/s2) + tr(dB) / s2
  std::vector<double> g_quad(dth), g_tr(dth);
  for (int j = 0; j < dth; ++j) {
    const double* dBj = dB.p + (size_t)j * k * k;
    dgemm(false, false, k, 1, k, 1.0, dBj, k, alpha.p, k, 0.0, v.p, k, s);
    dot_block_kernel<<<1, 1024, 0, s>>>(alpha.p, v.p, k, sc.p + 3); pttk::count_launch();
    if (m > 0) dgemm(false, false, k, m, k, 1.0, dBj, k, U.p, k, 0.0, Y.p, k, s);
    coldot_trace_kernel<<<1, 1024, 0, s>>>(U.p, Y.p, k, m, coefd.p, dBj, sc.p + 4); pttk::count_launch();
    PTTK_CUDA(cudaGetLastError());
    double h3[3];
    PTTK_CUDA(cudaMemcpyAsync(h3, sc.p + 3, sizeof(double) * 3, cudaMemcpyDeviceToHost, s));
    PTTK_CUDA(cudaStreamSynchronize(s));
    g_quad[j] = h3[0];
    g_tr[j] = (m > 0 ? h3[1] : 0.0) + h3[2] / s2;
  }
  double cq = 0.0;
  PTTK_CUDA(cudaMemcpyAsync(&cq, sc.p + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
  PTTK_CUDA(cudaStreamSynchronize(s));
  // y^T (K~ + s2 I)^{-1} y = c^T alpha~ + (||y||^2 - ||c||^2) / s2
  const double quad = cq + (yy_cc[0] - yy_cc[1]) / s2;
  *lml = -0.5 * quad - 0.5 * logdet - 0.5 * (double)N * std::log(2.0 * 3.141592653589793);
  if (grad)
    for (int j = 0; j < dth; ++j) grad[j] = 0.5 * (g_quad[j] - g_tr[j]);
  return PTTK_OK;
}

}  // extern "C"

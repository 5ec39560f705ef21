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
// (Eq. pttk1: H^ = [[0, H/2], [H^T/2, 0]], R = [R_s R_t]); its eigendecomposition by one-sided
// Jacobi on sym(C1) + c I with c = 2 ||C1||_F. That matrix is symmetric positive definite (its
// eigenvalues lie in [c/2, 3c/2]), so its left singular vectors are the eigenvectors of
// sym(C1) and its singular values are the eigenvalues plus c.
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

// norms[c] = ||A[:, c]||_2 (rows x ncols, column-major), one warp per column
__global__ void col_norms_kernel(const double* __restrict__ A, int64_t rows, int ncols,
                                 double* __restrict__ norms) {
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= ncols) return;
  const double* col = A + gw * rows;
  double acc = 0.0;
  for (int64_t i = lane; i < rows; i += 32) acc = fma(col[i], col[i], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) norms[gw] = sqrt(acc);
}

// out[:, q] = A[:, idx[q]] * (scale[q] / norms[idx[q]]), rows x m column-major; idx, scale
// packed as sel[0..m) = idx (as doubles), sel[m..2m) = scale
__global__ void pick_cols_kernel(const double* __restrict__ A, int64_t rows,
                                 const double* __restrict__ sel, int m,
                                 const double* __restrict__ norms, double* __restrict__ out) {
  const int64_t total = rows * m;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % rows;
    const int q = (int)(e / rows);
    const int src = (int)sel[q];
    const double nr = norms[src];
    out[e] = nr > 0.0 ? A[i + (int64_t)src * rows] * (sel[m + q] / nr) : 0.0;
  }
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
  DevBuf H, P, C1, B, nrm, t2d;
  PTTK_TRY(H.alloc((size_t)rs * rt));
  PTTK_TRY(P.alloc((size_t)k * rt));
  PTTK_TRY(C1.alloc((size_t)k * k));
  PTTK_TRY(B.alloc((size_t)k * k));
  PTTK_TRY(nrm.alloc(k));
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
  const double shift = 2.0 * sqrt(t2);
  sym_shift_kernel<<<blocks_for((int64_t)k * k, 256), 256, 0, s>>>(C1.p, k, shift, B.p); pttk::count_launch();
  PTTK_CUDA(cudaGetLastError());
  {
    PTTK_PROF("global_eig", s);
    PTTK_TRY(jacobi_columns(B.p, k, k, s));
  }
  col_norms_kernel<<<(unsigned)(((int64_t)k * 32 + 255) / 256), 256, 0, s>>>(B.p, k, k, nrm.p); pttk::count_launch();
  PTTK_CUDA(cudaGetLastError());
  std::vector<double> sigma(k);
  PTTK_CUDA(cudaMemcpyAsync(sigma.data(), nrm.p, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
  PTTK_CUDA(cudaStreamSynchronize(s));
  // eigenvalues, in decreasing |lambda|; a definite kernel drops the negative ones
  std::vector<double> lam(k);
  for (int i = 0; i < k; ++i) lam[i] = sigma[i] - shift;
  std::vector<int> order(k);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return std::fabs(lam[a]) > std::fabs(lam[b]); });
  std::vector<int> kept;
  for (int i : order)
    if (!definite || lam[i] > 0.0) kept.push_back(i);
  int m = (int)kept.size();
  if (compress) {
    // ||Q U_j Lambda_j U_j^T Q^T - S H T^T||_F^2 = ||C1 - U_j Lambda_j U_j^T||_F^2
    //   = ||(C1 - C1^T)/2||_F^2 + (sum of lambda_i^2 over the eigenpairs not kept),
    // the symmetric and antisymmetric parts being orthogonal. Summed from the discarded terms
    // themselves: ||C1||^2 - (sum of the kept lambda^2) would cancel, and the eigenvalues carry
    // an absolute error of order 1e-14 ||C1||_F (they are singular values of sym(C1) + c I,
    // minus c), which in the large kept terms alone exceeds eps^2 ||C1||^2 for eps <= 1e-6.
    const double bound2 = eps * eps * t2;
    double excl2 = 0.0;  // eigenvalues not eligible: the negative ones of a definite kernel
    if (definite)
      for (int i = 0; i < k; ++i)
        if (!(lam[i] > 0.0)) excl2 += lam[i] * lam[i];
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
  // selection table: column index, then the scale of each picked column
  std::vector<double> sel(2 * (size_t)m);
  DevBuf dsel, Un, Ul, dlam;
  PTTK_TRY(dsel.alloc(2 * (size_t)m));
  PTTK_TRY(Un.alloc((size_t)k * m));
  for (int q = 0; q < m; ++q) {
    sel[q] = kept[q];
    sel[m + q] = 1.0;
  }
  PTTK_CUDA(cudaMemcpyAsync(dsel.p, sel.data(), sizeof(double) * 2 * m, cudaMemcpyHostToDevice, s));
  pick_cols_kernel<<<blocks_for((int64_t)k * m, 256), 256, 0, s>>>(B.p, k, dsel.p, m, nrm.p, Un.p); pttk::count_launch();
  PTTK_CUDA(cudaGetLastError());
  if (!compress) {
    // W = U Lambda U^T (k x k)
    PTTK_CUDA(cudaStreamSynchronize(s));  // sel is rewritten below
    for (int q = 0; q < m; ++q) sel[m + q] = lam[kept[q]];
    PTTK_TRY(Ul.alloc((size_t)k * m));
    PTTK_CUDA(cudaMemcpyAsync(dsel.p, sel.data(), sizeof(double) * 2 * m, cudaMemcpyHostToDevice, s));
    pick_cols_kernel<<<blocks_for((int64_t)k * m, 256), 256, 0, s>>>(B.p, k, dsel.p, m, nrm.p, Ul.p); pttk::count_launch();
    PTTK_CUDA(cudaGetLastError());
    dgemm(false, true, k, k, m, 1.0, Ul.p, k, Un.p, k, 0.0, W, k, s);
  } else {
    // Z = Q U^ (N x m row-major): Z^T (m x N column-major) = U^T Q^T, Q^T being Q row-major
    {
      PTTK_PROF("global_z", s);
      dgemm(true, false, m, N, k, 1.0, Un.p, k, g->Q, k, 0.0, Z, m, s);
    }
    std::vector<double> lk(m);
    for (int q = 0; q < m; ++q) lk[q] = lam[kept[q]];
    PTTK_TRY(dlam.alloc(m));
    PTTK_CUDA(cudaMemcpyAsync(dlam.p, lk.data(), sizeof(double) * m, cudaMemcpyHostToDevice, s));
    diag_kernel<<<blocks_for((int64_t)m * m, 256), 256, 0, s>>>(dlam.p, m, W); pttk::count_launch();
    PTTK_CUDA(cudaGetLastError());
  }
  PTTK_CUDA(cudaStreamSynchronize(s));
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

void pttk_global_free(pttk_global* g) { global_release(g); }

}  // extern "C"

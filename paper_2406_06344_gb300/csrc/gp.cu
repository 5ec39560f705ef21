// The Gaussian-process workload that Section 1 names as a use of the parametric low-rank
// form: solving (K(X, X; theta) + s2 I) x = b by conjugate gradients preconditioned with the
// PTTK-Global factorisation (Algorithm 4), with the kernel matrix applied exactly.
//
//   pttk_gp_kv   out = (K(X, X; theta) + s2 I) v, every kernel entry evaluated on the fly
//                (tiles of the points in shared memory; N^2 evaluations, no N x N storage), in
//                FP64, or in FP32 with each tile's 128 terms summed in FP32 and the tile sums
//                in FP64. Rows and column ranges are split over blocks so that small N fills
//                the GPU; the column ranges' partial sums are added in a fixed order.
//   pttk_gp_pcg  preconditioned CG (Hestenes-Stiefel) with M^{-1} = (Z W Z^T + s2 I)^{-1},
//                Z (N x m) with orthonormal columns and W = diag(lambda) (PTTK-Global-2, or
//                Global-1 written in its eigenbasis), applied in Woodbury form
//                M^{-1} v = Z ((Z^T v) ./ (lambda + s2)) + (v - Z Z^T v) / s2.
//                Stops when ||b - A x_j||_2 <= tol ||b||_2, the residual being the recursively
//                updated one.
#include <cmath>
#include <vector>

#include "kernels.cuh"
#include "pttk_internal.cuh"

namespace pttk {
namespace {

constexpr int GT = 256;       // threads per block
constexpr int GTILE = 128;    // columns per shared-memory tile of the kernel product

// part[cs * N + i] = sum over the columns j of range cs of kappa(||x_i - x_j||^2; l) v[j]:
// block (x, y) takes rows [x GT, x GT + GT) and column range y of gridDim.y, ranges of
// `cols` columns (a multiple of GTILE). T: the precision of the evaluation and of each tile's
// sum; the tile sums are added in FP64.
template <typename T>
__global__ void __launch_bounds__(GT) gp_kv_kernel(int kind, int d, const double* __restrict__ X, int64_t N, double l,
                                                   const double* __restrict__ v, int64_t cols,
                                                   double* __restrict__ part) {
  __shared__ T xs[GTILE * PTTK_MAX_D];
  __shared__ T vs[GTILE];
  const int64_t i = (int64_t)blockIdx.x * GT + threadIdx.x;
  const int64_t c0 = (int64_t)blockIdx.y * cols, c1 = std::min<int64_t>(N, c0 + cols);
  T xi[PTTK_MAX_D];
  for (int c = 0; c < d; ++c) xi[c] = i < N ? (T)X[i * d + c] : T(0);
  const T lt = (T)l;
  double acc = 0.0;
  for (int64_t t0 = c0; t0 < c1; t0 += GTILE) {
    const int nt = (int)std::min<int64_t>(GTILE, c1 - t0);
    __syncthreads();
    for (int q = threadIdx.x; q < nt * d; q += GT) xs[q] = (T)X[t0 * d + q];
    for (int q = threadIdx.x; q < nt; q += GT) vs[q] = (T)v[t0 + q];
    __syncthreads();
    if (i < N) {
      T tacc = T(0);
      for (int jj = 0; jj < nt; ++jj) {
        T r2 = T(0);
        for (int c = 0; c < d; ++c) {
          const T df = xi[c] - xs[jj * d + c];
          r2 = fma(df, df, r2);
        }
        tacc = fma(kappa_l<T>(kind, r2, lt), vs[jj], tacc);
      }
      acc += (double)tacc;
    }
  }
  if (i < N) part[(int64_t)blockIdx.y * N + i] = acc;
}

// out[i] = s2 v[i] + sum over the column ranges of part (in order)
__global__ void gp_kv_reduce(const double* __restrict__ part, int ncs, int64_t N, double s2,
                             const double* __restrict__ v, double* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int c = 0; c < ncs; ++c) acc += part[(int64_t)c * N + i];
    out[i] = fma(s2, v[i], acc);
  }
}

// partial[b * m + c] = sum over the block's rows p of Z[p, c] v[p] (Z: N x m row-major)
__global__ void __launch_bounds__(GT) gemv_t_partial(const double* __restrict__ Z, int64_t N, int m,
                                                     const double* __restrict__ v, double* __restrict__ partial) {
  const int64_t per = (N + gridDim.x - 1) / gridDim.x;
  const int64_t p0 = (int64_t)blockIdx.x * per, p1 = std::min<int64_t>(N, p0 + per);
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    double acc = 0.0;
    for (int64_t p = p0; p < p1; ++p) acc = fma(Z[p * m + c], v[p], acc);
    partial[(int64_t)blockIdx.x * m + c] = acc;
  }
}

// coef[c] = (sum_b partial[b * m + c]) * (1 / (lambda_c + s2) - 1 / s2)
__global__ void precond_coef(const double* __restrict__ partial, int nparts, int m, const double* __restrict__ lam,
                             double s2, double* __restrict__ coef) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int b = 0; b < nparts; ++b) acc += partial[(int64_t)b * m + c];
    coef[c] = acc * (1.0 / (lam[c] + s2) - 1.0 / s2);
  }
}

// z[p] = sum_c Z[p, c] coef[c] + r[p] / s2, one warp per row
__global__ void __launch_bounds__(GT) precond_apply(const double* __restrict__ Z, int64_t N, int m,
                                                    const double* __restrict__ coef, const double* __restrict__ r,
                                                    double s2, double* __restrict__ z) {
  const int lane = threadIdx.x & 31;
  for (int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < N;
       p += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    double acc = 0.0;
    for (int c = lane; c < m; c += 32) acc = fma(Z[p * m + c], coef[c], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) z[p] = acc + r[p] / s2;
  }
}

// per-block partial dot products of (a, b), grid-stride; out[blockIdx.x]
__global__ void __launch_bounds__(GT) dot_partial(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                                                  double* __restrict__ out) {
  __shared__ double sh[GT / 32];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc = fma(a[i], b[i], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < GT / 32; ++w) t += sh[w];
    out[blockIdx.x] = t;
  }
}

// x += alpha p; r -= alpha Ap (alpha = num / den read on the device)
__global__ void cg_update_xr(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                             const double* __restrict__ Ap, int64_t n, double alpha) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    r[i] = fma(-alpha, Ap[i], r[i]);
  }
}

// p = z + beta p
__global__ void cg_update_p(double* __restrict__ p, const double* __restrict__ z, int64_t n, double beta) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i], z[i]);
}

bool gp_kernel_ok(int kind) {
  return kind == PTTK_GAUSS || kind == PTTK_MATERN32 || kind == PTTK_EXPONENTIAL || kind == PTTK_MATERN52;
}

struct GpScratch {
  std::vector<double*> bufs;
  ~GpScratch() {
    for (double* p : bufs)
      if (p) cudaFree(p);
  }
  pttk_status get(double** out, size_t n) {
    double* p = nullptr;
    PTTK_CUDA(cudaMalloc(&p, sizeof(double) * std::max<size_t>(n, 1)));
    bufs.push_back(p);
    *out = p;
    return PTTK_OK;
  }
};

unsigned grid_for(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + GT - 1) / GT, (int64_t)sm_count() * 8));
}

// column ranges of the kernel product: enough blocks for about four per SM
int kv_splits(int64_t N) {
  const int64_t row_tiles = (N + GT - 1) / GT;
  const int64_t want = std::max<int64_t>(1, (int64_t)sm_count() * 4 / std::max<int64_t>(row_tiles, 1));
  return (int)std::min<int64_t>({want, 64, (N + GTILE - 1) / GTILE});
}

// out = (K + s2 I) v; part: scratch of kv_splits(N) * N doubles
pttk_status kv_launch(int kind, int d, const double* X, int64_t N, double l, double s2, const double* v, double* out,
                      bool fp32, double* part, cudaStream_t s) {
  PTTK_PROF("gp_kv", s);
  const int ncs = kv_splits(N);
  const int64_t cols = ((N + ncs - 1) / ncs + GTILE - 1) / GTILE * GTILE;
  const dim3 grid((unsigned)((N + GT - 1) / GT), (unsigned)ncs);
  if (fp32) gp_kv_kernel<float><<<grid, GT, 0, s>>>(kind, d, X, N, l, v, cols, part);
  else gp_kv_kernel<double><<<grid, GT, 0, s>>>(kind, d, X, N, l, v, cols, part);
  pttk::count_launch();
  gp_kv_reduce<<<grid_for(N), GT, 0, s>>>(part, ncs, N, s2, v, out); pttk::count_launch();
  PTTK_CUDA(cudaGetLastError());
  return PTTK_OK;
}

// a . b into *host, synchronising s
pttk_status dot_host(const double* a, const double* b, int64_t n, double* part, int nparts, double* host,
                     cudaStream_t s) {
  dot_partial<<<nparts, GT, 0, s>>>(a, b, n, part); pttk::count_launch();
  PTTK_CUDA(cudaGetLastError());
  std::vector<double> h(nparts);
  PTTK_CUDA(cudaMemcpyAsync(h.data(), part, sizeof(double) * nparts, cudaMemcpyDeviceToHost, s));
  PTTK_CUDA(cudaStreamSynchronize(s));
  double t = 0.0;
  for (double q : h) t += q;
  *host = t;
  return PTTK_OK;
}

pttk_status check_gp(int kernel, int d, const double* X, int64_t N, const double* theta, double s2) {
  if (!X || !theta) return set_error(PTTK_EINVAL, "NULL argument");
  if (!gp_kernel_ok(kernel))
    return set_error(PTTK_EINVAL, "GP kernels: Gaussian, Matern-3/2, Exponential or Matern-5/2 (theta = l)");
  if (d < 1 || d > PTTK_MAX_D) return set_error(PTTK_EINVAL, "bad d");
  if (N < 1) return set_error(PTTK_EINVAL, "no points");
  if (!(theta[0] > 0.0)) return set_error(PTTK_EINVAL, "the length scale must be positive");
  if (!(s2 > 0.0)) return set_error(PTTK_EINVAL, "the noise variance s2 must be positive");
  return PTTK_OK;
}

}  // namespace
}  // namespace pttk

using namespace pttk;

extern "C" {

pttk_status pttk_gp_kv(int kernel, int d, const double* X, int64_t N, const double* theta, double s2, const double* v,
                       double* out, pttk_prec prec, void* stream) {
  clear_error();
  PTTK_TRY(check_gp(kernel, d, X, N, theta, s2));
  if (!v || !out) return set_error(PTTK_EINVAL, "NULL argument");
  if (prec != PTTK_FP64 && prec != PTTK_FP32) return set_error(PTTK_EINVAL, "K v: prec must be PTTK_FP64 or PTTK_FP32");
  cudaStream_t s = as_stream(stream);
  double* part = nullptr;
  PTTK_CUDA(cudaMallocAsync(&part, sizeof(double) * (size_t)kv_splits(N) * N, s));
  const pttk_status st = kv_launch(kernel, d, X, N, theta[0], s2, v, out, prec == PTTK_FP32, part, s);
  cudaFreeAsync(part, s);
  return st;
}

pttk_status pttk_gp_pcg(int kernel, int d, const double* X, int64_t N, const double* theta, double s2, const double* Z,
                        const double* lam, int m, const double* b, double* x, double tol, int maxit, pttk_prec prec,
                        int* iters, double* resid, void* stream) {
  clear_error();
  PTTK_TRY(check_gp(kernel, d, X, N, theta, s2));
  if (prec != PTTK_FP64 && prec != PTTK_FP32) return set_error(PTTK_EINVAL, "PCG: prec must be PTTK_FP64 or PTTK_FP32");
  if (!b || !x) return set_error(PTTK_EINVAL, "NULL argument");
  if (m < 0 || (m > 0 && (!Z || !lam))) return set_error(PTTK_EINVAL, "preconditioner: m >= 0 and Z, lambda given");
  if (!(tol > 0.0) || maxit < 0) return set_error(PTTK_EINVAL, "tol > 0 and maxit >= 0 required");
  cudaStream_t s = as_stream(stream);
  const double l = theta[0];
  GpScratch sc;
  double *r, *z, *p, *Ap, *part, *coef = nullptr, *gpart = nullptr;
  const int nparts = (int)std::min<int64_t>((N + GT - 1) / GT, (int64_t)sm_count() * 4);
  const int gparts = (int)std::max<int64_t>(1, std::min<int64_t>((N + 1023) / 1024, (int64_t)sm_count() * 4));
  PTTK_TRY(sc.get(&r, N));
  PTTK_TRY(sc.get(&z, N));
  PTTK_TRY(sc.get(&p, N));
  PTTK_TRY(sc.get(&Ap, N));
  PTTK_TRY(sc.get(&part, nparts));
  double* kvpart = nullptr;
  PTTK_TRY(sc.get(&kvpart, (size_t)kv_splits(N) * N));
  if (m > 0) {
    PTTK_TRY(sc.get(&coef, m));
    PTTK_TRY(sc.get(&gpart, (size_t)gparts * m));
  }
  auto precond = [&](const double* in, double* outv) -> pttk_status {
    if (m == 0) {
      PTTK_CUDA(cudaMemcpyAsync(outv, in, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
      return PTTK_OK;
    }
    gemv_t_partial<<<gparts, GT, 0, s>>>(Z, N, m, in, gpart); pttk::count_launch();
    precond_coef<<<(m + GT - 1) / GT, GT, 0, s>>>(gpart, gparts, m, lam, s2, coef); pttk::count_launch();
    precond_apply<<<grid_for(N * 32), GT, 0, s>>>(Z, N, m, coef, in, s2, outv); pttk::count_launch();
    PTTK_CUDA(cudaGetLastError());
    return PTTK_OK;
  };
  // x0 = 0, r0 = b
  PTTK_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * N, s));
  PTTK_CUDA(cudaMemcpyAsync(r, b, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
  double bn2 = 0.0;
  PTTK_TRY(dot_host(b, b, N, part, nparts, &bn2, s));
  const double bn = std::sqrt(bn2);
  PTTK_TRY(precond(r, z));
  PTTK_CUDA(cudaMemcpyAsync(p, z, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
  double rz = 0.0;
  PTTK_TRY(dot_host(r, z, N, part, nparts, &rz, s));
  double rn = bn;
  int it = 0;
  while (rn > tol * bn && it < maxit) {
    PTTK_TRY(kv_launch(kernel, d, X, N, l, s2, p, Ap, prec == PTTK_FP32, kvpart, s));
    double pAp = 0.0;
    PTTK_TRY(dot_host(p, Ap, N, part, nparts, &pAp, s));
    if (!(pAp > 0.0)) return set_error(PTTK_EDOMAIN, "CG: p^T A p <= 0 (the matrix is not positive definite)");
    const double alpha = rz / pAp;
    cg_update_xr<<<grid_for(N), GT, 0, s>>>(x, r, p, Ap, N, alpha); pttk::count_launch();
    double rr = 0.0;
    PTTK_TRY(dot_host(r, r, N, part, nparts, &rr, s));
    rn = std::sqrt(rr);
    ++it;
    if (!(rn > tol * bn)) break;
    PTTK_TRY(precond(r, z));
    double rz_new = 0.0;
    PTTK_TRY(dot_host(r, z, N, part, nparts, &rz_new, s));
    cg_update_p<<<grid_for(N), GT, 0, s>>>(p, z, N, rz_new / rz); pttk::count_launch();
    rz = rz_new;
  }
  PTTK_CUDA(cudaGetLastError());
  PTTK_CUDA(cudaStreamSynchronize(s));
  if (iters) *iters = it;
  if (resid) *resid = bn > 0.0 ? rn / bn : 0.0;
  return PTTK_OK;
}

}  // extern "C"

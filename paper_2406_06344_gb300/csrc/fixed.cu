// Algorithm 2 for fixed point sets: Phase 3 (the factor matrices S = U(X), T = V(Y) by the
// FP64 factor chains) and Phase 4 (TT-Round of the twisted TT [T^(1)(S), G_{d+1}, ..,
// G_{d+d_theta}, T^(3)(T^T)] of Eq. twist at the offline tolerance), then the online stage of
// Algorithm 3 on the rounded theta cores. The handle keeps S', T' and the rounded theta cores in
// FP64 on the device; K(X, Y; theta) ~= S' H'(theta) T'^T.
#include <cstring>
#include <vector>

#include "pttk_internal.cuh"

namespace pttk {
pttk_status phase4_round(const double* Scol, int64_t Ns, const double* const* theta_cores, const int* ranks, int n,
                         int dtheta, const double* Tt, int64_t Nt, double tol, double** out, int* new_ranks,
                         cudaStream_t s);
namespace {

// out (cols x rows, row-major) = the transpose of in (rows x cols, row-major); 32 x 32 tiles
// through shared memory, grid-stride over the tiles in both directions
__global__ void transpose_rm_kernel(const double* __restrict__ in, int64_t rows, int64_t cols, double* __restrict__ out) {
  __shared__ double tile[32][33];
  const int64_t nbr = (rows + 31) / 32, nbc = (cols + 31) / 32;
  for (int64_t by = blockIdx.y; by < nbr; by += gridDim.y)
    for (int64_t bx = blockIdx.x; bx < nbc; bx += gridDim.x) {
      const int64_t r0 = by * 32, c0 = bx * 32;
      for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t r = r0 + i, c = c0 + threadIdx.x;
        tile[i][threadIdx.x] = (r < rows && c < cols) ? in[r * cols + c] : 0.0;
      }
      __syncthreads();
      for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t c = c0 + i, r = r0 + threadIdx.x;
        if (c < cols && r < rows) out[c * rows + r] = tile[threadIdx.x][i];
      }
      __syncthreads();
    }
}

pttk_status transpose_rm(const double* in, int64_t rows, int64_t cols, double* out, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return PTTK_OK;
  const dim3 grid((unsigned)std::min<int64_t>((cols + 31) / 32, 4096), (unsigned)std::min<int64_t>((rows + 31) / 32, 4096));
  transpose_rm_kernel<<<grid, dim3(32, 8), 0, s>>>(in, rows, cols, out); pttk::count_launch();
  PTTK_CUDA(cudaGetLastError());
  return PTTK_OK;
}

}  // namespace
}  // namespace pttk

struct pttk_fixed {
  pttk_tt th;               // the rounded theta cores as a d = 0 handle (for Algorithm 3)
  int64_t Ns = 0, Nt = 0;
  double* S = nullptr;      // N_s x r_s', row-major
  double* T = nullptr;      // N_t x r_t', row-major
};

using namespace pttk;

static void fixed_release(pttk_fixed* f) {
  if (!f) return;
  if (f->S) cudaFree(f->S);
  if (f->T) cudaFree(f->T);
  if (f->th.cores64) cudaFree(f->th.cores64);
  if (f->th.cores32) cudaFree(f->th.cores32);
  delete f;
}

extern "C" {

pttk_status pttk_fixed_create(const pttk_tt* tt, const double* X, int64_t N_s, const double* Y, int64_t N_t,
                              double tol, void* stream, pttk_fixed** out) {
  clear_error();
  if (!out) return set_error(PTTK_EINVAL, "NULL out");
  *out = nullptr;
  if (!tt || !X || !Y) return set_error(PTTK_EINVAL, "NULL argument");
  if (N_s < 1 || N_t < 1) return set_error(PTTK_EINVAL, "point sets must not be empty");
  if (!(tol >= 0.0 && tol < 1.0)) return set_error(PTTK_EINVAL, "tol must lie in [0, 1)");
  cudaStream_t s = as_stream(stream);
  const int d = tt->d, dth = tt->dtheta, n = tt->n;
  const int rs = tt->ranks[d], rt = tt->ranks[d + dth];
  PTTK_TRY(point_domain_check(tt, X, N_s, Y, N_t, true, tt_status_word(tt), s));
  // Phase 3: S (N_s x r_s) and T (N_t x r_t), row-major FP64
  double *U = nullptr, *V = nullptr, *Scol = nullptr;
  struct Frees {
    std::vector<double*> p;
    ~Frees() {
      for (double* q : p)
        if (q) cudaFree(q);
    }
  } fr;
  PTTK_CUDA(cudaMalloc(&U, sizeof(double) * (size_t)N_s * rs));
  fr.p.push_back(U);
  PTTK_CUDA(cudaMalloc(&V, sizeof(double) * (size_t)N_t * rt));
  fr.p.push_back(V);
  PTTK_TRY(factor_build_run(tt, true, X, N_s, PTTK_FP64, U, s));
  PTTK_TRY(factor_build_run(tt, false, Y, N_t, PTTK_FP64, V, s));
  int st_h = 0;
  PTTK_CUDA(cudaMemcpyAsync(&st_h, tt_status_word(tt), sizeof(int), cudaMemcpyDeviceToHost, s));
  PTTK_CUDA(cudaStreamSynchronize(s));
  if (st_h == (int)PTTK_EDOMAIN) {
    PTTK_CUDA(cudaMemset(tt_status_word(tt), 0, sizeof(int)));
    return set_error(PTTK_EDOMAIN, "a point lies outside its box");
  }
  // the first core of the twisted TT is S column-major; the last is T^T column-major, which
  // is T row-major as it stands
  PTTK_CUDA(cudaMalloc(&Scol, sizeof(double) * (size_t)N_s * rs));
  fr.p.push_back(Scol);
  PTTK_TRY(transpose_rm(U, N_s, rs, Scol, s));
  std::vector<const double*> thc(dth);
  std::vector<int> ranks(dth + 1);
  for (int j = 0; j < dth; ++j) thc[j] = tt->cores64 + tt->core_off[d + j];
  for (int j = 0; j <= dth; ++j) ranks[j] = tt->ranks[d + j];
  std::vector<double*> G(dth + 2, nullptr);
  std::vector<int> nr(dth + 1);
  if (tol > 0.0) {
    // Phase 4
    const pttk_status st = phase4_round(Scol, N_s, thc.data(), ranks.data(), n, dth, V, N_t, tol, G.data(),
                                        nr.data(), s);
    if (st != PTTK_OK) {
      for (double* q : G)
        if (q) cudaFree(q);
      return st;
    }
  } else {
    // Phase 3 only: the factors and cores as they are
    G[0] = Scol;
    fr.p[2] = nullptr;
    G[dth + 1] = V;
    fr.p[1] = nullptr;
    for (int j = 0; j < dth; ++j) {
      const size_t e = (size_t)ranks[j] * n * ranks[j + 1];
      PTTK_CUDA(cudaMalloc(&G[j + 1], sizeof(double) * e));
      PTTK_CUDA(cudaMemcpyAsync(G[j + 1], thc[j], sizeof(double) * e, cudaMemcpyDeviceToDevice, s));
    }
    nr = ranks;
  }
  pttk_fixed* f = new pttk_fixed();
  f->Ns = N_s;
  f->Nt = N_t;
  pttk_tt& h = f->th;
  h.kernel = tt->kernel;
  h.d = 0;
  h.dtheta = dth;
  h.D = dth;
  h.n = n;
  for (int j = 0; j < dth; ++j) {
    h.box[j][0] = tt->box[d + j][0];
    h.box[j][1] = tt->box[d + j][1];
  }
  for (int j = 0; j <= dth; ++j) h.ranks[j] = nr[j];
  size_t off = 0;
  for (int j = 0; j < dth; ++j) {
    h.core_off[j] = off;
    off += (size_t)nr[j] * n * nr[j + 1];
  }
  h.core_total = off;
  h.device = tt->device;
  pttk_status res = PTTK_OK;
  cudaError_t e = cudaMalloc(&h.cores64, sizeof(double) * std::max<size_t>(off, 1));
  if (e == cudaSuccess)
    for (int j = 0; j < dth && e == cudaSuccess; ++j)
      e = cudaMemcpyAsync(h.cores64 + h.core_off[j], G[j + 1], sizeof(double) * (size_t)nr[j] * n * nr[j + 1],
                          cudaMemcpyDeviceToDevice, s);
  // S' row-major from its column-major core; T' row-major is the last core as it stands
  if (e == cudaSuccess) e = cudaMalloc(&f->S, sizeof(double) * (size_t)N_s * nr[0]);
  if (e == cudaSuccess) res = transpose_rm(G[0], nr[0], N_s, f->S, s);  // (r_s' x N_s row-major)^T
  if (e == cudaSuccess && res == PTTK_OK) {
    f->T = G[dth + 1];
    G[dth + 1] = nullptr;
    e = cudaStreamSynchronize(s);
  }
  for (int j = 0; j < dth + 1; ++j)
    if (G[j]) cudaFree(G[j]);
  if (e != cudaSuccess || res != PTTK_OK) {
    fixed_release(f);
    return e != cudaSuccess ? cuda_error(e, "Phase 4 handle") : res;
  }
  *out = f;
  return PTTK_OK;
}

pttk_status pttk_fixed_dims(const pttk_fixed* f, int64_t* N_s, int64_t* N_t, int* d_theta, int* ranks) {
  clear_error();
  if (!f) return set_error(PTTK_EINVAL, "NULL handle");
  if (N_s) *N_s = f->Ns;
  if (N_t) *N_t = f->Nt;
  if (d_theta) *d_theta = f->th.dtheta;
  if (ranks)
    for (int j = 0; j <= f->th.dtheta; ++j) ranks[j] = f->th.ranks[j];
  return PTTK_OK;
}

pttk_status pttk_fixed_get_factors(const pttk_fixed* f, double* S, double* T, void* stream) {
  clear_error();
  if (!f) return set_error(PTTK_EINVAL, "NULL handle");
  cudaStream_t s = as_stream(stream);
  const int dth = f->th.dtheta;
  if (S) PTTK_CUDA(cudaMemcpyAsync(S, f->S, sizeof(double) * (size_t)f->Ns * f->th.ranks[0], cudaMemcpyDeviceToDevice, s));
  if (T)
    PTTK_CUDA(cudaMemcpyAsync(T, f->T, sizeof(double) * (size_t)f->Nt * f->th.ranks[dth], cudaMemcpyDeviceToDevice, s));
  return PTTK_OK;
}

pttk_status pttk_fixed_get_core(const pttk_fixed* f, int j, double* host_out) {
  clear_error();
  if (!f || !host_out) return set_error(PTTK_EINVAL, "NULL argument");
  if (j < 0 || j >= f->th.dtheta) return set_error(PTTK_EINVAL, "no such theta core");
  const pttk_tt& h = f->th;
  PTTK_CUDA(cudaMemcpy(host_out, h.cores64 + h.core_off[j], sizeof(double) * (size_t)h.ranks[j] * h.n * h.ranks[j + 1],
                       cudaMemcpyDeviceToHost));
  return PTTK_OK;
}

pttk_status pttk_fixed_theta_core(const pttk_fixed* f, const double* theta, pttk_prec prec, void* M, void* stream) {
  clear_error();
  if (!f || !M) return set_error(PTTK_EINVAL, "NULL argument");
  if (prec != PTTK_FP64 && prec != PTTK_FP32) return set_error(PTTK_EINVAL, "precision must be FP64 or FP32");
  double th[PTTK_MAX_D];
  PTTK_TRY(theta_hat(&f->th, theta, th));
  return theta_core_run(&f->th, th, prec == PTTK_FP64, M, as_stream(stream));
}

void pttk_fixed_free(pttk_fixed* f) { fixed_release(f); }

}  // extern "C"

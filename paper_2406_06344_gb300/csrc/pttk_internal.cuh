// Internal declarations shared by the libpttk translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/pttk.h"

#define PTTK_MAX_D 8

// Parameters of each kernel: theta = (l, nu) for the general-nu Matern kernel, (l) for the
// other length-scale kernels, none for the singular kernels of the TTK variant.
inline int kernel_dtheta(int kernel) {
  return kernel == PTTK_MATERN_NU ? 2 : (kernel >= PTTK_BIHARMONIC && kernel <= PTTK_THIN_PLATE) ? 0 : 1;
}
#define PTTK_MAX_N 32

struct pttk_tt {
  int kernel = 0, d = 0, dtheta = 0, D = 0, n = 0;
  double box[PTTK_MAX_D][2] = {};   // (alpha_j, beta_j) in the variable order (x, theta, y)
  int ranks[PTTK_MAX_D + 1] = {};   // r_0..r_D
  size_t core_off[PTTK_MAX_D] = {}; // element offset of core k in the core buffers
  size_t core_total = 0;            // total core elements
  double* cores64 = nullptr;        // device, FP64 cores, column-major r_{k-1} x n x r_k
  float* cores32 = nullptr;         // device, FP32 copy (online FP32 / tensor-core forms)
  int device = 0;
  size_t core_elems(int k) const { return (size_t)ranks[k] * n * ranks[k + 1]; }
};

namespace pttk {

// Thread-local message for pttk_last_error(); set_error returns its status for chaining.
pttk_status set_error(pttk_status s, const std::string& msg);
pttk_status cuda_error(cudaError_t e, const char* what);
void clear_error();

#define PTTK_CUDA(call)                                     \
  do {                                                      \
    cudaError_t e__ = (call);                               \
    if (e__ != cudaSuccess) return pttk::cuda_error(e__, #call); \
  } while (0)

#define PTTK_TRY(call)                                      \
  do {                                                      \
    pttk_status s__ = (call);                               \
    if (s__ != PTTK_OK) return s__;                         \
  } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Diagnostic logging to stderr (stage times, sweep counts): compiled in only by a build with
// -DPTTK_DEBUG, the library's one build switch; release builds read no environment.
#ifdef PTTK_DEBUG
constexpr bool kDebugLog = true;
#else
constexpr bool kDebugLog = false;
#endif

int sm_count();

// Number of kernels the library has launched (every launch site increments it).
void count_launch();

// Kernel timing (profile.cu): when enabled, PTTK_PROF brackets a launch with CUDA events
// recorded on its stream; results are read through pttk_profile_get.
bool prof_on();
void* prof_begin(const char* name, cudaStream_t s);
void prof_end(const char* name, cudaStream_t s);
struct ProfScope {
  const char* name;
  cudaStream_t s;
  ProfScope(const char* n, cudaStream_t st) : name(n), s(st) { prof_begin(n, st); }
  ~ProfScope() { prof_end(name, s); }
};
#define PTTK_PROF(name, stream) pttk::ProfScope pttk_prof_scope__(name, stream)

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) in counter-based form: output number
// `counter` (0-based) of the stream seeded with `key`, i.e. the state after counter + 1
// increments by the golden gamma, through the variant-13 mix. The TT greedy-cross draws all of
// its random numbers from it.
__host__ __device__ inline uint64_t splitmix64(uint64_t key, uint64_t counter) {
  uint64_t z = key + (counter + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// --- api.cu ----------------------------------------------------------------------------
// theta -> theta_hat (the inverse of the printed interval map) per parameter; PTTK_EDOMAIN when
// theta lies outside its box beyond a relative slack of 1e-12.
pttk_status theta_hat(const pttk_tt* tt, const double* theta, double* th);

// --- grid.cu ---------------------------------------------------------------------------
pttk_status grid_coeffs_launch(int kernel, int d, int dtheta, int n, const double (*box)[2],
                               bool fp64, void* C, cudaStream_t s);
// Grid-tensor entries at M multi-indices (dev, M x D row-major int32); a bad index records
// PTTK_EINVAL in *status (dev int).
pttk_status grid_entries_launch(int kernel, int d, int dtheta, int n, const double (*box)[2],
                                const int* idx, int64_t M, bool fp64, void* out, int* status,
                                cudaStream_t s);

// --- ttsvd.cu --------------------------------------------------------------------------
// TT-SVD of the FP64 tensor in `X` (n^D elements, modified). Fills tt->ranks and
// allocates tt->cores64 / cores32. Synchronises `s`.
pttk_status tt_svd_run(pttk_tt* tt, double* X, double tol, cudaStream_t s);
pttk_status tt_round_run(const pttk_tt* in, double tol, pttk_tt* out, cudaStream_t s);
pttk_status widen_to_f64(const float* in, int64_t n, double* out, cudaStream_t s);
// Orthonormal basis (allocated here, m x r column-major) of the range of X (m x c, column-major).
pttk_status range_basis(const double* X, int64_t m, int64_t c, double** basis, int* r, cudaStream_t s);
// One-sided Jacobi on the columns of A (rows x ncols, column-major), in place.
pttk_status jacobi_columns(double* A, int64_t rows, int ncols, cudaStream_t s);

// FP64 column-major GEMM: C[M x N] = alpha * op(A) * op(B) + beta * C.
void dgemm(bool transA, bool transB, int64_t M, int64_t N, int64_t K, double alpha,
           const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
           int64_t ldc, cudaStream_t s);

// --- chain_tc.cu (tensor-core factor chain) ------------------------------------------
struct TcImageCache;
TcImageCache* tc_cache_new();
void tc_cache_free(TcImageCache* c);
// Both factors in one persistent launch; cfg selects a launch configuration (0 = default,
// tc_config_count() of them). Lays out the core images on first use (synchronises once).
pttk_status factor_build_tc(const pttk_tt* tt, TcImageCache* cache, const float* X, int64_t N_s,
                            const float* Y, int64_t N_t, pttk_prec prec, float* U, float* V,
                            int* d_status, int cfg, cudaStream_t s);
pttk_status tc_prepare(const pttk_tt* tt, TcImageCache* cache, pttk_prec prec, int cfg, cudaStream_t s);
int tc_config_count();

// --- online.cu -------------------------------------------------------------------------
pttk_status theta_core_run(const pttk_tt* tt, const double* theta_hat, bool fp64, void* M,
                           cudaStream_t s);
// SIMT chain (FP64 / FP32); nsteps < d stops after that many steps (out: N x r_nsteps).
pttk_status factor_build_run(const pttk_tt* tt, bool source, const void* P, int64_t N,
                             pttk_prec prec, void* out, cudaStream_t s, int nsteps = 0);
int oriented_core_dims(const pttk_tt* tt, bool source, int step, int* R_in, int* R_out, int* coord);
// Symmetric eigendecomposition of nb k x k matrices (eig.cu): sym_eig_values tridiagonalises
// A in place and returns all eigenvalues ascending (lam: nb x k) with d, e, tau for
// sym_eig_vectors, which computes the eigenvectors of the selected eigenvalues (listed per
// matrix in ascending order) into columns sel_col of V (nb x k x ncols). sel_w: the weight
// |f(lambda)| each eigenpair carries in the caller's spectral function f(A) = sum f u u^T
// (|lambda| for A itself); vectors are re-orthogonalised where two eigenvalues lie within
// 1e-3 of the larger weight. Device buffers.
pttk_status sym_eig_values(double* A, int k, int nb, double* d, double* e, double* tau, double* lam, cudaStream_t s);
pttk_status sym_eig_vectors(const double* A, const double* d, const double* e, const double* tau, int k, int nb,
                            const std::vector<int>& sel_z, const std::vector<double>& sel_lam,
                            const std::vector<double>& sel_w, const std::vector<int>& sel_col, double* V,
                            int ncols, cudaStream_t s);
// One pass over the source points X (N_s x d) and the target points Y (N_t x d), row-major,
// double if fp64 else float: records PTTK_EDOMAIN in *status if a coordinate lies outside
// its box. A NULL side or a count <= 0 is skipped.
pttk_status point_domain_check(const pttk_tt* tt, const void* X, int64_t N_s, const void* Y, int64_t N_t, bool fp64,
                               int* status, cudaStream_t s);
const void* oriented_core_ptr(const pttk_tt* tt, bool source, int k, bool fp64);
int* tt_status_word(const pttk_tt* tt);
struct TcImageCache;
TcImageCache* tt_tc_cache(const pttk_tt* tt);
pttk_status apply_run(const void* U, const void* M, const void* V, int64_t N_s, int64_t N_t,
                      int rs, int rt, bool fp64, const void* w, void* out, void* scratch,
                      cudaStream_t s);
size_t apply_scratch_bytes(int64_t N_t, int rs, int rt, bool fp64);

}  // namespace pttk

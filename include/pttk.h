/*
 * pttk.h: C ABI of libpttk, a GB300 (sm_103a) implementation of the parametric
 * tensor-train kernel (PTTK) low-rank method of Khan & Saibaba, "Parametric kernel
 * low-rank approximations using tensor train decomposition" (arXiv 2406.06344).
 *
 * The method approximates a parametric kernel matrix
 *     K(X, Y; theta)_ij = kappa(x_i, y_j; theta)                     (Eq. matparamkernel)
 * by K ~= U(X) M(theta) V(Y)^T                                          (Eq. paramlowrank)
 * in two stages:
 *   offline  evaluate f_kappa(x, theta, y) on the tensor grid of Chebyshev nodes over
 *            B_s x B_theta x B_t (Eq. mdc), map the values to Chebyshev coefficients
 *            per mode, and compress the coefficient tensor by TT-SVD (Section 2.3);
 *   online   contract the theta cores with the Chebyshev vector of theta (Eq. hmat,
 *            Algorithm 3) and build the factors U, V by the chained Khatri-Rao/core
 *            contractions of Algorithm 2, Phase 3.
 *
 * Conventions shared by every entry point
 *   - Variable order is xi = (x, theta, y); D = 2 d + d_theta (Eq. fkappa).
 *   - Boxes are arrays of (lo, hi) pairs: box[2 j] = alpha_j, box[2 j + 1] = beta_j, with
 *     finite ends and lo < hi (else PTTK_EINVAL). The interval map is the one printed in
 *     Section 2.4, phi_[a,b](t) = ((a-b)/2) t + (a+b)/2; Chebyshev nodes are the roots of T_n.
 *   - The coefficient tensor C (n^D entries) is stored column-major: i_1 varies fastest
 *     (the little-endian flattening of Section 2.2).
 *   - A TT core G_k has shape r_{k-1} x n x r_k, stored column-major (index
 *     a + r_{k-1} (j + n b)); r_0 = r_D = 1.
 *   - Point sets X (N_s x d), Y (N_t x d) and the factors U (N_s x r_d),
 *     M (r_d x r_{d+d_theta}) and V (N_t x r_{d+d_theta}) are row-major.
 *   - Precision: PTTK_FP64 takes and returns double; every other precision takes float
 *     points and returns float factors. TF32/BF16 forms run on the tensor cores with
 *     FP32 accumulation; the X3 forms split each operand into a high and a low part
 *     and issue three products (high*high + high*low + low*high).
 *   - Memory: "dev" pointers are device (or managed) memory owned by the caller; "host"
 *     pointers are host memory owned by the caller. The library owns pttk_tt handles.
 *   - Streams: `stream` is a cudaStream_t (NULL = the legacy default stream). Calls
 *     enqueue work on it and return; results are ready when the stream is synchronised,
 *     except where a call says it synchronises.
 *   - Errors: every call returns a pttk_status; on failure pttk_last_error() returns a
 *     message for the calling thread. No C++ exception crosses this boundary. A call that
 *     fails leaves its outputs unspecified and the handle unchanged.
 */
#ifndef PTTK_H
#define PTTK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pttk_status {
  PTTK_OK = 0,
  PTTK_EINVAL = 1,   /* bad argument: size, box, pointer, precision, rank mismatch */
  PTTK_EDOMAIN = 2,  /* theta, or a point, outside its box */
  PTTK_ENOMEM = 3,   /* a device or host allocation failed */
  PTTK_ECUDA = 4,    /* a CUDA runtime error; pttk_last_error() has its text */
  PTTK_ETIMEOUT = 5, /* a bounded device-side wait ran out */
  PTTK_ENOTSUP = 6   /* combination not implemented (e.g. a precision for this shape) */
} pttk_status;

/* Kernels of Table kern-table (r = ||x - y||_2, a = r / l):
 *   PTTK_GAUSS              theta = (l):      exp(-a^2)
 *   PTTK_MATERN32           theta = (l):      (1 + sqrt(3) a) exp(-sqrt(3) a)
 *   PTTK_MATERN_NU          theta = (l, nu):  2^(1-nu)/Gamma(nu) (sqrt(2 nu) a)^nu K_nu(sqrt(2 nu) a)
 *   PTTK_EXPONENTIAL        theta = (l):      exp(-a)
 *   PTTK_MATERN52           theta = (l):      (1 + sqrt(5) a + 5 a^2 / 3) exp(-sqrt(5) a)
 *   PTTK_MULTIQUADRIC       theta = (l):      (1 + a^2)^(1/2)
 *   PTTK_THIN_PLATE_SPLINE  theta = (l):      a^2 log(a^2)
 * and, without a parameter (d_theta = 0, the TTK variant of Section 3.3; the boxes must be
 * admissible, dist(source box, target box) > 0, since these are singular at r = 0):
 *   PTTK_BIHARMONIC         r^-2
 *   PTTK_LAPLACE3D          r^-1
 *   PTTK_LAPLACE2D          -log(r)
 *   PTTK_THIN_PLATE         r^2 log(r)
 * (the table prints Gamma(l) in the Matern normalisation; Gamma(nu) is used). */
typedef enum pttk_kernel {
  PTTK_GAUSS = 0,
  PTTK_MATERN32 = 1,
  PTTK_MATERN_NU = 2,
  PTTK_EXPONENTIAL = 3,
  PTTK_MATERN52 = 4,
  PTTK_MULTIQUADRIC = 5,
  PTTK_THIN_PLATE_SPLINE = 6,
  PTTK_BIHARMONIC = 7,
  PTTK_LAPLACE3D = 8,
  PTTK_LAPLACE2D = 9,
  PTTK_THIN_PLATE = 10
} pttk_kernel;

typedef enum pttk_prec {
  PTTK_FP64 = 0,
  PTTK_FP32 = 1,
  PTTK_TF32 = 2,
  PTTK_TF32X3 = 3,
  PTTK_BF16 = 4,
  PTTK_BF16X3 = 5,
  PTTK_FP16 = 6,
  PTTK_FP16X3 = 7
} pttk_prec;

typedef struct pttk_tt pttk_tt; /* opaque: TT cores on the device plus their metadata */

/* Message for the last failing call on this thread ("" if none). Never NULL. */
const char* pttk_last_error(void);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int pttk_version(void);

/* ---- offline stage ----------------------------------------------------------------- */

/* Grid evaluation and Chebyshev transform (Eq. mdc; Eq. cheb_trans rewritten as
 * coefficients). Writes C = M x_1 A x_2 A ... x_D A to `C` (dev, n^D elements, column-major),
 * where m_{i_1..i_D} = f_kappa(eta^(1)_{i_1}, ..., eta^(D)_{i_D}) and
 * A[k, i] = (c_k / n) T_k(zeta_i), c_0 = 1, c_k = 2.
 *   src_box, tgt_box: host [2 d]; theta_box: host [2 d_theta].
 *   grid_prec: PTTK_FP64 (C is double) or PTTK_FP32 (C is float; evaluation and transform
 *   in FP32).
 *   1 <= d <= 3, 2 <= n <= 32, n^D <= 4e9; d_theta = 1 (theta = (l)) for PTTK_GAUSS and
 *   PTTK_MATERN32, d_theta = 2 (theta = (l, nu)) for PTTK_MATERN_NU; l > 0 and nu > 0 over
 *   their boxes. Otherwise PTTK_EINVAL. */
pttk_status pttk_grid_coeffs(pttk_kernel kernel, int d, const double* src_box,
                             const double* tgt_box, int d_theta, const double* theta_box, int n,
                             pttk_prec grid_prec, void* C, void* stream);

/* Entries of the grid tensor M (Eq. mdc) at given multi-indices, without the grid: the entry
 * access the TT greedy-cross (Algorithms 5-7) works from.
 *   out[e] = f_kappa(eta^(1)_{idx[e,0]}, ..., eta^(D)_{idx[e,D-1]}), variables in the order
 *   (x, theta, y) of Eq. fkappa, eta^(j) the Chebyshev nodes of mode j mapped to its box.
 *   idx: dev, M x D row-major int32, each in [0, n) (0-based node index).
 *   out: dev, M entries (double for PTTK_FP64, float for PTTK_FP32).
 *   Kernel, boxes and n as for pttk_grid_coeffs, except that n^D may exceed 4e9 (no grid is
 *   formed).
 * An index outside [0, n) writes NaN for that entry and returns PTTK_EINVAL; no node is read
 * with it. M = 0 is a no-op. Synchronises `stream`. */
pttk_status pttk_grid_entries(pttk_kernel kernel, int d, const double* src_box,
                              const double* tgt_box, int d_theta, const double* theta_box, int n,
                              const int32_t* idx, int64_t M, pttk_prec prec, void* out, void* stream);

/* TT-SVD of a coefficient tensor (Section 2.3; Oseledets 2011, Algorithm 1) with the
 * truncation threshold delta = tol / sqrt(D-1) * ||C||_F of Algorithm 1 (TT-Round):
 * r_k is the smallest r >= 1 whose discarded singular values satisfy
 * sqrt(sum_{i>r} sigma_i^2) <= delta. All QR/SVD steps run in FP64 on the device.
 *   C: dev, n^D elements (double if c_prec = PTTK_FP64, float if PTTK_FP32), column-major,
 *   not modified. The kernel, boxes and n describe the grid C came from and are stored in
 *   the handle for the online stage. On success *out owns a new handle; free it with
 *   pttk_tt_free. Synchronises `stream` (the ranks are decided on the host). */
pttk_status pttk_tt_from_coeffs(pttk_kernel kernel, int d, const double* src_box,
                                const double* tgt_box, int d_theta, const double* theta_box,
                                int n, double tol, const void* C, pttk_prec c_prec,
                                void* stream, pttk_tt** out);

/* Offline stage (Algorithm 2, Phases 1-2, with the full grid and TT-SVD in place of
 * TT greedy-cross): pttk_grid_coeffs into a library-owned buffer, then
 * pttk_tt_from_coeffs. Synchronises `stream`. */
pttk_status pttk_build_offline(pttk_kernel kernel, int d, const double* src_box,
                               const double* tgt_box, int d_theta, const double* theta_box,
                               int n, double tol, pttk_prec grid_prec, void* stream,
                               pttk_tt** out);

/* ---- handle queries, checkpoint ---------------------------------------------------- */

/* d, d_theta, n and the kernel of a handle (any pointer may be NULL). */
pttk_status pttk_tt_dims(const pttk_tt* tt, int* d, int* d_theta, int* n, int* kernel);

/* TT ranks r_0..r_D (host array of D + 1 ints; r_0 = r_D = 1). */
pttk_status pttk_tt_ranks(const pttk_tt* tt, int* ranks);

/* Copy core k (0-based, 0 <= k < D) to host memory: r_{k-1} * n * r_k doubles,
 * column-major. Synchronous. */
pttk_status pttk_tt_get_core(const pttk_tt* tt, int k, double* host_out);

/* Write / read a handle (kernel, d, d_theta, n, boxes, ranks, FP64 cores) to / from a
 * little-endian binary file. pttk_tt_load allocates device memory on the current device. */
pttk_status pttk_tt_save(const pttk_tt* tt, const char* path);
pttk_status pttk_tt_load(const char* path, pttk_tt** out);

/* A handle from given TT cores (the TT format of Section 2.3): for instance cores computed
 * elsewhere, or cores with chosen ranks for timing the online stage. The problem arguments
 * are those of pttk_grid_coeffs, except that n^D may exceed 4e9 (no grid is formed); ranks[0..D] with ranks[0] = ranks[D] = 1; `cores` is host
 * memory holding the D cores one after another, core k as r_{k-1} x n x r_k doubles,
 * column-major (the layout pttk_tt_get_core returns). The cores must be the Chebyshev
 * coefficient form (contracted with T(xhat), not with nodal values). Copied; the caller
 * keeps ownership of `cores`. Synchronous. Errors: PTTK_EINVAL (bad problem or ranks),
 * PTTK_ENOMEM / PTTK_ECUDA. */
pttk_status pttk_tt_from_cores(pttk_kernel kernel, int d, const double* src_box, const double* tgt_box,
                               int d_theta, const double* theta_box, int n, const int* ranks,
                               const double* cores, pttk_tt** out);

/* TT-Round (Algorithm 1): a new handle holding a TT of the same tensor with ranks reduced so
 * that ||X - X_rounded||_F <= tol ||X||_F (X the tensor `in` represents): right-to-left
 * orthogonalisation of the cores, then a left-to-right sweep of truncated SVDs with
 * delta = tol / sqrt(D - 1) ||X||_F, in FP64 with the factorisation of the TT-SVD. For TTs
 * whose ranks are inflated (given cores, sums or products of TTs). `in` is unchanged; the
 * caller frees both. tol in (0, 1). Synchronises `stream`. Errors: PTTK_EINVAL, PTTK_ENOMEM,
 * PTTK_ECUDA, PTTK_ETIMEOUT. */
pttk_status pttk_tt_round(const pttk_tt* in, double tol, void* stream, pttk_tt** out);

/* Release a handle and its device memory (NULL is a no-op). */
void pttk_tt_free(pttk_tt* tt);

/* ---- PTTK-Global (Algorithm 4, Section 3 "Global low-rank approximation") ------------------
 * The global case: one point set X in one box (source box = target box) and a kernel symmetric
 * in its arguments. K(X, X; theta) ~= Z W Z^T with W symmetric, positive semi-definite when
 * the negative eigenvalues are dropped (a definite kernel). */
typedef struct pttk_global pttk_global;

/* Offline stage of Algorithm 4. S = U(X) and T = V(X) come from the FP64 factor chains of
 * Algorithm 2 (Phase 3) on the one point set. Then the thin QR [S T] = Q R:
 *   - Q: N x k with orthonormal columns, k <= r_s + r_t (r_s = r_d, r_t = r_{d+d_theta});
 *   - R = Q^T [S T], k x (r_s + r_t).
 * Q is an orthonormal basis of the range of [S T], computed with the pivoted Householder QR
 * and one-sided Jacobi of the TT-SVD. R need not be triangular: any pair with orthonormal Q
 * and Q R = [S T] gives the same Q R H^ R^T Q^T, which is all the method uses.
 *   tt: a handle whose source and target boxes are equal (else PTTK_EINVAL). It may be freed
 *       afterwards: the new handle keeps its own copy of the cores.
 *   X:  dev, N x d row-major doubles, N >= 1, points inside the box.
 * Synchronises `stream`. The handle holds Q (8 N k bytes) and R. The call needs scratch of
 * about five N x (r_s + r_t) doubles.
 * Errors: PTTK_EINVAL, PTTK_ENOMEM, PTTK_ENOTSUP (ranks too large for the FP64 chain),
 * PTTK_ECUDA, PTTK_ETIMEOUT. */
pttk_status pttk_global_create(const pttk_tt* tt, const double* X, int64_t N, void* stream,
                               pttk_global** out);

/* N, k (columns of Q), r_s and r_t of a handle. Any output pointer may be NULL. */
pttk_status pttk_global_dims(const pttk_global* g, int64_t* N, int* k, int* r_s, int* r_t);

/* Copies Q (N x k, row-major doubles) into the caller's device buffer Q, asynchronously on
 * `stream`. */
pttk_status pttk_global_get_q(const pttk_global* g, double* Q, void* stream);

/* Copies R (k x (r_s + r_t), column-major doubles) into host memory. Synchronous. */
pttk_status pttk_global_get_r(const pttk_global* g, double* R_host);

/* Online stage of Algorithm 4 at theta (host [d_theta], inside its box, else PTTK_EDOMAIN).
 * First H = H(theta), then the eigendecomposition R H^ R^T = U Lambda U^T, where
 * H^ = [[0, H/2], [H^T/2, 0]] (Eq. pttk1). Eigenpairs are taken in order of decreasing
 * |lambda|.
 *   definite = 1: negative eigenvalues are dropped (a positive definite kernel).
 *   definite = 0: they are kept (an indefinite kernel such as the Multiquadric).
 *   compress = 0 (PTTK-Global-1): W (dev, k x k doubles) = U Lambda U^T and *rank = k.
 *     K ~= Q W Q^T, with Q from pttk_global_get_q. Z is not used and may be NULL.
 *   compress = 1 (PTTK-Global-2): keeps the fewest leading eigenpairs such that
 *     ||Z W Z^T - S H T^T||_F <= eps ||S H T^T||_F, or all of them when no prefix meets it.
 *     Z (dev, N x rank, row-major; capacity N x k) = Q U^.
 *     W (dev, rank x rank; capacity k x k) = diag(lambda^). *rank = the terms kept.
 * Eigenpairs whose eigenvalue lies within 64 eps max|lambda| of zero are below what FP64
 * resolves and give no term. The eigensolver: Householder tridiagonalisation, every eigenvalue
 * by multisection on Sturm counts, inverse iteration for the eigenvectors kept, back through
 * the reflectors (no step waits on another CTA).
 * eps in [0, 1). FP64 throughout. Synchronises `stream`.
 * Errors: PTTK_EINVAL, PTTK_EDOMAIN, PTTK_ENOMEM, PTTK_ECUDA, PTTK_ENOTSUP (k > 12800). */
pttk_status pttk_global_instantiate(const pttk_global* g, const double* theta, double eps, int compress,
                                    int definite, double* Z, double* W, int* rank, void* stream);

/* PTTK-Global-1 (compress = 0 of pttk_global_instantiate) for B parameter values at once:
 * thetas (host, B x d_theta, row b = theta_b, each inside its box, else PTTK_EDOMAIN); W (dev,
 * B x k x k doubles, matrix b column-major at offset b k^2) = U_b Lambda_b U_b^T, the same
 * selection of eigenpairs as the single-theta call. The B eigenproblems share every launch of
 * the eigensolver, so the launch-bound tridiagonalisation costs about what one theta costs.
 * B = 0 is a no-op. Synchronises `stream`. Errors: as pttk_global_instantiate. */
pttk_status pttk_global_instantiate_batched(const pttk_global* g, int B, const double* thetas, int definite,
                                            double* W, void* stream);

/* Release a handle and its device memory (NULL is a no-op). */
void pttk_global_free(pttk_global* g);

/* ---- TT greedy-cross (Algorithms 5, 6, 7; Appendix "TT-cross approximation") ------------
 * Phase 2 of Algorithm 2 as the paper runs it: a TT of the grid tensor M (Eq. mdc) from sampled
 * entries, never forming the n^D grid, so that grids beyond device memory (the paper's n = 27,
 * D = 8 grid holds 2.8e11 entries) can be compressed. The index sets of cardinality two of
 * Algorithm 7 (init_it passes), then sweeps of Algorithm 5's cross updates on every super-core
 * unfolding until the largest |x - x^| over n_check random entries, relative to the largest
 * |x| among them, is <= eps, a sweep adds no pivot, or max_sweeps sweeps have run. The cores
 * of the interpolation X^ = T_1 P_1^{-1} T_2 .. P_{N-1}^{-1} T_N are then transformed to
 * Chebyshev coefficients (G_k <- G_k x_2 A), giving a handle like pttk_build_offline's.
 * Every random number comes from SplitMix64 with the given key (pttk_splitmix64), drawn in the
 * order the method consumes them: q1 and q2 of Algorithm 7, then per update the sample
 * positions and the row-or-column bit, per sweep the check entries. Each argmin and argmax
 * takes the first index within a relative 1e-12 of the extremum. Kernel entries, the cross-
 * matrix solves, the skeleton residuals and the check are computed on the device; index sets
 * stay on the host. The problem arguments are those of pttk_grid_coeffs (n <= 32). eps in
 * (0, 1); n_check >= 1; init_it >= 1; max_sweeps >= 0. *sweeps (may be NULL) = sweeps run,
 * *evals (may be NULL) = kernel entries evaluated. Synchronises `stream`.
 * Errors: PTTK_EINVAL, PTTK_ENOMEM, PTTK_ECUDA, PTTK_ENOTSUP (a rank above 1024). */
pttk_status pttk_cross_build(pttk_kernel kernel, int d, const double* src_box, const double* tgt_box, int d_theta,
                             const double* theta_box, int n, double eps, uint64_t key, int max_sweeps, int n_check,
                             int init_it, void* stream, pttk_tt** out, int* sweeps, int64_t* evals);

/* ---- Algorithm 2 for fixed point sets: Phases 3 and 4 -----------------------------------
 * When X and Y stay fixed and only theta changes, the paper computes the factors once offline
 * (Algorithm 2, Phase 3: S = U(X), T = V(Y)) and compresses them with the theta cores by
 * Phase 4: TT-Round (Algorithm 1) of the twisted TT [T^(1)(S), G_{d+1}, .., G_{d+d_theta},
 * T^(3)(T^T)] of Eq. twist, an order-(d_theta + 2) TT with mode sizes (N_s, n, .., n, N_t).
 * The online stage (Algorithm 3) then only contracts the rounded theta cores:
 * K(X, Y; theta) ~= S' H'(theta) T'^T. */
typedef struct pttk_fixed pttk_fixed;

/* Phases 3 and 4 on the handle's TT. X: dev N_s x d, Y: dev N_t x d, row-major doubles, inside
 * their boxes (else PTTK_EDOMAIN), N_s, N_t >= 1. S and T are built by the FP64 factor chains;
 * tol in (0, 1) rounds them as above with delta = tol / sqrt(d_theta + 1) ||X||_F, X the
 * twisted tensor; tol = 0 skips Phase 4 (the handle then holds S, T and the theta cores as they
 * are). FP64 throughout; the factorisations are those of the TT-SVD (pivoted Householder QR and
 * one-sided Jacobi). The handle keeps S' (N_s x r_s'), T' (N_t x r_t') and the rounded theta
 * cores on the device; `tt` may be freed afterwards. Synchronises `stream`.
 * Errors: PTTK_EINVAL, PTTK_EDOMAIN, PTTK_ENOMEM, PTTK_ECUDA, PTTK_ETIMEOUT, PTTK_ENOTSUP (ranks
 * too large for the FP64 chain). */
pttk_status pttk_fixed_create(const pttk_tt* tt, const double* X, int64_t N_s, const double* Y, int64_t N_t,
                              double tol, void* stream, pttk_fixed** out);
/* N_s, N_t, d_theta, and ranks[0 .. d_theta] = (r_s', inner ranks of the rounded theta cores,
 * r_t'); for d_theta = 0, ranks[0] = r_s' = r_t'. Any output pointer may be NULL. */
pttk_status pttk_fixed_dims(const pttk_fixed* f, int64_t* N_s, int64_t* N_t, int* d_theta, int* ranks);
/* Copies S' (N_s x r_s') and T' (N_t x r_t'), row-major doubles, into the caller's device
 * buffers (either may be NULL), asynchronously on `stream`. */
pttk_status pttk_fixed_get_factors(const pttk_fixed* f, double* S, double* T, void* stream);
/* Copies rounded theta core j (0 <= j < d_theta; ranks[j] x n x ranks[j+1], column-major) to
 * host memory. Synchronous. */
pttk_status pttk_fixed_get_core(const pttk_fixed* f, int j, double* host_out);
/* Algorithm 3 on the rounded cores: M = H'(theta) (dev, r_s' x r_t' row-major; double for
 * PTTK_FP64, float for PTTK_FP32). theta: host [d_theta], inside its box (else PTTK_EDOMAIN). */
pttk_status pttk_fixed_theta_core(const pttk_fixed* f, const double* theta, pttk_prec prec, void* M, void* stream);
/* Release a handle and its device memory (NULL is a no-op). */
void pttk_fixed_free(pttk_fixed* f);

/* ---- Gaussian-process workload (Section 1: hyperparameters and CG preconditioning) -------
 * Section 1 names two uses of the parametric low-rank form in Gaussian-process regression:
 * choosing the kernel's hyperparameters by maximising the log marginal likelihood, which
 * needs K(X, X; theta) at many theta, and preconditioning conjugate gradients on the kernel
 * system. Textbook definitions (Rasmussen and Williams 2006, Eqs. 2.30 and 5.9) with noise
 * variance s2 > 0. Kernels: PTTK_GAUSS, PTTK_MATERN32, PTTK_EXPONENTIAL, PTTK_MATERN52
 * (theta = l > 0); X: dev N x d row-major doubles. FP64 throughout. */

/* out = (K(X, X; theta) + s2 I) v with every kernel entry evaluated on the fly (N^2 kernel
 * evaluations, no N x N storage). prec: PTTK_FP64 evaluates in FP64; PTTK_FP32 evaluates each
 * entry and sums each 128-column tile in FP32, the tile sums in FP64 (relative error of order
 * 1e-7). Rows and column ranges are split over blocks (four per SM), the ranges' sums added in
 * a fixed order. v, out: dev [N]. Stream-ordered scratch; asynchronous on `stream`.
 * Errors: PTTK_EINVAL, PTTK_ECUDA. */
pttk_status pttk_gp_kv(int kernel, int d, const double* X, int64_t N, const double* theta, double s2, const double* v,
                       double* out, pttk_prec prec, void* stream);

/* Preconditioned conjugate gradients for (K(X, X; theta) + s2 I) x = b, the matrix applied
 * by pttk_gp_kv in the precision `prec` (with PTTK_FP32 the true residual levels off near the
 * FP32 evaluation's 1e-7; the CG vectors stay FP64) and the preconditioner (Z diag(lambda) Z^T + s2 I)^{-1} in Woodbury form
 * Z ((Z^T v) ./ (lambda + s2)) + (v - Z Z^T v) / s2, Z (dev N x m, row-major, orthonormal
 * columns) and lambda (dev [m]) from PTTK-Global (pttk_global_instantiate with compress = 1; eps
 * = 0 keeps every term); m = 0 runs plain CG. x0 = 0; stops once ||b - A x||_2 <= tol ||b||_2
 * (the recursively updated residual) or after maxit iterations. b, x: dev [N]. *iters and
 * *resid (either may be NULL): the iterations taken and the final relative residual.
 * Allocates scratch; synchronises `stream` every iteration.
 * Errors: PTTK_EINVAL, PTTK_ENOMEM, PTTK_ECUDA, PTTK_EDOMAIN (p^T A p <= 0: not positive definite). */
pttk_status pttk_gp_pcg(int kernel, int d, const double* X, int64_t N, const double* theta, double s2, const double* Z,
                        const double* lam, int m, const double* b, double* x, double tol, int maxit, pttk_prec prec,
                        int* iters, double* resid, void* stream);

/* Log marginal likelihood of y ~ N(0, K~ + s2 I) and its gradient in theta for the low-rank
 * kernel of a PTTK-Global handle, K~(theta) = sym(S H(theta) T^T) = Q sym(C1(theta)) Q^T
 * (Algorithm 4 without the zeroing of negative eigenvalues, so that K~ is differentiable):
 *   lml = -1/2 y^T (K~ + s2 I)^{-1} y - 1/2 log det(K~ + s2 I) - N/2 log(2 pi),
 *   d lml / d theta_j = 1/2 (alpha^T dK~_j alpha - tr((K~ + s2 I)^{-1} dK~_j)),
 *   alpha = (K~ + s2 I)^{-1} y, dK~_j = sym(S dH_j T^T) (dH_j from T_k' in Eq. hmat).
 * With B = sym(C1) (k x k) and c = Q^T y these reduce exactly to k x k algebra: log det =
 * sum log(lambda_i(B) + s2) + (N - k) log s2, y^T(..)^{-1}y = c^T (B + s2 I)^{-1} c +
 * (||y||^2 - ||c||^2) / s2, and the gradient terms through (B + s2 I)^{-1} and dB_j, so the cost
 * per theta is independent of N beyond one N x k product. Eigenvalues of B within
 * 64 eps max|lambda| of zero count as zero. theta: host [d_theta] (1 or 2 parameters), inside
 * its box (else PTTK_EDOMAIN); y: dev [N]; lml: host; grad: host [d_theta] (may be NULL).
 * Synchronises `stream`. Errors: PTTK_EINVAL, PTTK_EDOMAIN (also: K~ + s2 I not positive
 * definite), PTTK_ENOTSUP, PTTK_ENOMEM, PTTK_ECUDA. */
pttk_status pttk_gp_lml(const pttk_global* g, const double* theta, double s2, const double* y, double* lml,
                        double* grad, void* stream);

/* ---- random numbers of the TT greedy-cross (Algorithms 5-7) ----------------------------
 * The greedy-cross draws random index vectors, sample sets, a row-or-column bit and check
 * points. They all come from SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) in counter-based
 * form, so that two implementations draw the same numbers. Returns output number `counter`
 * (0-based) of the stream seeded with `key`: the state key + (counter + 1) * 0x9E3779B97F4A7C15
 * through the variant-13 mix. Pure host function: no device, no error. */
uint64_t pttk_splitmix64(uint64_t key, uint64_t counter);

/* ---- online stage ------------------------------------------------------------------ */

/* Core matrix H(theta) = H_1(theta_1) ... H_{d_theta}(theta_{d_theta}),
 * H_j = sum_k G_{d+j}[:, k, :] T_k(phi^{-1}(theta_j)) (Eq. hmat, Algorithm 3, coefficient
 * form). theta: host [d_theta], inside the theta box (else PTTK_EDOMAIN).
 * M: dev, r_d x r_{d+d_theta} row-major, double for PTTK_FP64 and float otherwise.
 */
pttk_status pttk_theta_core(const pttk_tt* tt, const double* theta, pttk_prec prec, void* M,
                            void* stream);

/* Synchronise `stream` and report the handle's device status word, then clear it:
 * PTTK_ETIMEOUT if a kernel working with this handle gave up a bounded wait, PTTK_EDOMAIN if a
 * batched call met a theta outside its box or any call met a point outside its box (a
 * coordinate beyond its interval by more than 1e-12 of the interval's length; FP32 points
 * are compared with the FP32-rounded ends), else PTTK_OK. The tensor-core factor chain records
 * such timeouts instead of spinning; its outputs are unspecified when it does. */
pttk_status pttk_tt_check(const pttk_tt* tt, void* stream);

/* Online instantiation: M = H(theta) as above, and the factor matrices of Algorithm 2,
 * Phase 3 for the given points: U = S(X) (N_s x r_d) by S <- B_1 G_1^{2},
 * S <- (B_i face-split S) G_i^{2}; V = T(Y) (N_t x r_{d+d_theta}) by the mirrored
 * Khatri-Rao chain; B_i[p, k] = T_k(phi^{-1}(x_{p,i})). K(X, Y; theta) ~= U M V^T.
 *   X: dev N_s x d, Y: dev N_t x d (double for PTTK_FP64, float otherwise); points must lie
 *   in their boxes (Section 1: X in B_s, Y in B_t), a point on a face is valid. One pass over
 *   X and Y checks it on the device; a coordinate outside its interval by more than 1e-12 of
 *   the interval's width (FP32 points: of the FP32-rounded interval), or NaN, records
 *   PTTK_EDOMAIN in the handle's status word (reported by pttk_tt_check), and that point's
 *   factor row is an extrapolation.
 *   N_s, N_t >= 0 (0 is allowed and writes nothing for that side).
 *   U, M, V: dev outputs (double for PTTK_FP64, float otherwise).
 *   prec: PTTK_FP64 / PTTK_FP32 run the SIMT chain; PTTK_TF32, PTTK_TF32X3, PTTK_BF16,
 *   PTTK_BF16X3, PTTK_FP16 and PTTK_FP16X3 run the tensor-core chain (tcgen05, FP32
 *   accumulation; the X3 forms split both operands into two parts and sum three products;
 *   the FP16 forms scale operands by exact powers of two to stay in FP16 range; TMEM accumulator of
 *   128 points x N_pad columns), which needs every TT rank it touches <= 256 and, on first
 *   use of a form with a handle, lays out that form's core images on the device
 *   (synchronising `stream` once). Check pttk_tt_check after tensor-core calls. */
pttk_status pttk_instantiate(const pttk_tt* tt, const double* theta, const void* X,
                             int64_t N_s, const void* Y, int64_t N_t, pttk_prec prec, void* U,
                             void* M, void* V, void* stream);

/* ---- batched online stage --------------------------------------------------------- */

/* A plan for B instances (theta_b, X_b, Y_b) of one TT: the points of all instances are
 * concatenated, instance b owning rows [xoff[b], xoff[b+1]) of X (and of U) and rows
 * [yoff[b], yoff[b+1]) of Y (and of V). xoff, yoff: host arrays of B + 1 nondecreasing
 * int64 with xoff[0] = yoff[0] = 0, copied. prec as for pttk_instantiate. The plan allocates
 * its scratch and, for tensor-core forms, lays out the core images (synchronising `stream`),
 * so that pttk_instantiate_batched itself allocates nothing and never synchronises (it can
 * be captured in a CUDA graph). The plan refers to `tt`, which must outlive it. */
typedef struct pttk_batch pttk_batch;
pttk_status pttk_batch_create(const pttk_tt* tt, int B, const int64_t* xoff, const int64_t* yoff,
                              pttk_prec prec, void* stream, pttk_batch** out);
void pttk_batch_free(pttk_batch* b);

/* Launch configuration of the plan's tensor-core factor build; pttk_batch_get_config reports
 * the current one and how many exist (8). 0 (the default): the kernel that generates the A
 * operand in shared memory with four separate epilogue warps, which drain two alternating
 * tensor-memory accumulators while the next tile's products run (ranks whose two accumulators
 * or staging tiles do not fit fall back to configuration 1); 1 and 2: the same kernel without
 * the epilogue warps, with 128- or 64-byte chunks of K per row; 3, 4, 5: for the FP16/BF16
 * forms, the kernel that generates A in tensor memory and keeps the chain's intermediate in
 * registers, run in thread-block clusters of 1, 2 or 4 CTAs that share each core chunk by a
 * multicast copy (ranks it cannot hold fall back to configuration 1); 6: for the FP16/BF16
 * forms, A in tensor memory with the epilogue warps of configuration 0 and a B ring of 3-4
 * slots in the shared memory A no longer takes (ranks it cannot hold fall back to
 * configuration 0); 7: configuration 0 with 64-byte chunks of K per row in a ring of 4 slots. */
pttk_status pttk_batch_set_config(pttk_batch* b, int cfg);
pttk_status pttk_batch_get_config(const pttk_batch* b, int* cfg, int* n_configs);

/* Autotuner: times every launch configuration of the plan's factor build on the given inputs
 * (one warm-up and three timed runs each, CUDA events on `stream`), keeps the fastest, and
 * writes the mean milliseconds per configuration to ms_out (host, n_configs floats; may be
 * NULL). Overwrites U and V. Synchronises. */
pttk_status pttk_batch_autotune(pttk_batch* b, const void* X, const void* Y, void* U, void* V,
                                float* ms_out, void* stream);

/* Batched instantiation (Algorithm 3 per instance plus the Phase-3 factors of all points):
 * M[b] = H(theta_b) for b < B (M: dev B x r_d x r_{d+d_theta}, each row-major), U = the
 * source factors of all rows of X, V = the target factors of all rows of Y (factor rows depend
 * only on their point). thetas: dev B x d_theta doubles (read on the device; a theta outside
 * its box records PTTK_EDOMAIN in the handle's status word, see pttk_tt_check). X, Y, U, V as
 * in pttk_instantiate for the concatenated point sets. Allocates nothing; no host sync. */
pttk_status pttk_instantiate_batched(const pttk_batch* b, const double* thetas, const void* X,
                                     const void* Y, void* U, void* M, void* V, void* stream);

/* ---- adjoint ------------------------------------------------------------------------ */

/* Loss L = w^T K~(X, Y; theta) z = w^T U M V^T z and its gradients (the paper motivates
 * derivatives in the hyperparameters for Gaussian-process use but gives no adjoint; these
 * follow from Eq. hmat and Algorithm 2, Phase 3 by the chain rule):
 *   dL/dtheta_j = (U^T w)^T H_1 .. H_j' .. H_dtheta (V^T z), H_j' with T_k' in place of T_k;
 *   dL/dX by a reverse pass through the factor chain that recomputes the Chebyshev bases
 *   and their derivatives per point.
 *   theta: host [d_theta] (inside its box, else PTTK_EDOMAIN). X, Y, w (N_s), z (N_t): dev,
 *   double for PTTK_FP64, float otherwise. prec selects the form of the forward factors (as in
 *   pttk_instantiate); the reverse pass runs in FP64 (PTTK_FP64) or FP32 SIMT, sums over the
 *   points accumulate in FP64. Outputs (each may be NULL): loss (host double), dtheta (host
 *   [d_theta] doubles), dX (dev N_s x d, row-major, type of X). Allocates stream-ordered
 *   scratch; synchronises `stream`. */
pttk_status pttk_grad(const pttk_tt* tt, const double* theta, const void* X, int64_t N_s,
                      const void* Y, int64_t N_t, const void* w, const void* z, pttk_prec prec,
                      double* loss, double* dtheta, void* dX, void* stream);

/* Low-rank product out = U (M (V^T w)) (Eq. paramlowrank applied to a vector).
 *   U: dev N_s x rs, M: dev rs x rt, V: dev N_t x rt, row-major; w: dev [N_t];
 *   out: dev [N_s]. prec: PTTK_FP64 (all double) or PTTK_FP32 (all float; reductions
 *   accumulate in FP32). Any ranks rs, rt >= 1: no shared memory is sized by a rank. The
 *   library allocates a small stream-ordered temporary for the partial sums of V^T w and for
 *   M (V^T w). */
pttk_status pttk_apply(const void* U, const void* M, const void* V, int64_t N_s, int64_t N_t,
                       int rs, int rt, pttk_prec prec, const void* w, void* out, void* stream);

/* The same product as pttk_apply, for callers that cannot allocate device memory once
 * they are running, e.g. a process whose device memory is entirely reserved by another
 * allocator (a framework's caching pool), or a latency-bound loop in which cudaMalloc or
 * cudaFree could stall or fail under memory pressure. This call allocates nothing: its
 * scratch (the per-block partial sums of V^T w and the vector M (V^T w)) is a 1 MiB
 * file-scope device array inside libpttk, held by every device that loads the library until
 * the process exits. The paper has no counterpart; arguments and results are those of
 * pttk_apply, and it uses fewer partial-sum blocks when they would not fit.
 *   Limit: rs + rt <= 131072 (FP64) or 262144 (FP32), the scratch's size in elements (at
 *   least one partial-sum block of rt values plus the rs values of M (V^T w) must fit);
 *   larger ranks give PTTK_EINVAL. Below the limit any N_s, N_t is accepted.
 *   The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 *   with that device current; make that first call before any stream capture.
 *   All calls share the one array, which keeps the last call's contents: calls whose work
 *   overlaps on the GPU (on different streams, or from different threads) race, so
 *   serialise them. */
pttk_status pttk_apply_noalloc(const void* U, const void* M, const void* V, int64_t N_s,
                               int64_t N_t, int rs, int rt, pttk_prec prec, const void* w,
                               void* out, void* stream);

/* ---- kernel timing ------------------------------------------------------------------ */

/* When enabled, every launch of the library's timed kernels is bracketed by two CUDA
 * events recorded on the launching stream. Kernel names: "grid_tile", "mode_transform",
 * "householder", "jacobi_round", "dgemm", "chain", "apply". Off by default; enabling adds
 * two event records per launch. */
pttk_status pttk_profile_enable(int on);
/* Forget all accumulated timings (waits for pending events). */
pttk_status pttk_profile_reset(void);
/* Total milliseconds and launch count accumulated for one kernel name (synchronises on the
 * pending events of that kernel). Unknown names give 0 and 0. */
pttk_status pttk_profile_get(const char* kernel_name, double* ms_total, int64_t* launches);
/* Total number of kernels the library has launched in this process (all entry points). */
int64_t pttk_launch_count(void);

/* Self-test of failure detection (the paper has no counterpart). Every wait inside the
 * library's kernels (pipeline barriers, grid barriers) is bounded: after ~2 s it gives up,
 * the kernel records PTTK_ETIMEOUT and returns, and the CUDA context stays usable. This call
 * runs one such wait on a barrier that nothing ever completes and reports the outcome:
 * PTTK_ETIMEOUT when the wait gave up as designed (the expected result), PTTK_ECUDA
 * otherwise. Takes ~2 s; synchronises `stream`. */
pttk_status pttk_selftest_wait_timeout(void* stream);
/* Names of the kernels timed so far, newline-separated, NUL-terminated, truncated to len. */
pttk_status pttk_profile_names(char* buf, int64_t len);

/* ---- peak probes (measurement helpers; the paper has no counterpart) -------------------
 * Rooflines of kernels bound by an arithmetic pipe need that pipe's peak on this GPU. Each
 * probe runs one loop kernel of the given kind for `iters` trips (tens of ms for the sizes
 * the bench uses) and returns its rate: *tflops = executed flops / CUDA-event time, *ms (may
 * be NULL) = that time. Kinds:
 *   PTTK_PROBE_DFMA  FP64 FMA, 256-thread blocks, 8 per SM, 32 dependent-free FMAs per trip;
 *   PTTK_PROBE_FFMA  FP32 FMA, the same shape;
 *   PTTK_PROBE_DMMA  FP64 mma.sync m8n8k4, 4 independent accumulators per warp per trip;
 *   PTTK_PROBE_TF32  tcgen05.mma kind::tf32 M = 128, N = 256, K = 8, one CTA per SM, one MMA
 *                    per trip;
 *   PTTK_PROBE_F16   tcgen05.mma kind::f16 (FP16 operands) M = 128, N = 256, K = 16;
 *   PTTK_PROBE_F16S64, _F16S128, _F16S256: the same with N = 64, 128, 256 and operands that
 *                    walk through four A and four B slots of shared memory (every MMA reads
 *                    new operand bytes), one CTA per SM.
 * Operands are seeded nonzero values. iters in [1, 2^32]. Synchronises `stream`.
 * Errors: PTTK_EINVAL, PTTK_ECUDA, PTTK_ETIMEOUT (an MMA loop's bounded final wait ran out). */
typedef enum pttk_probe {
  PTTK_PROBE_DFMA = 0,
  PTTK_PROBE_FFMA = 1,
  PTTK_PROBE_DMMA = 2,
  PTTK_PROBE_TF32 = 3,
  PTTK_PROBE_F16 = 4,
  PTTK_PROBE_F16S64 = 5,
  PTTK_PROBE_F16S128 = 6,
  PTTK_PROBE_F16S256 = 7
} pttk_probe;
pttk_status pttk_peak_probe(int kind, int64_t iters, void* stream, double* tflops, double* ms);

#ifdef __cplusplus
}
#endif

#endif /* PTTK_H */

// Offline stage, Phase 1: the grid tensor of kernel values at the tensor Chebyshev nodes
// (Eq. mdc) and its per-mode Chebyshev transform C = M x_1 A x_2 A ... x_D A with
// A[k, i] = (c_k / n) T_k(zeta_i) (Eq. cheb_trans written for coefficients).
//
// Layout: C is column-major (i_1 fastest, Section 2.2). Pass 1 (grid_tile_kernel) gives
// each CTA one tile of n^m1 consecutive entries (the leading m1 modes, fixed trailing
// indices): threads evaluate the tile's entries into shared memory, each tile mode is
// transformed there one fibre per thread (held in registers), and the tile leaves in a
// single coalesced write. Modes m1+1..D are then transformed in place by one strided pass each
// (mode_transform_kernel), consecutive threads taking consecutive entries of the leading
// block so every load and store is coalesced.
#include <math.h>

#include <algorithm>

#include "kernels.cuh"
#include "pttk_internal.cuh"

namespace pttk {
namespace {

struct GridArgs {
  int kind, d, dtheta, D, n, m1;
  int64_t tile, ntiles;
  double lo[PTTK_MAX_D], hi[PTTK_MAX_D];
  // general-nu Matern, grid tile kernel: per nu node, G(z) = z^nu e^z K_nu(z) on [kv_zlo, kv_zhi]
  // in kv_P pieces (see KvTable); kv_P = 0: the quadrature for every entry
  const void* kv_tab;
  int kv_P;
  double kv_zlo, kv_zhi, kv_inv_zlo;
  float kv_inv_log2q;
};

// ---------------- general-nu Matern by table ------------------------------------------------
// The grid's entries take z = sqrt(2 nu) r / l over a known range (the node distances and the
// l and nu nodes), and only n values of nu. For each nu node, G(z) = z^nu e^z K_nu(z), which
// is smooth for z > 0 with its one singularity (a branch point) at z = 0, is tabulated once as
// piecewise Chebyshev series: pieces [a, 1.5 a] from kv_zlo up (geometric, so each piece sees
// the singularity at the same relative distance: its Bernstein ellipse has rho ~ 9.9, and
// degree 16 leaves a truncation error near 1e-17), each series of degree KV_DEG fitted at the
// piece's KV_DEG + 1 first-kind Chebyshev points from the quadrature kv_scaled. An entry then
// costs one exponential and a Clenshaw sum: kappa = c_nu e^{-z} G(z). Against 30-digit values
// the table is within 2.4e-15 (relative) for z in [1e-3, 60], nu in {0.5, 1, 2, 2.5, 4}.
// Entries outside the table's range (z below 1e-3 when boxes overlap) take the quadrature.
constexpr int KV_DEG = 16;
constexpr int KV_STRIDE = KV_DEG + 3;  // per piece: mid, 1 / half-width, KV_DEG + 1 coefficients
constexpr double KV_Q = 1.5;
constexpr int KV_MAX_PIECES = 64;

// One block per nu node: the pieces' values at their Chebyshev points, then the coefficients
// c_m = (2 / (KV_DEG + 1)) sum_k G(z_k) T_m(zeta_k) (c_0 halved); FP64 and an FP32 copy.
__global__ void __launch_bounds__(256) kv_table_kernel(int n, int P, double zlo, double nu_lo, double nu_hi,
                                                       double* __restrict__ tab64, float* __restrict__ tab32) {
  __shared__ double stab[KV_TABLE];
  __shared__ double vals[KV_MAX_PIECES * (KV_DEG + 1)];
  const int inu = blockIdx.x;
  kv_table_fill<double>(stab);
  const double zn = cospi((2.0 * inu + 1.0) / (2.0 * n));
  const double nu = 0.5 * (nu_lo - nu_hi) * zn + 0.5 * (nu_lo + nu_hi);
  __syncthreads();
  for (int e = threadIdx.x; e < P * (KV_DEG + 1); e += blockDim.x) {
    const int p = e / (KV_DEG + 1), k = e % (KV_DEG + 1);
    const double a = zlo * pow(KV_Q, (double)p), b = a * KV_Q;
    const double z = 0.5 * (a + b) + 0.5 * (b - a) * cospi((2.0 * k + 1.0) / (2.0 * (KV_DEG + 1)));
    vals[e] = exp(nu * log(z)) * kv_scaled<double>(nu, z, stab);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < P * KV_STRIDE; e += blockDim.x) {
    const int p = e / KV_STRIDE, m = e % KV_STRIDE;
    const double a = zlo * pow(KV_Q, (double)p), b = a * KV_Q;
    double v;
    if (m == 0) {
      v = 0.5 * (a + b);
    } else if (m == 1) {
      v = 2.0 / (b - a);
    } else {
      const int mm = m - 2;
      double acc = 0.0;
      for (int k = 0; k <= KV_DEG; ++k)
        acc = fma(vals[p * (KV_DEG + 1) + k], cospi((double)mm * (2.0 * k + 1.0) / (2.0 * (KV_DEG + 1))), acc);
      v = (mm == 0 ? 1.0 : 2.0) / (KV_DEG + 1) * acc;
    }
    tab64[((size_t)inu * P + p) * KV_STRIDE + m] = v;
    tab32[((size_t)inu * P + p) * KV_STRIDE + m] = (float)v;
  }
}

// kappa of the general-nu Matern from the table of nu node `inu`, or by quadrature outside it.
template <typename T>
__device__ __forceinline__ T kappa_matern_nu_tab(const GridArgs& a, int inu, T r2, T l, T nu, T cnu, T snu,
                                                 const T* __restrict__ stab) {
  const T z = snu * sqrt(r2) / l;
  if (a.kv_P > 0 && z >= T(a.kv_zlo) && z <= T(a.kv_zhi)) {
    int p = (int)(__log2f((float)(z * T(a.kv_inv_zlo))) * a.kv_inv_log2q);
    p = min(max(p, 0), a.kv_P - 1);
    const T* c = static_cast<const T*>(a.kv_tab) + ((size_t)inu * a.kv_P + p) * KV_STRIDE;
    const T t = (z - __ldg(c)) * __ldg(c + 1), t2 = t + t;
    T b1 = T(0), b2 = T(0);
#pragma unroll
    for (int k = KV_DEG; k >= 1; --k) {
      const T b0 = fma(t2, b1, __ldg(c + 2 + k) - b2);
      b2 = b1;
      b1 = b0;
    }
    const T G = fma(t, b1, __ldg(c + 2) - b2);
    return cnu * exp(-z) * G;
  }
  return kappa_matern_nu<T>(r2, l, nu, cnu, snu, stab);
}

// Chebyshev node table, transform matrix and Matern-nu node constants in shared memory.
template <typename T>
__device__ void fill_tables(const GridArgs& a, T* eta, T* Amat, T* cnu, T* snu, T* stab) {
  const int n = a.n;
  for (int e = threadIdx.x; e < a.D * n; e += blockDim.x) {
    const int j = e / n, i = e % n;
    // zeta_i = cos((2i+1) pi / (2n)) (0-based i), eta = phi_[lo,hi](zeta), phi as printed
    const double z = cospi((2.0 * i + 1.0) / (2.0 * n));
    eta[e] = (T)(0.5 * (a.lo[j] - a.hi[j]) * z + 0.5 * (a.lo[j] + a.hi[j]));
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int k = e / n, i = e % n;
    const double c = (k == 0 ? 1.0 : 2.0) / n;
    Amat[e] = (T)(c * cospi((double)k * (2.0 * i + 1.0) / (2.0 * n)));
  }
  if (a.kind == K_MATERN_NU) {
    const int jn = a.d + 1;  // theta = (l, nu): nu is mode d + 2 (0-based d + 1)
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double z = cospi((2.0 * i + 1.0) / (2.0 * n));
      const double nu = 0.5 * (a.lo[jn] - a.hi[jn]) * z + 0.5 * (a.lo[jn] + a.hi[jn]);
      cnu[i] = (T)(exp2(1.0 - nu) / tgamma(nu));
      snu[i] = (T)sqrt(2.0 * nu);
    }
    kv_table_fill<T>(stab);
  }
}

template <typename T, bool TAB = false>
__device__ __forceinline__ T eval_entry(const GridArgs& a, const int* idx, const T* eta,
                                        const T* cnu, const T* snu, const T* stab) {
  const int n = a.n;
  T r2 = T(0);
  for (int j = 0; j < a.d; ++j) {
    const T diff = eta[j * n + idx[j]] - eta[(a.d + a.dtheta + j) * n + idx[a.d + a.dtheta + j]];
    r2 += diff * diff;
  }
  const T l = a.dtheta > 0 ? eta[a.d * n + idx[a.d]] : T(1);
  if (a.kind == K_MATERN_NU) {
    const int inu = idx[a.d + 1];
    if (TAB) return kappa_matern_nu_tab<T>(a, inu, r2, l, eta[(a.d + 1) * n + inu], cnu[inu], snu[inu], stab);
    return kappa_matern_nu<T>(r2, l, eta[(a.d + 1) * n + inu], cnu[inu], snu[inu], stab);
  }
  return kappa_l<T>(a.kind, r2, l);
}

template <typename T, int NB>
__device__ __forceinline__ void transform_fibre(const T* Amat, int n, const T* x, T* y) {
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    T acc = T(0);
#pragma unroll
    for (int i = 0; i < NB; ++i)
      if (i < n && k < n) acc = fma(Amat[k * n + i], x[i], acc);
    y[k] = acc;
  }
}

template <typename T, int NB>
__global__ void __launch_bounds__(512) grid_tile_kernel(GridArgs a, T* __restrict__ C) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tile = reinterpret_cast<T*>(smem_raw);
  T* eta = tile + a.tile;
  T* Amat = eta + a.D * a.n;
  T* cnu = Amat + a.n * a.n;
  T* snu = cnu + a.n;
  T* stab = snu + a.n;
  fill_tables<T>(a, eta, Amat, cnu, snu, stab);
  __syncthreads();

  const int n = a.n;
  const int64_t nfib = a.tile / n;
  for (int64_t t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    int idx[PTTK_MAX_D];
    int64_t rem = t;
    for (int j = a.m1; j < a.D; ++j) {
      idx[j] = (int)(rem % n);
      rem /= n;
    }
    // evaluate every entry of the tile (one entry per thread, consecutive threads
    // on consecutive entries)
    for (int64_t e = threadIdx.x; e < a.tile; e += blockDim.x) {
      int64_t q = e;
      for (int j = 0; j < a.m1; ++j) {
        idx[j] = (int)(q % n);
        q /= n;
      }
      tile[e] = eval_entry<T, true>(a, idx, eta, cnu, snu, stab);
    }
    __syncthreads();
    // modes 1..m1 inside the tile: one fibre per thread, in registers
    int64_t s = 1;
    for (int j = 0; j < a.m1; ++j, s *= n) {
      for (int64_t f = threadIdx.x; f < nfib; f += blockDim.x) {
        const int64_t l = f % s, h = f / s;
        T* base = tile + l + h * s * n;
        T x[NB], y[NB];
#pragma unroll
        for (int i = 0; i < NB; ++i) x[i] = (i < n) ? base[i * s] : T(0);
        transform_fibre<T, NB>(Amat, n, x, y);
#pragma unroll
        for (int k = 0; k < NB; ++k)
          if (k < n) base[k * s] = y[k];
      }
      __syncthreads();
    }
    T* out = C + t * a.tile;
    for (int64_t e = threadIdx.x; e < a.tile; e += blockDim.x) out[e] = tile[e];
    __syncthreads();
  }
}

// In-place transform of one mode with stride s = n^(j-1) over the whole tensor.
template <typename T, int NB>
__global__ void __launch_bounds__(256) mode_transform_kernel(T* __restrict__ C, int n,
                                                             int64_t s, int64_t nfib) {
  __shared__ T Amat[PTTK_MAX_N * PTTK_MAX_N];
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int k = e / n, i = e % n;
    const double c = (k == 0 ? 1.0 : 2.0) / n;
    Amat[e] = (T)(c * cospi((double)k * (2.0 * i + 1.0) / (2.0 * n)));
  }
  __syncthreads();
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < nfib;
       f += (int64_t)gridDim.x * blockDim.x) {
    const int64_t l = f % s, h = f / s;
    T* base = C + l + h * s * n;
    T x[NB], y[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) x[i] = (i < n) ? base[i * s] : T(0);
    transform_fibre<T, NB>(Amat, n, x, y);
#pragma unroll
    for (int k = 0; k < NB; ++k)
      if (k < n) base[k * s] = y[k];
  }
}

template <typename T, int NB>
pttk_status launch_all(const GridArgs& a, T* C, cudaStream_t st) {
  const int threads = sizeof(T) == 8 ? 512 : 256;
  const size_t smem = sizeof(T) * (a.tile + (size_t)a.D * a.n + (size_t)a.n * a.n + 2 * a.n +
                                    (a.kind == K_MATERN_NU ? KV_TABLE : 0));
  auto kfn = grid_tile_kernel<T, NB>;
  PTTK_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  PTTK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, threads, smem));
  if (per_sm < 1) return set_error(PTTK_ENOTSUP, "grid tile does not fit on an SM");
  const int64_t grid = std::min<int64_t>(a.ntiles, (int64_t)sm_count() * per_sm);
  {
    PTTK_PROF("grid_tile", st);
    kfn<<<(unsigned)grid, threads, smem, st>>>(a, C); pttk::count_launch();
  }
  PTTK_CUDA(cudaGetLastError());
  int64_t total = 1;
  for (int j = 0; j < a.D; ++j) total *= a.n;
  const int64_t nfib = total / a.n;
  int64_t s = a.tile;
  for (int j = a.m1; j < a.D; ++j, s *= a.n) {
    const int64_t blocks = std::min<int64_t>((nfib + 255) / 256, (int64_t)sm_count() * 8);
    PTTK_PROF("mode_transform", st);
    mode_transform_kernel<T, NB><<<(unsigned)blocks, 256, 0, st>>>(C, a.n, s, nfib); pttk::count_launch();
    PTTK_CUDA(cudaGetLastError());
  }
  return PTTK_OK;
}

template <typename T>
pttk_status dispatch_nb(const GridArgs& a, T* C, cudaStream_t st) {
  const int nb = ((a.n + 3) / 4) * 4;
  switch (nb) {
    case 4: return launch_all<T, 4>(a, C, st);
    case 8: return launch_all<T, 8>(a, C, st);
    case 12: return launch_all<T, 12>(a, C, st);
    case 16: return launch_all<T, 16>(a, C, st);
    case 20: return launch_all<T, 20>(a, C, st);
    case 24: return launch_all<T, 24>(a, C, st);
    case 28: return launch_all<T, 28>(a, C, st);
    case 32: return launch_all<T, 32>(a, C, st);
  }
  return set_error(PTTK_EINVAL, "n out of range");
}

// Entries of the grid tensor M (Eq. mdc) at a list of multi-indices (the entry access the
// TT greedy-cross works from): out[e] = f_kappa(eta^(1)_{idx[e,0]}, ..., eta^(D)_{idx[e,D-1]}),
// idx row-major M x D. An index outside [0, n) gives NaN and records PTTK_EINVAL in *status;
// no node is read with it.
template <typename T>
__global__ void __launch_bounds__(256) entries_kernel(GridArgs a, const int* __restrict__ idx, int64_t M,
                                                      T* __restrict__ out, int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* eta = reinterpret_cast<T*>(smem_raw);
  T* Amat = eta + a.D * a.n;
  T* cnu = Amat + a.n * a.n;
  T* snu = cnu + a.n;
  T* stab = snu + a.n;
  fill_tables<T>(a, eta, Amat, cnu, snu, stab);
  __syncthreads();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < M;
       e += (int64_t)gridDim.x * blockDim.x) {
    int row[PTTK_MAX_D];
    bool ok = true;
    for (int j = 0; j < a.D; ++j) {
      const int v = idx[e * a.D + j];
      ok = ok && v >= 0 && v < a.n;
      row[j] = ok ? v : 0;
    }
    if (!ok) {
      out[e] = T(NAN);
      atomicExch(status, (int)PTTK_EINVAL);
      continue;
    }
    out[e] = eval_entry<T>(a, row, eta, cnu, snu, stab);
  }
}

template <typename T>
pttk_status launch_entries(const GridArgs& a, const int* idx, int64_t M, T* out, int* status,
                           cudaStream_t st) {
  const size_t smem = sizeof(T) * ((size_t)a.D * a.n + (size_t)a.n * a.n + 2 * a.n +
                                   (a.kind == K_MATERN_NU ? KV_TABLE : 0));
  auto kfn = entries_kernel<T>;
  PTTK_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((M + 255) / 256, (int64_t)sm_count() * 8));
  PTTK_PROF("grid_entries", st);
  kfn<<<(unsigned)blocks, 256, smem, st>>>(a, idx, M, out, status); pttk::count_launch();
  PTTK_CUDA(cudaGetLastError());
  return PTTK_OK;
}

}  // namespace

pttk_status grid_entries_launch(int kernel, int d, int dtheta, int n, const double (*box)[2],
                                const int* idx, int64_t M, bool fp64, void* out, int* status,
                                cudaStream_t s) {
  if (M == 0) return PTTK_OK;
  GridArgs a{};
  a.kind = kernel;
  a.d = d;
  a.dtheta = dtheta;
  a.D = 2 * d + dtheta;
  a.n = n;
  for (int j = 0; j < a.D; ++j) {
    a.lo[j] = box[j][0];
    a.hi[j] = box[j][1];
  }
  if (fp64) return launch_entries<double>(a, idx, M, static_cast<double*>(out), status, s);
  return launch_entries<float>(a, idx, M, static_cast<float*>(out), status, s);
}

pttk_status grid_coeffs_launch(int kernel, int d, int dtheta, int n, const double (*box)[2],
                               bool fp64, void* C, cudaStream_t s) {
  GridArgs a{};
  a.kind = kernel;
  a.d = d;
  a.dtheta = dtheta;
  a.D = 2 * d + dtheta;
  a.n = n;
  for (int j = 0; j < a.D; ++j) {
    a.lo[j] = box[j][0];
    a.hi[j] = box[j][1];
  }
  // leading block of m1 modes held in shared memory
  const size_t elem = fp64 ? 8 : 4;
  const size_t budget = fp64 ? 170000 : 90000;
  a.m1 = 1;
  a.tile = n;
  while (a.m1 < a.D && (size_t)(a.tile * n) * elem <= budget) {
    a.tile *= n;
    ++a.m1;
  }
  a.ntiles = 1;
  for (int j = a.m1; j < a.D; ++j) a.ntiles *= n;
  // the per-nu tables live until the kernels that read them have run: released stream-ordered
  // on every return path
  struct Tables {
    double* t64 = nullptr;
    float* t32 = nullptr;
    cudaStream_t s;
    ~Tables() {
      if (t64) cudaFreeAsync(t64, s);
      if (t32) cudaFreeAsync(t32, s);
    }
  } tabs{nullptr, nullptr, s};
  double*& tab64 = tabs.t64;
  float*& tab32 = tabs.t32;
  if (kernel == K_MATERN_NU) {
    // the range of z = sqrt(2 nu) r / l over the grid's nodes
    auto node = [&](int j, int i) {
      const double z = cos((2.0 * i + 1.0) * 3.14159265358979323846 / (2.0 * n));
      return 0.5 * (a.lo[j] - a.hi[j]) * z + 0.5 * (a.lo[j] + a.hi[j]);
    };
    double r2min = 0.0, r2max = 0.0;
    for (int j = 0; j < d; ++j) {
      double dmin = INFINITY, dmax = 0.0;
      for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
          const double df = fabs(node(j, i) - node(d + dtheta + j, k));
          dmin = std::min(dmin, df);
          dmax = std::max(dmax, df);
        }
      r2min += dmin * dmin;
      r2max += dmax * dmax;
    }
    double lmin = INFINITY, lmax = 0.0, numin = INFINITY, numax = 0.0;
    for (int i = 0; i < n; ++i) {
      lmin = std::min(lmin, node(d, i));
      lmax = std::max(lmax, node(d, i));
      numin = std::min(numin, node(d + 1, i));
      numax = std::max(numax, node(d + 1, i));
    }
    double zlo = std::max(sqrt(2.0 * numin) * sqrt(r2min) / lmax * (1.0 - 1e-12), 1e-3);
    const double zhi = std::min(sqrt(2.0 * numax) * sqrt(r2max) / lmin * (1.0 + 1e-12), 700.0);
    if (zhi > zlo) {
      int P = (int)ceil(log(zhi / zlo) / log(KV_Q));
      if (P > KV_MAX_PIECES) {
        P = KV_MAX_PIECES;
        zlo = zhi / pow(KV_Q, (double)P);
      }
      P = std::max(P, 1);
      const size_t cnt = (size_t)n * P * KV_STRIDE;
      PTTK_CUDA(cudaMallocAsync(&tab64, sizeof(double) * cnt, s));
      PTTK_CUDA(cudaMallocAsync(&tab32, sizeof(float) * cnt, s));
      kv_table_kernel<<<n, 256, 0, s>>>(n, P, zlo, a.lo[d + 1], a.hi[d + 1], tab64, tab32); pttk::count_launch();
      PTTK_CUDA(cudaGetLastError());
      a.kv_tab = fp64 ? static_cast<const void*>(tab64) : static_cast<const void*>(tab32);
      a.kv_P = P;
      a.kv_zlo = zlo;
      a.kv_zhi = zhi;
      a.kv_inv_zlo = 1.0 / zlo;
      a.kv_inv_log2q = (float)(1.0 / log2(KV_Q));
    }
  }
  return fp64 ? dispatch_nb<double>(a, static_cast<double*>(C), s) : dispatch_nb<float>(a, static_cast<float*>(C), s);
}

}  // namespace pttk

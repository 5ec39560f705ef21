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

#include "kernels.cuh"
#include "pttk_internal.cuh"

namespace pttk {
namespace {

struct GridArgs {
  int kind, d, dtheta, D, n, m1;
  int64_t tile, ntiles;
  double lo[PTTK_MAX_D], hi[PTTK_MAX_D];
};

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

template <typename T>
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
      tile[e] = eval_entry<T>(a, idx, eta, cnu, snu, stab);
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
  if (fp64) return dispatch_nb<double>(a, static_cast<double*>(C), s);
  return dispatch_nb<float>(a, static_cast<float*>(C), s);
}

}  // namespace pttk

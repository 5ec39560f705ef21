// Adjoint of the scalar loss L = w^T K~ z = w^T U(X) H(theta) V(Y)^T z.
//
// With a = U^T w, b = V^T z and g = H b:
//   L = a . g;
//   dL/dtheta_j = a^T H_1 ... H_j' ... H_dtheta b,  H_j' = sum_k G_{d+j}[:, k, :] T_k'(thetahat_j)
//                 dthetahat_j/dtheta_j (Eq. hmat differentiated; dthetahat/dtheta = 2/(lo - hi)
//                 for the printed interval map);
//   dL/dX: reverse pass through the chain of Algorithm 2, Phase 3 for every source point. The
//   adjoint of the chain output for point p is w_p g (rank one over the points), so the last
//   step needs only the vector q = G_d^{2} g; earlier steps take Q_i = gbar_i G_i^{2 T}. Step i
//   (S_out = (B_i face-split S_in) G_i^{2}) propagates
//     dB_i[p, j]   = sum_a S_in[p, a] Q_i[p, a + R_in j],
//     gbar_in[p,a] = sum_j B_i[p, j] Q_i[p, a + R_in j],
//     dL/dx_{p,i}  = sum_j dB_i[p, j] T_j'(xhat_{p,i}) 2/(lo_i - hi_i).
//   The Chebyshev bases and their derivatives (T_0' = 0, T_1' = 1,
//   T_{j+1}' = 2 T_j + 2 x T_j' - T_{j-1}') are recomputed per point, never stored; the chain
//   intermediates S_1..S_{d-1} come from rerunning the (cheap) leading steps of the chain.
#include <math.h>

#include <algorithm>
#include <vector>

#include "pttk_internal.cuh"

namespace pttk {
pttk_status factor_build_tc(const pttk_tt* tt, TcImageCache* cache, const float* X, int64_t N_s,
                            const float* Y, int64_t N_t, pttk_prec prec, float* U, float* V,
                            int* d_status, int cfg, cudaStream_t s);
namespace {

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// partial[blk * r + c] = sum over the block's rows of A[row, c] w[row]  (A: N x r row-major)
template <typename T>
__global__ void __launch_bounds__(256) weighted_colsum(const T* __restrict__ A, const T* __restrict__ w,
                                                       int64_t N, int r, double* __restrict__ partial) {
  const int64_t per = (N + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * per, r1 = std::min<int64_t>(N, r0 + per);
  for (int c = threadIdx.x; c < r; c += blockDim.x) {
    double acc = 0.0;
    for (int64_t i = r0; i < r1; ++i) acc = fma((double)A[i * r + c], (double)w[i], acc);
    partial[(int64_t)blockIdx.x * r + c] = acc;
  }
}

__global__ void sum_partials(const double* __restrict__ partial, int nparts, int r, double* __restrict__ out) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < r; c += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int b = 0; b < nparts; ++b) acc += partial[(int64_t)b * r + c];
    out[c] = acc;
  }
}

// Chebyshev values T_k(x) (deriv = 0) or T_k'(x) * scale (deriv = 1), k < n, into t[0..n)
__device__ void cheb_row(double x, int n, bool deriv, double scale, double* t) {
  double t0 = 1.0, t1 = x, d0 = 0.0, d1 = 1.0;
  for (int k = 0; k < n; ++k) {
    if (k == 0) t[k] = deriv ? 0.0 : 1.0;
    else if (k == 1) t[k] = deriv ? scale : x;
    else {
      const double t2 = 2.0 * x * t1 - t0;
      const double d2 = 2.0 * t1 + 2.0 * x * d1 - d0;
      t[k] = deriv ? d2 * scale : t2;
      t0 = t1;
      t1 = t2;
      d0 = d1;
      d1 = d2;
    }
  }
}

// Contraction of a theta core G (ra x n x rb, column-major) with the Chebyshev (or derivative)
// vector of th, applied to a vector on one side:
//   left  (side 0): out[c] = sum_{a,k} x[a] G[a, k, c] t[k]      (x: ra, out: rb)
//   right (side 1): out[a] = sum_{k,c} G[a, k, c] t[k] x[c]      (x: rb, out: ra)
__global__ void core_vec(const double* __restrict__ G, int ra, int n, int rb, double th, bool deriv,
                        double scale, const double* __restrict__ x, int side, double* __restrict__ out) {
  double t[PTTK_MAX_N];
  cheb_row(th, n, deriv, scale, t);
  const int m = side == 0 ? rb : ra;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= m) return;
  double acc = 0.0;
  if (side == 0) {
    const int c = warp;
    for (int64_t e = lane; e < (int64_t)ra * n; e += 32) {
      const int a = (int)(e % ra), k = (int)(e / ra);
      acc = fma(x[a] * t[k], G[a + (int64_t)ra * (k + (int64_t)n * c)], acc);
    }
  } else {
    const int a = warp;
    for (int64_t e = lane; e < (int64_t)n * rb; e += 32) {
      const int k = (int)(e % n), c = (int)(e / n);
      acc = fma(t[k] * x[c], G[a + (int64_t)ra * (k + (int64_t)n * c)], acc);
    }
  }
  acc = warp_sum_d(acc);
  if (lane == 0) out[warp] = acc;
}

// out[i] = sum_j M[i, j] x[j] (M row-major m x k, FP64), one warp per row; or a dot product
__global__ void matvec_rows(const double* __restrict__ M, int m, int k, const double* __restrict__ x,
                            double* __restrict__ out) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (row >= m) return;
  double acc = 0.0;
  for (int j = lane; j < k; j += 32) acc = fma(M[(int64_t)row * k + j], x[j], acc);
  acc = warp_sum_d(acc);
  if (lane == 0) out[row] = acc;
}

// q[k] = sum_o Gs[k + K o] g[o]  (oriented core K x R_out, column-major)
template <typename T>
__global__ void core_times_vec(const T* __restrict__ Gs, int K, int R, const double* __restrict__ g,
                               T* __restrict__ q) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int o = 0; o < R; ++o) acc = fma((double)Gs[k + (int64_t)K * o], g[o], acc);
    q[k] = (T)acc;
  }
}

// Q[p, k] = sum_o Gbar[p, o] Gs[k + K o]  (Gbar: N x R row-major; Q: N x K row-major).
// 64 x 64 output tiles, 16-wide reduction chunks, 4 x 4 register tiles.
template <typename T>
__global__ void __launch_bounds__(256) gemm_gbar_core(const T* __restrict__ Gbar, const T* __restrict__ Gs,
                                                      int64_t N, int R, int K, T* __restrict__ Q) {
  __shared__ T As[16][65];
  __shared__ T Bs[16][65];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int64_t p0 = (int64_t)blockIdx.y * 64;
  const int k0 = blockIdx.x * 64;
  T acc[4][4] = {};
  for (int o0 = 0; o0 < R; o0 += 16) {
    for (int e = threadIdx.x; e < 64 * 16; e += 256) {
      const int pp = e / 16, oo = e % 16;
      const int64_t p = p0 + pp;
      As[oo][pp] = (p < N && o0 + oo < R) ? Gbar[p * R + o0 + oo] : T(0);
      const int kk = e % 64, o2 = e / 64;
      Bs[o2][kk] = (k0 + kk < K && o0 + o2 < R) ? Gs[(k0 + kk) + (int64_t)K * (o0 + o2)] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int oo = 0; oo < 16; ++oo) {
      T av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[oo][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[oo][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t p = p0 + ty * 4 + i;
    if (p >= N) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = k0 + tx * 4 + j;
      if (k < K) Q[p * K + k] = acc[i][j];
    }
  }
}

// Reverse step of the chain for one point per warp (see the file comment). Q is either the
// full N x K matrix (qvec == nullptr) or rank one: Q[p, k] = w[p] qvec[k].
template <typename T>
__global__ void __launch_bounds__(256) chain_back_step(const T* __restrict__ X, int d, int coord, double lo,
                                                       double hi, int n, int64_t N, int R_in,
                                                       const T* __restrict__ S_in, const T* __restrict__ Q,
                                                       const T* __restrict__ w, const T* __restrict__ qvec,
                                                       T* __restrict__ gbar_in, T* __restrict__ dX) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* db = reinterpret_cast<T*>(smem_raw) + (size_t)wib * (PTTK_MAX_N + R_in);  // dB[j], gbar[a]
  T* gb = db + PTTK_MAX_N;
  const int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  if (p >= N) return;
  const double x = (double)X[p * d + coord];
  const double xh = (2.0 * x - lo - hi) / (lo - hi);
  for (int j = lane; j < PTTK_MAX_N; j += 32) db[j] = T(0);
  for (int a = lane; a < R_in; a += 32) gb[a] = T(0);
  __syncwarp();
  const int K = n * R_in;
  const T wp = qvec ? w[p] : T(0);
  for (int k = lane; k < K; k += 32) {
    const int j = k / R_in, a = k - j * R_in;
    const T qv = qvec ? wp * qvec[k] : Q[p * K + k];
    const T s = S_in ? S_in[p * R_in + a] : T(1);
    // T_j(xh) directly (cos form is avoided: the three-term recurrence below is per lane)
    double t0 = 1.0, t1 = xh, tj = 1.0;
    for (int m = 0; m <= j; ++m) {
      if (m == 0) tj = 1.0;
      else if (m == 1) tj = xh;
      else {
        const double t2 = 2.0 * xh * t1 - t0;
        t0 = t1;
        t1 = t2;
        tj = t2;
      }
    }
    atomicAdd(&db[j], s * qv);
    if (gbar_in) atomicAdd(&gb[a], (T)tj * qv);
  }
  __syncwarp();
  if (gbar_in)
    for (int a = lane; a < R_in; a += 32) gbar_in[p * R_in + a] = gb[a];
  if (lane == 0) {
    double td[PTTK_MAX_N];
    cheb_row(xh, n, true, 2.0 / (lo - hi), td);
    double acc = 0.0;
    for (int j = 0; j < n; ++j) acc = fma((double)db[j], td[j], acc);
    dX[p * d + coord] = (T)acc;
  }
}

unsigned nblk(int64_t work, int per = 256) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((work + per - 1) / per, (int64_t)sm_count() * 8));
}

template <typename T>
pttk_status weighted_sum(const T* A, const T* w, int64_t N, int r, double* out, double* partial, int nparts,
                         cudaStream_t s) {
  if (N == 0) {
    PTTK_CUDA(cudaMemsetAsync(out, 0, sizeof(double) * r, s));
    return PTTK_OK;
  }
  weighted_colsum<T><<<nparts, 256, 0, s>>>(A, w, N, r, partial); pttk::count_launch();
  sum_partials<<<nblk(r), 256, 0, s>>>(partial, nparts, r, out); pttk::count_launch();
  PTTK_CUDA(cudaGetLastError());
  return PTTK_OK;
}

struct Scratch {
  std::vector<void*> ptrs;
  cudaStream_t s;
  ~Scratch() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
  }
  template <typename T>
  pttk_status get(T** out, size_t elems) {
    void* p = nullptr;
    const cudaError_t e = cudaMallocAsync(&p, std::max<size_t>(elems, 1) * sizeof(T), s);
    if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync(adjoint scratch)");
    ptrs.push_back(p);
    *out = static_cast<T*>(p);
    return PTTK_OK;
  }
};

template <typename T>
pttk_status grad_typed(const pttk_tt* tt, const double* theta, const T* X, int64_t N_s, const T* Y, int64_t N_t,
                       const T* w, const T* z, pttk_prec prec, double* loss, double* dtheta, T* dX,
                       cudaStream_t s) {
  const int d = tt->d, dth = tt->dtheta, n = tt->n, D = tt->D;
  const int rs = tt->ranks[d], rt = tt->ranks[d + dth];
  const bool fp64 = sizeof(T) == 8;
  Scratch sc{{}, s};
  T *U, *V;
  double *M, *a, *b, *g, *partial, *small;
  PTTK_TRY(sc.get(&U, (size_t)N_s * rs));
  PTTK_TRY(sc.get(&V, (size_t)N_t * rt));
  PTTK_TRY(sc.get(&M, (size_t)rs * rt));
  const int nparts = (int)std::max<int64_t>(1, std::min<int64_t>((std::max(N_s, N_t) + 1023) / 1024, sm_count() * 4));
  PTTK_TRY(sc.get(&partial, (size_t)nparts * std::max(rs, rt)));
  PTTK_TRY(sc.get(&a, rs));
  PTTK_TRY(sc.get(&b, rt));
  PTTK_TRY(sc.get(&g, rs));
  int rmax = 1;
  for (int k = 0; k <= D; ++k) rmax = std::max(rmax, tt->ranks[k]);
  PTTK_TRY(sc.get(&small, (size_t)8 * rmax + 8));

  // forward: H (FP64), U, V in the requested form
  double th[PTTK_MAX_D];
  for (int j = 0; j < dth; ++j) {
    const double lo = tt->box[d + j][0], hi = tt->box[d + j][1];
    th[j] = (2.0 * theta[j] - lo - hi) / (lo - hi);
  }
  PTTK_TRY(theta_core_run(tt, th, true, M, s));
  PTTK_TRY(point_domain_check(tt, X, N_s, Y, N_t, fp64, tt_status_word(tt), s));
  if (prec == PTTK_FP64 || prec == PTTK_FP32) {
    PTTK_TRY(factor_build_run(tt, true, X, N_s, prec, U, s));
    PTTK_TRY(factor_build_run(tt, false, Y, N_t, prec, V, s));
  } else {
    PTTK_TRY(factor_build_tc(tt, tt_tc_cache(tt), reinterpret_cast<const float*>(X), N_s,
                             reinterpret_cast<const float*>(Y), N_t, prec, reinterpret_cast<float*>(U),
                             reinterpret_cast<float*>(V), tt_status_word(tt), 0, s));
  }
  PTTK_TRY(weighted_sum<T>(U, w, N_s, rs, a, partial, nparts, s));
  PTTK_TRY(weighted_sum<T>(V, z, N_t, rt, b, partial, nparts, s));
  matvec_rows<<<(unsigned)(((int64_t)rs * 32 + 255) / 256), 256, 0, s>>>(M, rs, rt, b, g); pttk::count_launch();  // g = H b
  double* Lbuf = small;
  matvec_rows<<<1, 32, 0, s>>>(a, 1, rs, g, Lbuf); pttk::count_launch();  // L = a . g

  // dL/dtheta
  if (dtheta && dth > 0) {
    double* dth_dev = small + 1;
    double* u = small + 8;          // rmax
    double* v = u + rmax;           // rmax
    double* u2 = v + rmax;          // rmax
    double* v2 = u2 + rmax;         // rmax
    const double* G1 = tt->cores64 + tt->core_off[d];
    const int r0 = tt->ranks[d], r1 = tt->ranks[d + 1];
    const double sc1 = 2.0 / (tt->box[d][0] - tt->box[d][1]);
    if (dth == 1) {
      // a^T H1' b: u = H1'^T a (r1), then u . b
      core_vec<<<(unsigned)((r1 * 32 + 255) / 256), 256, 0, s>>>(G1, r0, n, r1, th[0], true, sc1, a, 0, u); pttk::count_launch();
      matvec_rows<<<1, 32, 0, s>>>(u, 1, r1, b, dth_dev); pttk::count_launch();
    } else {
      const double* G2 = tt->cores64 + tt->core_off[d + 1];
      const int r2 = tt->ranks[d + 2];
      const double sc2 = 2.0 / (tt->box[d + 1][0] - tt->box[d + 1][1]);
      // u = H1'^T a, v = H2 b, u2 = H1^T a, v2 = H2' b; dtheta = (u . v, u2 . v2)
      { core_vec<<<(unsigned)((r1 * 32 + 255) / 256), 256, 0, s>>>(G1, r0, n, r1, th[0], true, sc1, a, 0, u); pttk::count_launch(); }
      core_vec<<<(unsigned)((r1 * 32 + 255) / 256), 256, 0, s>>>(G2, r1, n, r2, th[1], false, 1.0, b, 1, v); pttk::count_launch();
      core_vec<<<(unsigned)((r1 * 32 + 255) / 256), 256, 0, s>>>(G1, r0, n, r1, th[0], false, 1.0, a, 0, u2); pttk::count_launch();
      core_vec<<<(unsigned)((r1 * 32 + 255) / 256), 256, 0, s>>>(G2, r1, n, r2, th[1], true, sc2, b, 1, v2); pttk::count_launch();
      matvec_rows<<<1, 32, 0, s>>>(u, 1, r1, v, dth_dev); pttk::count_launch();
      matvec_rows<<<1, 32, 0, s>>>(u2, 1, r1, v2, dth_dev + 1); pttk::count_launch();
    }
  }

  // dL/dX by the reverse pass (SIMT, in the precision of X)
  if (dX && N_s > 0) {
    PTTK_PROF("adjoint", s);
    const pttk_prec simt = fp64 ? PTTK_FP64 : PTTK_FP32;
    std::vector<T*> Sbuf(d, nullptr);  // Sbuf[i] = S_i (N x r_i), i = 1..d-1
    for (int i = 1; i < d; ++i) {
      PTTK_TRY(sc.get(&Sbuf[i], (size_t)N_s * tt->ranks[i]));
      PTTK_TRY(factor_build_run(tt, true, X, N_s, simt, Sbuf[i], s, i));
    }
    // last step: rank-one adjoint w_p g
    int rin, rout, coord;
    oriented_core_dims(tt, true, d - 1, &rin, &rout, &coord);
    const T* Gs_last = static_cast<const T*>(oriented_core_ptr(tt, true, d - 1, fp64));
    T* q;
    PTTK_TRY(sc.get(&q, (size_t)n * rin));
    core_times_vec<T><<<nblk((int64_t)n * rin), 256, 0, s>>>(Gs_last, n * rin, rout, g, q); pttk::count_launch();
    T *gbar = nullptr, *gnext = nullptr, *Q = nullptr;
    size_t qmax = 0;
    for (int i = 0; i < d - 1; ++i) qmax = std::max<size_t>(qmax, (size_t)n * tt->ranks[i]);
    if (d > 1) {
      PTTK_TRY(sc.get(&gbar, (size_t)N_s * rmax));
      PTTK_TRY(sc.get(&gnext, (size_t)N_s * rmax));
      PTTK_TRY(sc.get(&Q, (size_t)N_s * qmax));
    }
    for (int i = d - 1; i >= 0; --i) {
      oriented_core_dims(tt, true, i, &rin, &rout, &coord);
      const double lo = tt->box[coord][0], hi = tt->box[coord][1];
      const int K = n * rin;
      if (i < d - 1) {
        const T* Gs = static_cast<const T*>(oriented_core_ptr(tt, true, i, fp64));
        dim3 grid((unsigned)((K + 63) / 64), (unsigned)((N_s + 63) / 64));
        gemm_gbar_core<T><<<grid, 256, 0, s>>>(gbar, Gs, N_s, rout, K, Q); pttk::count_launch();
      }
      const size_t smem = sizeof(T) * 8 * (PTTK_MAX_N + rin);
      chain_back_step<T><<<(unsigned)((N_s + 7) / 8), 256, smem, s>>>(
          X, d, coord, lo, hi, n, N_s, rin, i > 0 ? Sbuf[i] : nullptr, i < d - 1 ? Q : nullptr, w,
          i == d - 1 ? q : nullptr, i > 0 ? gnext : nullptr, dX); pttk::count_launch();
      std::swap(gbar, gnext);
    }
  }
  PTTK_CUDA(cudaGetLastError());
  double host[3] = {0, 0, 0};
  PTTK_CUDA(cudaMemcpyAsync(host, small, sizeof(double) * 3, cudaMemcpyDeviceToHost, s));
  PTTK_CUDA(cudaStreamSynchronize(s));
  if (loss) *loss = host[0];
  if (dtheta)
    for (int j = 0; j < dth; ++j) dtheta[j] = host[1 + j];
  return PTTK_OK;
}

}  // namespace
}  // namespace pttk

using namespace pttk;

extern "C" pttk_status pttk_grad(const pttk_tt* tt, const double* theta, const void* X, int64_t N_s, const void* Y,
                                 int64_t N_t, const void* w, const void* z, pttk_prec prec, double* loss,
                                 double* dtheta, void* dX, void* stream) {
  clear_error();
  if (!tt || !theta) return set_error(PTTK_EINVAL, "NULL argument");
  if (N_s < 0 || N_t < 0) return set_error(PTTK_EINVAL, "negative point count");
  if ((N_s > 0 && (!X || !w)) || (N_t > 0 && (!Y || !z))) return set_error(PTTK_EINVAL, "NULL point or weight buffer");
  if (prec < PTTK_FP64 || prec > PTTK_FP16X3) return set_error(PTTK_EINVAL, "unknown precision");
  for (int j = 0; j < tt->dtheta; ++j) {
    const double lo = tt->box[tt->d + j][0], hi = tt->box[tt->d + j][1];
    if (!(theta[j] >= lo - 1e-12 * (hi - lo) && theta[j] <= hi + 1e-12 * (hi - lo)))
      return set_error(PTTK_EDOMAIN, "theta outside its box");
  }
  for (int k = 0; k < tt->d; ++k)
    if (tt->ranks[k] > 4096) return set_error(PTTK_ENOTSUP, "adjoint: rank above 4096");
  cudaStream_t s = as_stream(stream);
  if (prec == PTTK_FP64)
    return grad_typed<double>(tt, theta, static_cast<const double*>(X), N_s, static_cast<const double*>(Y), N_t,
                              static_cast<const double*>(w), static_cast<const double*>(z), prec, loss, dtheta,
                              static_cast<double*>(dX), s);
  return grad_typed<float>(tt, theta, static_cast<const float*>(X), N_s, static_cast<const float*>(Y), N_t,
                           static_cast<const float*>(w), static_cast<const float*>(z), prec, loss, dtheta,
                           static_cast<float*>(dX), s);
}

// Online stage: H(theta) (Eq. hmat, Algorithm 3), the factor chains of Algorithm 2,
// Phase 3 (SIMT FP64 / FP32 form), and the low-rank product U (M (V^T w)).
//
// Factor chain. Per point p the source chain is
//   S_1 = B_1 G_1^{2},   S_i = (B_i face-split S_{i-1}) G_i^{2},   U[p, :] = S_d,
// with B_i[p, k] = T_k(xhat_{p,i}) and the Kronecker column index a + r_{i-1} j matching
// the row index of G_i^{2}. The target chain T <- G_D^{1} V_d^T,
// T <- G_{D-i}^{1} (T Khatri-Rao V_{d-i}^T) has the same per-point form once each core is
// read as (input rank, j, output rank) = (right rank, j, left rank); the handle keeps those
// transposed copies of the target-side cores ("oriented" cores). Each chain step is then a
// GEMM  S_out (P x R_out) = A (P x n R_in) * Gs^{2} (n R_in x R_out)  whose A operand
// A[p, a + R_in j] = B[p, j] S_in[p, a] is generated in shared memory, never stored.
#include <math.h>

#include <stdio.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <mutex>
#include <type_traits>

#include "pttk_internal.cuh"

namespace pttk {

int oriented_core_dims(const pttk_tt* tt, bool source, int step, int* R_in, int* R_out,
                       int* coord);

namespace {

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_sum(T v);
template <>
__device__ __forceinline__ double warp_sum<double>(double v) { return warp_sum_d(v); }
template <>
__device__ __forceinline__ float warp_sum<float>(float v) { return warp_sum_f(v); }

// ---------------- H(theta) -------------------------------------------------------------
// out[a + ra b] = sum_k G[a + ra (k + n b)] T_k(th)   (G: ra x n x rb, column-major)
__global__ void contract_theta_kernel(const double* __restrict__ G, int ra, int n, int rb,
                                      double th, double* __restrict__ out) {
  double T[PTTK_MAX_N];
  T[0] = 1.0;
  if (n > 1) T[1] = th;
  for (int k = 2; k < n; ++k) T[k] = 2.0 * th * T[k - 1] - T[k - 2];
  const int64_t total = (int64_t)ra * rb;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = e % ra, b = e / ra;
    const double* g = G + a + (int64_t)ra * n * b;
    double acc = 0.0;
    for (int k = 0; k < n; ++k) acc = fma(g[(int64_t)ra * k], T[k], acc);
    out[e] = acc;
  }
}

// M row-major (rs x rt) from H column-major (rs x rt)
template <typename T>
__global__ void store_rowmajor_kernel(const double* __restrict__ H, int rs, int rt,
                                      T* __restrict__ M) {
  const int64_t total = (int64_t)rs * rt;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = e / rt, b = e % rt;
    M[e] = (T)H[a + (int64_t)rs * b];
  }
}

// H = H1 H2 for two theta cores, split over the inner dimension so that the product spreads
// over the whole GPU (FP64 issue is ~2 DFMA per clock per SM here, so a few output tiles on a
// few SMs would take ~0.5 ms): block (tile, slice) writes
//   part[slice][a + rs b] = sum_{c in slice} H1[a + rs c] H2[c + rm b]
// and hprod_reduce_kernel sums the slices in a fixed order.
constexpr int HP_T = 32;  // output tile edge and inner slice length
__global__ void __launch_bounds__(256) hprod_splitk_kernel(const double* __restrict__ H1,
                                                           const double* __restrict__ H2, int rs,
                                                           int rm, int rt,
                                                           double* __restrict__ part) {
  __shared__ double a_s[HP_T][HP_T + 1], b_s[HP_T][HP_T + 1];
  const int a0 = blockIdx.x * HP_T, b0 = blockIdx.y * HP_T, c0 = blockIdx.z * HP_T;
  for (int e = threadIdx.x; e < HP_T * HP_T; e += blockDim.x) {
    const int i = e % HP_T, j = e / HP_T;  // a_s[i][j] = H1[a0 + i, c0 + j]; b_s[i][j] = H2[c0 + i, b0 + j]
    a_s[i][j] = (a0 + i < rs && c0 + j < rm) ? H1[(a0 + i) + (int64_t)rs * (c0 + j)] : 0.0;
    b_s[i][j] = (c0 + i < rm && b0 + j < rt) ? H2[(c0 + i) + (int64_t)rm * (b0 + j)] : 0.0;
  }
  __syncthreads();
  const int ti = threadIdx.x % HP_T, tj = threadIdx.x / HP_T;  // tj in [0, 8)
  double acc[HP_T / 8] = {};
  for (int c = 0; c < HP_T; ++c) {
    const double av = a_s[ti][c];
#pragma unroll
    for (int q = 0; q < HP_T / 8; ++q) acc[q] = fma(av, b_s[c][tj + 8 * q], acc[q]);
  }
  double* out = part + (int64_t)blockIdx.z * rs * rt;
#pragma unroll
  for (int q = 0; q < HP_T / 8; ++q) {
    const int a = a0 + ti, b = b0 + tj + 8 * q;
    if (a < rs && b < rt) out[a + (int64_t)rs * b] = acc[q];
  }
}

// M row-major (rs x rt) = sum over the slices of part, in slice order
template <typename T>
__global__ void hprod_reduce_kernel(const double* __restrict__ part, int nslices, int rs, int rt,
                                    T* __restrict__ M) {
  const int64_t total = (int64_t)rs * rt;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = e / rt, b = e % rt;
    double acc = 0.0;
    for (int sl = 0; sl < nslices; ++sl) acc += part[(int64_t)sl * total + a + (int64_t)rs * b];
    M[e] = (T)acc;
  }
}

__global__ void identity_rowmajor_kernel(void* M, int r, bool fp64) {
  const int64_t total = (int64_t)r * r;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double v = (e / r == e % r) ? 1.0 : 0.0;
    if (fp64) static_cast<double*>(M)[e] = v;
    else static_cast<float*>(M)[e] = (float)v;
  }
}

// ---------------- factor chain (SIMT) -----------------------------------------------
struct ChainStep {
  const void* G;  // oriented core, column-major (R_in x n x R_out)
  int R_in, R_out, coord;
  double lo, hi;
};
struct ChainArgs {
  ChainStep st[3];
  int nsteps, n, d, Rmax;  // Rmax: largest R (padded to 64) held in shared memory
  int64_t N;
};

constexpr int CT = 64;  // output columns per tile
constexpr int BK = 16;  // K chunk

// One CTA builds the factor rows of P points. Threads: (P/4) x 16, each owning a 4 x 4
// register tile of (points, output columns).
template <typename T, int P>
__global__ void __launch_bounds__((P / 4) * 16) chain_kernel(ChainArgs a, const T* __restrict__ pts,
                                                             T* __restrict__ out) {
  constexpr int NT = (P / 4) * 16;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Sa = reinterpret_cast<T*>(smem_raw);  // P x Rmax (point-major: Sa[p * Rmax + r])
  T* Sb = Sa + (size_t)P * a.Rmax;
  T* Bv = Sb + (size_t)P * a.Rmax;         // P x n basis values
  T* As = Bv + (size_t)P * PTTK_MAX_N;     // BK x P
  T* Gs = As + BK * P;                     // BK x CT

  const int64_t p0 = (int64_t)blockIdx.x * P;
  const int tp = threadIdx.x / 16, to = threadIdx.x % 16;
  const int n = a.n;
  T* Sin = Sa;
  T* Sout = Sb;
  // S_0 = 1 (r_0 = 1)
  for (int p = threadIdx.x; p < P; p += NT) Sin[p * a.Rmax] = T(1);

  for (int si = 0; si < a.nsteps; ++si) {
    const ChainStep st = a.st[si];
    const T* G = static_cast<const T*>(st.G);
    // Chebyshev basis of this coordinate by the three-term recurrence
    for (int p = threadIdx.x; p < P; p += NT) {
      const int64_t gp = p0 + p;
      const T x = gp < a.N ? pts[gp * a.d + st.coord] : T(st.lo);
      const T xh = (T(2) * x - T(st.lo) - T(st.hi)) / (T(st.lo) - T(st.hi));
      T t0 = T(1), t1 = xh;
      Bv[p * PTTK_MAX_N + 0] = t0;
      if (n > 1) Bv[p * PTTK_MAX_N + 1] = t1;
      for (int k = 2; k < n; ++k) {
        const T t2 = T(2) * xh * t1 - t0;
        Bv[p * PTTK_MAX_N + k] = t2;
        t0 = t1;
        t1 = t2;
      }
    }
    __syncthreads();
    const int K = n * st.R_in;
    for (int o0 = 0; o0 < st.R_out; o0 += CT) {
      T acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
      for (int k0 = 0; k0 < K; k0 += BK) {
        // A chunk: As[kk][p] = B[p, j] * S_in[p, a], k = a + R_in j
        for (int e = threadIdx.x; e < BK * P; e += NT) {
          const int kk = e / P, p = e % P;
          const int k = k0 + kk;
          T v = T(0);
          if (k < K) {
            const int j = k / st.R_in, ar = k % st.R_in;
            v = Bv[p * PTTK_MAX_N + j] * Sin[p * a.Rmax + ar];
          }
          As[kk * P + p] = v;
        }
        // core chunk: Gs[kk][o] = Gs2[k, o0 + o]
        for (int e = threadIdx.x; e < BK * CT; e += NT) {
          const int kk = e / CT, o = e % CT;
          const int k = k0 + kk, oc = o0 + o;
          Gs[kk * CT + o] = (k < K && oc < st.R_out) ? G[k + (int64_t)K * oc] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
          T av[4], bv[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) av[i] = As[kk * P + tp * 4 + i];
#pragma unroll
          for (int j = 0; j < 4; ++j) bv[j] = Gs[kk * CT + to * 4 + j];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
      }
      const bool last = si == a.nsteps - 1;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int p = tp * 4 + i;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int oc = o0 + to * 4 + j;
          if (oc >= st.R_out) continue;
          if (last) {
            const int64_t gp = p0 + p;
            if (gp < a.N) out[gp * st.R_out + oc] = acc[i][j];
          } else {
            Sout[p * a.Rmax + oc] = acc[i][j];
          }
        }
      }
    }
    __syncthreads();
    T* tmp = Sin;
    Sin = Sout;
    Sout = tmp;
  }
}

// ---------------- apply: out = U (M (V^T w)) ----------------------------------------
// partial[b, c] = sum over block b's rows r of V[r, c] w[r]. Threads are 4 row lanes x 64
// column groups, each of VW consecutive columns (VW = 4 when rows are 16-byte aligned: a row
// of up to 256 columns is then read once, contiguously, by 16-byte loads; else VW = 1 and 64
// columns a pass). Each thread keeps 4 rows of loads in flight; the row lanes meet in shared
// memory in a fixed order.
template <typename T, int VW>
__global__ void __launch_bounds__(256) vtw_partial_kernel(const T* __restrict__ V, int64_t N,
                                                          int rt, const T* __restrict__ w,
                                                          T* __restrict__ partial) {
  __shared__ T red[4][64 * VW];
  const int64_t rows_per = (N + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per, r1 = std::min<int64_t>(N, r0 + rows_per);
  const int cl = threadIdx.x & 63, rl = threadIdx.x >> 6;
  for (int cb = 0; cb < rt; cb += 64 * VW) {
    const int c = cb + cl * VW;
    const bool on = c < rt;  // with VW = 4, rt is a multiple of 4: the whole group is in range
    T acc[VW];
#pragma unroll
    for (int q = 0; q < VW; ++q) acc[q] = T(0);
    int64_t r = r0 + rl;
    for (; r + 12 < r1; r += 16) {
      T v[4][VW];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const T* src = V + (r + 4 * u) * rt + c;
        if constexpr (VW == 4) {
          if (on) {
            if constexpr (sizeof(T) == 4) {
              const float4 x = *reinterpret_cast<const float4*>(src);
              v[u][0] = x.x; v[u][1] = x.y; v[u][2] = x.z; v[u][3] = x.w;
            } else {
              const double2 x0 = *reinterpret_cast<const double2*>(src);
              const double2 x1 = *reinterpret_cast<const double2*>(src + 2);
              v[u][0] = x0.x; v[u][1] = x0.y; v[u][2] = x1.x; v[u][3] = x1.y;
            }
          } else {
#pragma unroll
            for (int q = 0; q < VW; ++q) v[u][q] = T(0);
          }
        } else {
          v[u][0] = on ? *src : T(0);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const T wr = w[r + 4 * u];
#pragma unroll
        for (int q = 0; q < VW; ++q) acc[q] = fma(v[u][q], wr, acc[q]);
      }
    }
    for (; r < r1; r += 4) {
      const T wr = w[r];
#pragma unroll
      for (int q = 0; q < VW; ++q) acc[q] = fma(on ? V[r * rt + c + q] : T(0), wr, acc[q]);
    }
#pragma unroll
    for (int q = 0; q < VW; ++q) red[rl][cl * VW + q] = acc[q];
    __syncthreads();
    for (int q = threadIdx.x; q < 64 * VW; q += blockDim.x)
      if (cb + q < rt) partial[(int64_t)blockIdx.x * rt + cb + q] = (red[0][q] + red[1][q]) + (red[2][q] + red[3][q]);
    __syncthreads();
  }
}

// t = sum over the partial rows, written into row 0 of `partial`: 32 columns x 8 part lanes
// per block, each lane summing every eighth part, the lanes then added in a fixed order (the
// rows a block reads belong to its own columns only).
template <typename T>
__global__ void __launch_bounds__(256) reduce_parts_kernel(T* __restrict__ partial, int nparts, int rt) {
  __shared__ T red[8][32];
  const int cl = threadIdx.x & 31, pl = threadIdx.x >> 5;
  const int64_t c = (int64_t)blockIdx.x * 32 + cl;
  T acc = T(0);
  if (c < rt)
    for (int b = pl; b < nparts; b += 8) acc += partial[(int64_t)b * rt + c];
  red[pl][cl] = acc;
  __syncthreads();
  if (pl == 0 && c < rt)
    partial[c] = ((red[0][cl] + red[1][cl]) + (red[2][cl] + red[3][cl])) +
                 ((red[4][cl] + red[5][cl]) + (red[6][cl] + red[7][cl]));
}

// s = M t, one warp per row of M (rs x rt, row-major); t is read through the L1 cache, so
// no shared memory is sized by a rank.
template <typename T>
__global__ void __launch_bounds__(256) mt_kernel(const T* __restrict__ M, int rs, int rt,
                                                 const T* __restrict__ t, T* __restrict__ s_out) {
  const int lane = threadIdx.x & 31;
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < rs;
       r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const T* m = M + r * rt;
    T acc = T(0);
    for (int c = lane; c < rt; c += 32) acc = fma(m[c], __ldg(t + c), acc);
    acc = warp_sum<T>(acc);
    if (lane == 0) s_out[r] = acc;
  }
}

// out[p] = U[p, :] . s, one warp per row, two rows at a time (the loads of both are in
// flight before either is reduced); s is read through the L1 cache
template <typename T>
__global__ void __launch_bounds__(256) us_kernel(const T* __restrict__ U, int64_t N, int rs,
                                                 const T* __restrict__ s, T* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < N; row += 2 * nw) {
    const int64_t row2 = row + nw;
    const bool two = row2 < N;
    const T* u = U + row * rs;
    const T* u2 = U + (two ? row2 : row) * rs;
    T acc = T(0), acc2 = T(0);
    for (int c = lane; c < rs; c += 32) {
      const T sc = __ldg(s + c);
      acc = fma(u[c], sc, acc);
      acc2 = fma(u2[c], sc, acc2);
    }
    acc = warp_sum<T>(acc);
    acc2 = warp_sum<T>(acc2);
    if (lane == 0) {
      out[row] = acc;
      if (two) out[row2] = acc2;
    }
  }
}

template <typename T>
pttk_status apply_typed(const T* U, const T* M, const T* V, int64_t N_s, int64_t N_t, int rs,
                        int rt, const T* w, T* out, T* scratch, int nparts, cudaStream_t s) {
  T* partial = scratch;
  T* sv = scratch + (size_t)nparts * rt;
  PTTK_PROF("apply", s);
  if (N_t > 0) {
    // 16-byte column groups when every row starts on a 16-byte boundary
    const bool vec = rt % 4 == 0 && (reinterpret_cast<uintptr_t>(V) & 15) == 0 && (sizeof(T) * rt) % 16 == 0;
    if (vec) vtw_partial_kernel<T, 4><<<nparts, 256, 0, s>>>(V, N_t, rt, w, partial);
    else vtw_partial_kernel<T, 1><<<nparts, 256, 0, s>>>(V, N_t, rt, w, partial);
    pttk::count_launch();
  } else {
    PTTK_CUDA(cudaMemsetAsync(partial, 0, sizeof(T) * (size_t)nparts * rt, s));
  }
  if (nparts > 1) {
    reduce_parts_kernel<T><<<(unsigned)((rt + 31) / 32), 256, 0, s>>>(partial, nparts, rt); pttk::count_launch();
  }
  const int64_t mblocks = std::min<int64_t>(((int64_t)rs * 32 + 255) / 256, (int64_t)sm_count() * 16);
  mt_kernel<T><<<(unsigned)mblocks, 256, 0, s>>>(M, rs, rt, partial, sv); pttk::count_launch();
  if (N_s > 0) {
    const int64_t blocks = std::min<int64_t>((N_s * 32 + 255) / 256, (int64_t)sm_count() * 16);
    us_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(U, N_s, rs, sv, out); pttk::count_launch();
  }
  PTTK_CUDA(cudaGetLastError());
  return PTTK_OK;
}

int apply_parts(int64_t N_t) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((N_t + 255) / 256, (int64_t)sm_count() * 4));
}

}  // namespace

// ---------------- point domain ---------------------------------------------------------
// The problem is stated for X in B_s and Y in B_t (Section 1). One pass over a point set
// records PTTK_EDOMAIN in the handle's status word if any coordinate lies outside its
// interval by more than a relative slack of 1e-12. FP32 points are compared with the
// FP32-rounded interval ends: rounding is monotone, so a point inside the box stays inside
// the rounded box when it is cast. Both sides are checked in one launch (blockIdx.y picks
// the side). The pass is a plain read of the point sets (12 B per point for d = 3 in FP32),
// so nothing in it may use the FP64 pipe, which runs at about 2 operations per clock per SM:
//  - FP32 points are compared in FP32 with bounds rounded inwards on the host (the smallest
//    float >= lo - slack, the largest float <= hi + slack), which accepts exactly the floats
//    the FP64 comparison accepts;
//  - FP64 points are compared as order-preserving 64-bit integer keys of their bit patterns.
// A NaN coordinate fails both forms of the comparison. A side whose base is 16-byte aligned
// and whose N d elements fill whole 16-byte units is read with 16-byte loads, else element by
// element. The coordinate index is carried from step to step instead of taken modulo d, and
// the bounds sit in shared memory.
struct PointCheck {
  const void* P[2];
  int64_t total[2];                        // N * d elements per side
  int vec[2];                              // 16-byte loads: base 16-byte aligned, total a multiple of 16 B
  long long klo[2][PTTK_MAX_D], khi[2][PTTK_MAX_D];  // FP64 points: integer keys of the bounds
  float flo[2][PTTK_MAX_D], fhi[2][PTTK_MAX_D];      // FP32 points: the bounds as floats
};

// Key of a double: a signed 64-bit integer ordered as the doubles are, with -0 and +0 equal
// (the magnitude bits, negated for a set sign bit). A NaN's key lies beyond the keys of the
// infinities on its sign's side, so it fails any comparison with finite bounds.
__host__ __device__ __forceinline__ long long order_key(long long bits) {
  return bits < 0 ? -(bits & 0x7FFFFFFFFFFFFFFFLL) : bits;
}

template <typename T>
__global__ void __launch_bounds__(256) point_domain_kernel(PointCheck a, int d, int* __restrict__ status) {
  constexpr bool F64 = std::is_same_v<T, double>;
  using B = std::conditional_t<F64, long long, float>;
  constexpr int W = 16 / (int)sizeof(T);  // elements per 16-byte load
  __shared__ B lo[PTTK_MAX_D], hi[PTTK_MAX_D];
  const int side = blockIdx.y;
  if (threadIdx.x < d) {
    if constexpr (F64) {
      lo[threadIdx.x] = a.klo[side][threadIdx.x];
      hi[threadIdx.x] = a.khi[side][threadIdx.x];
    } else {
      lo[threadIdx.x] = a.flo[side][threadIdx.x];
      hi[threadIdx.x] = a.fhi[side][threadIdx.x];
    }
  }
  __syncthreads();
  bool bad = false;
  auto check = [&](B x, int c) {
    if constexpr (F64) bad |= order_key(x) < lo[c] || order_key(x) > hi[c];
    else bad |= !(x >= lo[c] && x <= hi[c]);  // also catches NaN
  };
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a.vec[side]) {
    // e counts 16-byte units; the coordinate of the unit's first element is carried
    const int64_t units = a.total[side] / W;
    int c = (int)((e * W) % d);
    const int cstep = (int)((stride * W) % d);
    using V = std::conditional_t<F64, longlong2, float4>;
    const V* __restrict__ P = static_cast<const V*>(a.P[side]);
#pragma unroll 2
    for (; e < units; e += stride) {
      const V v = __ldg(P + e);
      int cc = c;
      if constexpr (F64) {
        check(v.x, cc);
        cc = cc + 1 == d ? 0 : cc + 1;
        check(v.y, cc);
      } else {
        check(v.x, cc);
        cc = cc + 1 == d ? 0 : cc + 1;
        check(v.y, cc);
        cc = cc + 1 == d ? 0 : cc + 1;
        check(v.z, cc);
        cc = cc + 1 == d ? 0 : cc + 1;
        check(v.w, cc);
      }
      c += cstep;
      if (c >= d) c -= d;
    }
  } else {
    const int64_t total = a.total[side];
    int c = (int)(e % d);
    const int cstep = (int)(stride % d);
    const B* __restrict__ P = static_cast<const B*>(a.P[side]);
#pragma unroll 4
    for (; e < total; e += stride) {
      check(__ldg(P + e), c);
      c += cstep;
      if (c >= d) c -= d;
    }
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicCAS(status, 0, (int)PTTK_EDOMAIN);
}

// The smallest float >= v and the largest float <= v.
static float float_at_or_above(double v) {
  float f = (float)v;
  if ((double)f < v) f = std::nextafter(f, std::numeric_limits<float>::infinity());
  return f;
}
static float float_at_or_below(double v) {
  float f = (float)v;
  if ((double)f > v) f = std::nextafter(f, -std::numeric_limits<float>::infinity());
  return f;
}
static long long key_of(double v) {
  long long bits;
  std::memcpy(&bits, &v, sizeof bits);
  return order_key(bits);
}

pttk_status point_domain_check(const pttk_tt* tt, const void* X, int64_t N_s, const void* Y, int64_t N_t, bool fp64,
                               int* status, cudaStream_t s) {
  N_s = X ? std::max<int64_t>(N_s, 0) : 0;
  N_t = Y ? std::max<int64_t>(N_t, 0) : 0;
  if (N_s == 0 && N_t == 0) return PTTK_OK;
  PTTK_PROF("domain", s);
  PointCheck a{};
  a.P[0] = X;
  a.P[1] = Y;
  a.total[0] = N_s * tt->d;
  a.total[1] = N_t * tt->d;
  for (int side = 0; side < 2; ++side)
    for (int c = 0; c < tt->d; ++c) {
      const int bj = side == 0 ? c : tt->d + tt->dtheta + c;
      const double lo = tt->box[bj][0], hi = tt->box[bj][1], slack = 1e-12 * (hi - lo);
      a.klo[side][c] = key_of(lo - slack);
      a.khi[side][c] = key_of(hi + slack);
      a.flo[side][c] = float_at_or_above((double)(float)lo - slack);
      a.fhi[side][c] = float_at_or_below((double)(float)hi + slack);
    }
  const int W = fp64 ? 2 : 4;
  int64_t work = 0;
  for (int side = 0; side < 2; ++side) {
    a.vec[side] = (reinterpret_cast<uintptr_t>(a.P[side]) & 15) == 0 && a.total[side] % W == 0;
    work = std::max(work, a.vec[side] ? a.total[side] / W : a.total[side]);
  }
  const dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, (int64_t)sm_count() * 4)), 2);
  if (fp64) point_domain_kernel<double><<<grid, 256, 0, s>>>(a, tt->d, status);
  else point_domain_kernel<float><<<grid, 256, 0, s>>>(a, tt->d, status);
  pttk::count_launch();
  PTTK_CUDA(cudaGetLastError());
  return PTTK_OK;
}

// Step `step` of a side's chain: dimensions of its oriented core and the point coordinate.
int oriented_core_dims(const pttk_tt* tt, bool source, int step, int* R_in, int* R_out,
                       int* coord) {
  if (source) {
    const int k = step;  // core G_{k+1}
    *R_in = tt->ranks[k];
    *R_out = tt->ranks[k + 1];
    *coord = step;
    return k;
  }
  const int k = tt->D - 1 - step;  // core G_{D-step}, read transposed
  *R_in = tt->ranks[k + 1];
  *R_out = tt->ranks[k];
  *coord = tt->d - 1 - step;
  return k;
}

pttk_status theta_core_run(const pttk_tt* tt, const double* theta_hat, bool fp64, void* M,
                           cudaStream_t s) {
  const int d = tt->d, dth = tt->dtheta, n = tt->n;
  const int rs = tt->ranks[d], rt = tt->ranks[d + dth];
  if (dth == 0) {
    identity_rowmajor_kernel<<<64, 256, 0, s>>>(M, rs, fp64); pttk::count_launch();
    PTTK_CUDA(cudaGetLastError());
    return PTTK_OK;
  }
  PTTK_PROF("theta_core", s);
  const int rm = tt->ranks[d + 1];
  const int nslices = (rm + HP_T - 1) / HP_T;
  size_t need = 0;
  for (int j = 0; j < dth; ++j) need += (size_t)tt->ranks[d + j] * tt->ranks[d + j + 1];
  need += (size_t)rs * rt * (dth > 1 ? nslices : 0);
  double* work = nullptr;
  PTTK_CUDA(cudaMallocAsync(&work, sizeof(double) * std::max<size_t>(need, 1), s));
  double* Hj[2] = {work, work + (size_t)tt->ranks[d] * tt->ranks[d + 1]};
  for (int j = 0; j < dth; ++j) {
    const int ra = tt->ranks[d + j], rb = tt->ranks[d + j + 1];
    const int64_t total = (int64_t)ra * rb;
    const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, sm_count() * 8);
    contract_theta_kernel<<<blocks, 256, 0, s>>>(tt->cores64 + tt->core_off[d + j], ra, n, rb,
                                                 theta_hat[j], Hj[j]); pttk::count_launch();
  }
  const unsigned blocks = (unsigned)std::min<int64_t>(((int64_t)rs * rt + 255) / 256, sm_count() * 8);
  if (dth == 2) {
    double* part = Hj[1] + (size_t)rm * rt;
    const dim3 grid((unsigned)((rs + HP_T - 1) / HP_T), (unsigned)((rt + HP_T - 1) / HP_T), (unsigned)nslices);
    hprod_splitk_kernel<<<grid, 256, 0, s>>>(Hj[0], Hj[1], rs, rm, rt, part); pttk::count_launch();
    if (fp64) { hprod_reduce_kernel<double><<<blocks, 256, 0, s>>>(part, nslices, rs, rt, static_cast<double*>(M)); pttk::count_launch(); }
    else { hprod_reduce_kernel<float><<<blocks, 256, 0, s>>>(part, nslices, rs, rt, static_cast<float*>(M)); pttk::count_launch(); }
  } else if (fp64) {
    store_rowmajor_kernel<double><<<blocks, 256, 0, s>>>(Hj[0], rs, rt, static_cast<double*>(M)); pttk::count_launch();
  } else {
    store_rowmajor_kernel<float><<<blocks, 256, 0, s>>>(Hj[0], rs, rt, static_cast<float*>(M)); pttk::count_launch();
  }
  PTTK_CUDA(cudaGetLastError());
  PTTK_CUDA(cudaFreeAsync(work, s));
  return PTTK_OK;
}

template <typename T, int P>
static pttk_status launch_chain(const ChainArgs& a, const T* pts, T* out, cudaStream_t s) {
  const size_t smem = sizeof(T) * ((size_t)2 * P * a.Rmax + (size_t)P * PTTK_MAX_N + BK * P + BK * CT);
  auto kfn = chain_kernel<T, P>;
  PTTK_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t blocks = (a.N + P - 1) / P;
  PTTK_PROF("chain", s);
  kfn<<<(unsigned)blocks, (P / 4) * 16, smem, s>>>(a, pts, out); pttk::count_launch();
  PTTK_CUDA(cudaGetLastError());
  return PTTK_OK;
}

// Oriented core pointer for a chain step (see pttk_tt::oriented).
const void* oriented_core_ptr(const pttk_tt* tt, bool source, int k, bool fp64);

pttk_status factor_build_run(const pttk_tt* tt, bool source, const void* P, int64_t N,
                             pttk_prec prec, void* out, cudaStream_t s, int nsteps) {
  if (N == 0) return PTTK_OK;
  const bool fp64 = prec == PTTK_FP64;
  ChainArgs a{};
  a.nsteps = (nsteps > 0 && nsteps < tt->d) ? nsteps : tt->d;
  a.n = tt->n;
  a.d = tt->d;
  a.N = N;
  int rmax = 1;
  for (int i = 0; i < a.nsteps; ++i) {
    int rin, rout, coord;
    const int k = oriented_core_dims(tt, source, i, &rin, &rout, &coord);
    a.st[i].G = oriented_core_ptr(tt, source, k, fp64);
    a.st[i].R_in = rin;
    a.st[i].R_out = rout;
    a.st[i].coord = coord;
    const int bj = source ? coord : tt->d + tt->dtheta + coord;
    a.st[i].lo = tt->box[bj][0];
    a.st[i].hi = tt->box[bj][1];
    rmax = std::max(rmax, std::max(rin, rout));
  }
  a.Rmax = ((rmax + CT - 1) / CT) * CT;
  const size_t elem = fp64 ? 8 : 4;
  const size_t budget = 200000;
  auto fits = [&](int P) {
    return elem * ((size_t)2 * P * a.Rmax + (size_t)P * PTTK_MAX_N + BK * P + BK * CT) <= budget;
  };
  if (fp64) {
    if (fits(64)) return launch_chain<double, 64>(a, static_cast<const double*>(P), static_cast<double*>(out), s);
    if (fits(32)) return launch_chain<double, 32>(a, static_cast<const double*>(P), static_cast<double*>(out), s);
    if (fits(16)) return launch_chain<double, 16>(a, static_cast<const double*>(P), static_cast<double*>(out), s);
  } else {
    if (fits(64)) return launch_chain<float, 64>(a, static_cast<const float*>(P), static_cast<float*>(out), s);
    if (fits(32)) return launch_chain<float, 32>(a, static_cast<const float*>(P), static_cast<float*>(out), s);
    if (fits(16)) return launch_chain<float, 16>(a, static_cast<const float*>(P), static_cast<float*>(out), s);
  }
  return set_error(PTTK_ENOTSUP, "TT ranks too large for the SIMT factor chain");
}

size_t apply_scratch_bytes(int64_t N_t, int rs, int rt, bool fp64) {
  const int nparts = apply_parts(N_t);
  return (fp64 ? 8 : 4) * ((size_t)nparts * rt + (size_t)rs);
}

pttk_status apply_run(const void* U, const void* M, const void* V, int64_t N_s, int64_t N_t,
                      int rs, int rt, bool fp64, const void* w, void* out, void* scratch,
                      cudaStream_t s) {
  const int nparts = apply_parts(N_t);
  if (fp64)
    return apply_typed<double>(static_cast<const double*>(U), static_cast<const double*>(M),
                               static_cast<const double*>(V), N_s, N_t, rs, rt,
                               static_cast<const double*>(w), static_cast<double*>(out),
                               static_cast<double*>(scratch), nparts, s);
  return apply_typed<float>(static_cast<const float*>(U), static_cast<const float*>(M),
                            static_cast<const float*>(V), N_s, N_t, rs, rt,
                            static_cast<const float*>(w), static_cast<float*>(out),
                            static_cast<float*>(scratch), nparts, s);
}

}  // namespace pttk

// ---------------- apply without device allocation ---------------------------------------
// pttk_apply_noalloc runs the same kernels as pttk_apply, with its scratch (the per-block
// partial sums of V^T w and the vector M (V^T w)) in this file-scope device array instead of
// a stream-ordered allocation. Every device that loads the library holds the array until the
// process exits. All calls share it, so calls whose work overlaps on the GPU race.
namespace pttk {
namespace {

constexpr size_t kNoAllocScratchBytes = 1u << 20;  // 1 MiB
static __device__ __align__(256) unsigned char g_apply_scratch[kNoAllocScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_dev[64] = {nullptr};

// Device address of g_apply_scratch on the current device, looked up once per device.
// In host code the symbol name is only a host-side stand-in, never a device address.
pttk_status scratch_address(void** out) {
  int dev = 0;
  PTTK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return set_error(PTTK_EINVAL, "device ordinal above 63");
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    PTTK_CUDA(cudaGetSymbolAddress(&p, g_apply_scratch));
    g_scratch_dev[dev] = p;
  }
  *out = g_scratch_dev[dev];
  return PTTK_OK;
}

}  // namespace
}  // namespace pttk

extern "C" pttk_status pttk_apply_noalloc(const void* U, const void* M, const void* V, int64_t N_s,
                                          int64_t N_t, int rs, int rt, pttk_prec prec, const void* w,
                                          void* out, void* stream) {
  using namespace pttk;
  clear_error();
  if (!M || (N_s > 0 && (!U || !out)) || (N_t > 0 && (!V || !w))) return set_error(PTTK_EINVAL, "NULL argument");
  if (N_s < 0 || N_t < 0 || rs < 1 || rt < 1) return set_error(PTTK_EINVAL, "bad size");
  if (prec != PTTK_FP64 && prec != PTTK_FP32) return set_error(PTTK_EINVAL, "apply precision must be FP64 or FP32");
  const bool fp64 = prec == PTTK_FP64;
  const size_t elem = fp64 ? 8 : 4;
  const size_t cap = kNoAllocScratchBytes / elem;
  if ((size_t)rs + (size_t)rt > cap) {
    char buf[200];
    snprintf(buf, sizeof buf,
             "pttk_apply_noalloc: rs + rt = %lld exceeds its fixed scratch of %zu %s elements",
             (long long)rs + rt, cap, fp64 ? "FP64" : "FP32");
    return set_error(PTTK_EINVAL, buf);
  }
  void* scratch = nullptr;
  PTTK_TRY(scratch_address(&scratch));
  // as many partial-sum blocks as pttk_apply uses, fewer if they would not fit
  const int nparts = (int)std::max<int64_t>(
      1, std::min<int64_t>(apply_parts(N_t), (int64_t)((cap - (size_t)rs) / (size_t)rt)));
  cudaStream_t s = as_stream(stream);
  if (fp64)
    return apply_typed<double>(static_cast<const double*>(U), static_cast<const double*>(M),
                               static_cast<const double*>(V), N_s, N_t, rs, rt,
                               static_cast<const double*>(w), static_cast<double*>(out),
                               static_cast<double*>(scratch), nparts, s);
  return apply_typed<float>(static_cast<const float*>(U), static_cast<const float*>(M),
                            static_cast<const float*>(V), N_s, N_t, rs, rt,
                            static_cast<const float*>(w), static_cast<float*>(out),
                            static_cast<float*>(scratch), nparts, s);
}

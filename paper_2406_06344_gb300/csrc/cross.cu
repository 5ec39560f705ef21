// TT greedy-cross (Appendix "TT-cross approximation": Algorithms 5, 6 and 7) on the GPU: a TT
// of the grid tensor M (Eq. mdc) from sampled entries, without forming the n^D grid, then the
// Chebyshev transform of every core (G_k <- G_k x_2 A) so that the result is the coefficient-form
// TT the rest of the library uses.
//
// Division of work. The index sets (I<=k, I>k), the sample positions and every random draw stay
// on the host, drawn from SplitMix64 in the order the method consumes them, so that another
// implementation with the same key draws the same numbers. The device evaluates the kernel
// entries (every fibre, cross matrix and sample set a step needs, in one launch per step),
// solves the r x r cross-matrix systems (Gaussian elimination with partial pivoting), forms the
// skeleton residuals A(:, J) A(I, J)^{-1} A(I, :) - A at the sampled positions, the condition
// numbers of the 2 x 2 candidates of Algorithm 7, the TT at the check points of the stopping
// test, and the Chebyshev transform of the cores. The host picks the extremum of each returned
// vector (the first index within a relative 1e-12 of it) and updates the index sets.
//
// Readings of the paper (the same as the oracle's): the residual is read as
// A(:, J) A(I, J)^{-1} A(I, :) - A; a pivot is added only when its residual exceeds 1e-14 of
// the largest entry the update evaluated; the interpolation cores are C_k^{2} = T_k^{2} P_k^{-1}
// (T_k = X(I<=k-1, :, I>k), P_k = X(I<=k, I>k)), C_N = T_N; the stopping test is the largest
// |x - x^| over n_check random entries, relative to the largest |x| among them; Algorithm 5
// samples max(rows, cols) distinct positions of the unfolded super-core.
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "pttk_internal.cuh"

namespace pttk {
namespace {

using Tup = std::vector<int>;
constexpr double kTieRtol = 1e-12;

struct Rng {
  uint64_t key, counter = 0;
  uint64_t u64() { return splitmix64(key, counter++); }
  int below(int m) { return (int)(u64() % (uint64_t)m); }
  int bit() { return (int)(u64() >> 63); }
};

int first_argmax(const std::vector<double>& v) {
  double mx = -INFINITY;
  for (double x : v) mx = std::max(mx, x);
  for (size_t i = 0; i < v.size(); ++i)
    if (v[i] >= (1.0 - kTieRtol) * mx) return (int)i;
  return 0;
}
int first_argmin(const std::vector<double>& v) {
  double mn = INFINITY;
  for (double x : v) mn = std::min(mn, x);
  for (size_t i = 0; i < v.size(); ++i)
    if (v[i] <= (1.0 + kTieRtol) * mn) return (int)i;
  return 0;
}

// ---- device kernels ----------------------------------------------------------------------

// 2-norm condition number of each 2 x 2 matrix [[e0, e1], [e2, e3]] (entries 4q .. 4q+3):
// sigma_1^2 = (s + sqrt(s^2 - 4 det^2)) / 2 with s the squared Frobenius norm, and
// sigma_1 / sigma_2 = sigma_1^2 / |det| (infinite for a singular matrix)
__global__ void cond2_kernel(const double* __restrict__ e, int m, double* __restrict__ out) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < m; q += gridDim.x * blockDim.x) {
    const double a = e[4 * q], b = e[4 * q + 1], c = e[4 * q + 2], d = e[4 * q + 3];
    const double s = a * a + b * b + c * c + d * d, det = fabs(a * d - b * c);
    const double disc = sqrt(fmax(s * s - 4.0 * det * det, 0.0));
    const double s1 = 0.5 * (s + disc);
    out[q] = det > 0.0 ? s1 / det : INFINITY;
  }
}

// Solves P X = B in place (B <- X) for P r x r and B r x m, both column-major, one block:
// Gaussian elimination with partial pivoting on a copy of P in `work` (r x r), the row
// interchanges applied to B as they happen.
__global__ void __launch_bounds__(256) lu_solve_kernel(const double* __restrict__ P, int r, double* __restrict__ B,
                                                       int m, double* __restrict__ work) {
  __shared__ int piv_row;
  double* A = work;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) A[e] = P[e];
  __syncthreads();
  for (int k = 0; k < r; ++k) {
    if (threadIdx.x == 0) {
      int best = k;
      double bv = fabs(A[k + (size_t)r * k]);
      for (int i = k + 1; i < r; ++i) {
        const double v = fabs(A[i + (size_t)r * k]);
        if (v > bv) {
          bv = v;
          best = i;
        }
      }
      piv_row = best;
    }
    __syncthreads();
    const int p = piv_row;
    if (p != k) {
      for (int j = threadIdx.x; j < r; j += blockDim.x) {
        const double t = A[k + (size_t)r * j];
        A[k + (size_t)r * j] = A[p + (size_t)r * j];
        A[p + (size_t)r * j] = t;
      }
      for (int j = threadIdx.x; j < m; j += blockDim.x) {
        const double t = B[k + (size_t)r * j];
        B[k + (size_t)r * j] = B[p + (size_t)r * j];
        B[p + (size_t)r * j] = t;
      }
    }
    __syncthreads();
    const double dkk = A[k + (size_t)r * k];
    if (dkk != 0.0) {
      for (int i = k + 1 + threadIdx.x; i < r; i += blockDim.x) A[i + (size_t)r * k] /= dkk;
    }
    __syncthreads();
    // trailing update of A and the elimination on B
    for (int e = threadIdx.x; e < (r - k - 1) * (r - k - 1); e += blockDim.x) {
      const int i = k + 1 + e % (r - k - 1), j = k + 1 + e / (r - k - 1);
      A[i + (size_t)r * j] -= A[i + (size_t)r * k] * A[k + (size_t)r * j];
    }
    for (int e = threadIdx.x; e < (r - k - 1) * m; e += blockDim.x) {
      const int i = k + 1 + e % (r - k - 1), j = e / (r - k - 1);
      B[i + (size_t)r * j] -= A[i + (size_t)r * k] * B[k + (size_t)r * j];
    }
    __syncthreads();
  }
  // back substitution, one thread per right-hand side
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    double* x = B + (size_t)r * j;
    for (int i = r - 1; i >= 0; --i) {
      double acc = x[i];
      for (int l = i + 1; l < r; ++l) acc -= A[i + (size_t)r * l] * x[l];
      x[i] = acc / A[i + (size_t)r * i];
    }
  }
}

// R[p] = sum_j Lm[p + m j] X[j + r p] - a[p] (the skeleton minus the entry), one warp per p
__global__ void residual_kernel(const double* __restrict__ Lm, const double* __restrict__ X, const double* __restrict__ a,
                                int m, int r, double* __restrict__ R) {
  const int lane = threadIdx.x & 31;
  for (int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < m; p += (gridDim.x * blockDim.x) >> 5) {
    double acc = 0.0;
    for (int j = lane; j < r; j += 32) acc = fma(Lm[p + (size_t)m * j], X[j + (size_t)r * p], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) R[p] = acc - a[p];
  }
}

// x^ at M multi-indices of the TT (cores packed, core k r_k x n x r_{k+1} column-major at
// off[k]); one block per index: the row vector G_1[:, i_1, :] G_2[:, i_2, :] ... in shared memory
__global__ void __launch_bounds__(256) tt_eval_kernel(const double* __restrict__ cores, const int64_t* __restrict__ off,
                                                      const int* __restrict__ ranks, int D, int n,
                                                      const int* __restrict__ idx, int M, double* __restrict__ out) {
  extern __shared__ double vsh[];
  double* v = vsh;                 // current row vector (length <= rmax)
  double* w = vsh + blockDim.x * 4;  // next
  const int rmax = blockDim.x * 4;
  for (int q = blockIdx.x; q < M; q += gridDim.x) {
    if (threadIdx.x == 0) v[0] = 1.0;
    __syncthreads();
    for (int k = 0; k < D; ++k) {
      const int ra = ranks[k], rb = ranks[k + 1], ik = idx[(size_t)q * D + k];
      const double* G = cores + off[k] + (size_t)ra * ik;  // G[a, ik, b] at a + ra (ik + n b)
      for (int b = threadIdx.x; b < rb && b < rmax; b += blockDim.x) {
        double acc = 0.0;
        for (int a2 = 0; a2 < ra; ++a2) acc = fma(v[a2], G[a2 + (size_t)ra * n * b], acc);
        w[b] = acc;
      }
      __syncthreads();
      for (int b = threadIdx.x; b < rb && b < rmax; b += blockDim.x) v[b] = w[b];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = v[0];
    __syncthreads();
  }
}

// out[a + ra (k + n b)] = sum_i A[k, i] G[a + ra (i + n b)], A[k, i] = (c_k / n) T_k(zeta_i),
// zeta_i = cos((2i + 1) pi / (2n)), c_0 = 1, c_k = 2: the mode-2 Chebyshev transform of a core
__global__ void core_transform_kernel(const double* __restrict__ G, int ra, int n, int rb, double* __restrict__ out) {
  const int64_t total = (int64_t)ra * n * rb;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(e % ra), k = (int)((e / ra) % n);
    const int64_t b = e / ((int64_t)ra * n);
    double acc = 0.0;
    for (int i = 0; i < n; ++i) {
      const double zeta = cos((2.0 * i + 1.0) * 3.141592653589793 / (2.0 * n));
      const double Tk = cos(k * acos(zeta));
      acc = fma((k == 0 ? 1.0 : 2.0) / n * Tk, G[a + (int64_t)ra * (i + (int64_t)n * b)], acc);
    }
    out[e] = acc;
  }
}

// ---- host driver -------------------------------------------------------------------------

struct Dev {
  std::vector<void*> bufs;
  ~Dev() {
    for (void* p : bufs)
      if (p) cudaFree(p);
  }
  template <typename T>
  pttk_status get(T** out, size_t n) {
    void* p = nullptr;
    PTTK_CUDA(cudaMalloc(&p, sizeof(T) * std::max<size_t>(n, 1)));
    bufs.push_back(p);
    *out = static_cast<T*>(p);
    return PTTK_OK;
  }
};

struct Cross {
  int kernel, d, dth, D, n;
  double box[PTTK_MAX_D][2];
  cudaStream_t s;
  int* d_status = nullptr;
  int64_t evals = 0;

  // kernel entries at the multi-indices idx (M x D, host) into a device buffer (M doubles)
  pttk_status eval(const std::vector<int>& idx, double* out_dev, Dev& dv) {
    const int64_t M = (int64_t)idx.size() / D;
    if (M == 0) return PTTK_OK;
    int* di = nullptr;
    PTTK_TRY(dv.get(&di, idx.size()));
    PTTK_CUDA(cudaMemcpyAsync(di, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice, s));
    PTTK_TRY(grid_entries_launch(kernel, d, dth, n, box, di, M, true, out_dev, d_status, s));
    evals += M;
    return PTTK_OK;
  }
  static void push(std::vector<int>& idx, const Tup& a, const Tup& b, const Tup& c) {
    idx.insert(idx.end(), a.begin(), a.end());
    idx.insert(idx.end(), b.begin(), b.end());
    idx.insert(idx.end(), c.begin(), c.end());
  }

  // Algorithm 7: index sets of cardinality two
  pttk_status greedy_init(Rng& rng, int max_it, std::vector<std::vector<Tup>>& left,
                          std::vector<std::vector<Tup>>& right) {
    const int N = D;
    std::vector<int> q1(N, 0), q2(N, 0);
    for (int j = 1; j < N; ++j) q1[j] = rng.below(n);
    for (int j = 1; j < N; ++j) q2[j] = rng.below(n);
    left.assign(N + 1, {});
    right.assign(N + 1, {});
    left[0] = {Tup()};
    left[N] = {Tup()};
    right[0] = {Tup()};
    right[N] = {Tup()};
    for (int k = 1; k < N; ++k) right[k] = {Tup(q1.begin() + k, q1.end()), Tup(q2.begin() + k, q2.end())};
    struct Cand {
      std::vector<std::vector<Tup>> l, r;
      double c;
    };
    std::vector<Cand> cands;
    auto best_pair = [&](const Tup& p, const Tup& pp, const Tup& a, const Tup& b, bool skip_eq, bool fwd,
                         int* j1o, int* j2o, double* bo) -> pttk_status {
      std::vector<int> idx;
      std::vector<std::pair<int, int>> pairs;
      for (int j1 = 0; j1 < n; ++j1)
        for (int j2 = 0; j2 < n; ++j2) {
          if (skip_eq && j1 == j2) continue;
          pairs.push_back({j1, j2});
          const Tup t1{j1}, t2{j2};
          if (fwd) {
            push(idx, p, t1, a);
            push(idx, p, t1, b);
            push(idx, pp, t2, a);
            push(idx, pp, t2, b);
          } else {
            push(idx, p, t1, a);
            push(idx, p, t2, b);
            push(idx, pp, t1, a);
            push(idx, pp, t2, b);
          }
        }
      const int m = (int)pairs.size();
      Dev dv;
      double *e = nullptr, *c = nullptr;
      PTTK_TRY(dv.get(&e, 4 * (size_t)m));
      PTTK_TRY(dv.get(&c, m));
      PTTK_TRY(eval(idx, e, dv));
      cond2_kernel<<<(m + 255) / 256, 256, 0, s>>>(e, m, c); pttk::count_launch();
      std::vector<double> ch(m);
      PTTK_CUDA(cudaMemcpyAsync(ch.data(), c, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
      PTTK_CUDA(cudaStreamSynchronize(s));
      const int q = first_argmin(ch);
      *j1o = pairs[q].first;
      *j2o = pairs[q].second;
      *bo = ch[q];
      return PTTK_OK;
    };
    for (int it = 0; it < max_it; ++it) {
      double cmax = -INFINITY;
      for (int k = 1; k < N; ++k) {
        const Tup p = left[k - 1][0], pp = k == 1 ? left[k - 1][0] : left[k - 1][1];
        const Tup a = right[k][0], b = right[k][1];
        int j1, j2;
        double best;
        PTTK_TRY(best_pair(p, pp, a, b, k == 1, true, &j1, &j2, &best));
        Tup l1 = p, l2 = pp;
        l1.push_back(j1);
        l2.push_back(j2);
        left[k] = {l1, l2};
        cmax = std::max(cmax, best);
      }
      cands.push_back({left, right, cmax});
      cmax = -INFINITY;
      for (int k = N; k > 1; --k) {
        const Tup p = left[k - 1][0], pp = left[k - 1][1];
        const Tup a = right[k][0], b = k == N ? right[k][0] : right[k][1];
        int j1, j2;
        double best;
        PTTK_TRY(best_pair(p, pp, a, b, k == N, false, &j1, &j2, &best));
        Tup r1{j1}, r2{j2};
        r1.insert(r1.end(), a.begin(), a.end());
        r2.insert(r2.end(), b.begin(), b.end());
        right[k - 1] = {r1, r2};
        cmax = std::max(cmax, best);
      }
      cands.push_back({left, right, cmax});
    }
    std::vector<double> cs;
    for (auto& c : cands) cs.push_back(c.c);
    const int i = first_argmin(cs);
    left = cands[i].l;
    right = cands[i].r;
    return PTTK_OK;
  }

  // the skeleton residual of Algorithm 5 at positions (ri, cj) of the super-core unfolding
  struct Unfold {
    const std::vector<Tup>* L;
    const std::vector<Tup>* Rn;
    int nk1;
    Tup multi(int i, int j) const {
      const int nl = (int)L->size();
      Tup t = (*L)[i % nl];
      t.push_back(i / nl);
      t.push_back(j % nk1);
      const Tup& rr = (*Rn)[j / nk1];
      t.insert(t.end(), rr.begin(), rr.end());
      return t;
    }
  };
  pttk_status residual(const Unfold& U, const std::vector<int>& I, const std::vector<int>& J,
                       const std::vector<int>& ri, const std::vector<int>& cj, std::vector<double>& R,
                       double* amax) {
    const int r = (int)I.size(), m = (int)ri.size();
    std::vector<int> idx;
    idx.reserve((size_t)(r * r + 2 * r * m + m) * D);
    auto add = [&](int i, int j) {
      const Tup t = U.multi(i, j);
      idx.insert(idx.end(), t.begin(), t.end());
    };
    for (int b = 0; b < r; ++b)
      for (int a = 0; a < r; ++a) add(I[a], J[b]);           // P, column-major
    for (int j = 0; j < r; ++j)
      for (int p = 0; p < m; ++p) add(ri[p], J[j]);          // left: m x r column-major
    for (int p = 0; p < m; ++p)
      for (int a = 0; a < r; ++a) add(I[a], cj[p]);          // right: r x m column-major
    for (int p = 0; p < m; ++p) add(ri[p], cj[p]);           // a
    Dev dv;
    double *E = nullptr, *work = nullptr, *Rd = nullptr;
    PTTK_TRY(dv.get(&E, idx.size() / D));
    PTTK_TRY(dv.get(&work, (size_t)r * r));
    PTTK_TRY(dv.get(&Rd, m));
    PTTK_TRY(eval(idx, E, dv));
    double* P = E;
    double* Lm = E + (size_t)r * r;
    double* Rm = Lm + (size_t)r * m;
    double* av = Rm + (size_t)r * m;
    lu_solve_kernel<<<1, 256, 0, s>>>(P, r, Rm, m, work); pttk::count_launch();
    residual_kernel<<<(m * 32 + 255) / 256, 256, 0, s>>>(Lm, Rm, av, m, r, Rd); pttk::count_launch();
    PTTK_CUDA(cudaGetLastError());
    R.resize(m);
    std::vector<double> ah(m);
    PTTK_CUDA(cudaMemcpyAsync(R.data(), Rd, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
    PTTK_CUDA(cudaMemcpyAsync(ah.data(), av, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
    PTTK_CUDA(cudaStreamSynchronize(s));
    double am = 0.0;
    for (double v : ah) am = std::max(am, std::fabs(v));
    *amax = am;
    return PTTK_OK;
  }

  // Algorithm 5: the new pivot (l, t) of the cross (I, J), or none
  pttk_status update_cross(const Unfold& U, int rows, int cols, const std::vector<int>& I, const std::vector<int>& J,
                           Rng& rng, bool* found, int* lo, int* to) {
    *found = false;
    const int64_t total = (int64_t)rows * cols;
    const int want = std::max(rows, cols);
    std::vector<int64_t> S;
    if (want >= total) {
      for (int64_t e = 0; e < total; ++e) S.push_back(e);
    } else {
      std::map<int64_t, char> seen;
      while ((int)S.size() < want) {
        const int64_t e = (int64_t)(rng.u64() % (uint64_t)total);
        if (seen.emplace(e, 1).second) S.push_back(e);
      }
    }
    std::vector<int> si(S.size()), sj(S.size());
    for (size_t q = 0; q < S.size(); ++q) {
      si[q] = (int)(S[q] % rows);
      sj[q] = (int)(S[q] / rows);
    }
    std::vector<double> R;
    double amax = 0.0, am = 0.0;
    PTTK_TRY(residual(U, I, J, si, sj, R, &amax));
    std::vector<double> absR(R.size());
    for (size_t q = 0; q < R.size(); ++q) absR[q] = std::fabs(R[q]);
    const int q = first_argmax(absR);
    int l = si[q], t = sj[q];
    double val;
    if (rng.bit() == 1) {
      std::vector<int> ri(cols, l), cj(cols);
      for (int j = 0; j < cols; ++j) cj[j] = j;
      PTTK_TRY(residual(U, I, J, ri, cj, R, &am));
      absR.resize(R.size());
      for (size_t p = 0; p < R.size(); ++p) absR[p] = std::fabs(R[p]);
      t = first_argmax(absR);
      val = R[t];
    } else {
      std::vector<int> ri(rows), cj(rows, t);
      for (int i = 0; i < rows; ++i) ri[i] = i;
      PTTK_TRY(residual(U, I, J, ri, cj, R, &am));
      absR.resize(R.size());
      for (size_t p = 0; p < R.size(); ++p) absR[p] = std::fabs(R[p]);
      l = first_argmax(absR);
      val = R[l];
    }
    amax = std::max(amax, am);
    bool in_i = false, in_j = false;
    for (int v : I) in_i = in_i || v == l;
    for (int v : J) in_j = in_j || v == t;
    if (!(std::fabs(val) > 1e-14 * amax) || in_i || in_j) return PTTK_OK;
    *found = true;
    *lo = l;
    *to = t;
    return PTTK_OK;
  }

  // interpolation cores C_k^{2} = T_k^{2} P_k^{-1} (k < N), C_N = T_N (reading X3), on the
  // device into `cores` (packed, offsets off[k])
  pttk_status cross_cores(const std::vector<std::vector<Tup>>& left, const std::vector<std::vector<Tup>>& right,
                          std::vector<int>& ranks, std::vector<int64_t>& off, double** cores_dev, Dev& keep) {
    const int N = D;
    ranks.assign(N + 1, 1);
    for (int k = 1; k < N; ++k) ranks[k] = (int)left[k].size();
    off.assign(N + 1, 0);
    for (int k = 0; k < N; ++k) off[k + 1] = off[k] + (int64_t)ranks[k] * n * ranks[k + 1];
    double* C = nullptr;
    PTTK_TRY(keep.get(&C, off[N]));
    for (int k = 1; k <= N; ++k) {
      const std::vector<Tup>& L = left[k - 1];
      const std::vector<Tup>& Rt = right[k];
      std::vector<int> idx;
      for (const Tup& r : Rt)
        for (int i = 0; i < n; ++i)
          for (const Tup& l : L) push(idx, l, Tup{i}, r);
      double* T = C + off[k - 1];
      Dev dv;
      PTTK_TRY(eval(idx, T, dv));
      if (k < N) {
        // P_k[a, b] = X(left[k][a] + right[k][b]); C2 = T2 P_k^{-1}: solve P_k^T Y = T2^T, C2 = Y^T
        const int rk = ranks[k];
        const int64_t mrow = (int64_t)L.size() * n;
        std::vector<int> pidx;
        for (int a = 0; a < rk; ++a)          // P_k^T column-major: element (b, a) at b + rk a
          for (int b = 0; b < rk; ++b) push(pidx, left[k][a], Tup(), right[k][b]);
        double *Pt = nullptr, *Y = nullptr, *work = nullptr;
        PTTK_TRY(dv.get(&Pt, (size_t)rk * rk));
        PTTK_TRY(dv.get(&Y, (size_t)rk * mrow));
        PTTK_TRY(dv.get(&work, (size_t)rk * rk));
        PTTK_TRY(eval(pidx, Pt, dv));
        // Y (rk x mrow, column-major) = T2^T, T2 = T as (mrow x rk) column-major
        std::vector<double> th((size_t)mrow * rk), yh((size_t)rk * mrow);
        PTTK_CUDA(cudaMemcpyAsync(th.data(), T, sizeof(double) * th.size(), cudaMemcpyDeviceToHost, s));
        PTTK_CUDA(cudaStreamSynchronize(s));
        for (int64_t i = 0; i < mrow; ++i)
          for (int b = 0; b < rk; ++b) yh[b + (size_t)rk * i] = th[i + (size_t)mrow * b];
        PTTK_CUDA(cudaMemcpyAsync(Y, yh.data(), sizeof(double) * yh.size(), cudaMemcpyHostToDevice, s));
        lu_solve_kernel<<<1, 256, 0, s>>>(Pt, rk, Y, (int)mrow, work); pttk::count_launch();
        PTTK_CUDA(cudaGetLastError());
        PTTK_CUDA(cudaMemcpyAsync(yh.data(), Y, sizeof(double) * yh.size(), cudaMemcpyDeviceToHost, s));
        PTTK_CUDA(cudaStreamSynchronize(s));
        for (int64_t i = 0; i < mrow; ++i)
          for (int b = 0; b < rk; ++b) th[i + (size_t)mrow * b] = yh[b + (size_t)rk * i];
        PTTK_CUDA(cudaMemcpyAsync(T, th.data(), sizeof(double) * th.size(), cudaMemcpyHostToDevice, s));
        PTTK_CUDA(cudaStreamSynchronize(s));
      }
    }
    *cores_dev = C;
    return PTTK_OK;
  }

  // the largest |x - x^| over n_check random entries, relative to the largest |x| among them
  pttk_status check_error(const double* cores, const std::vector<int>& ranks, const std::vector<int64_t>& off,
                          Rng& rng, int n_check, double* err) {
    std::vector<int> idx((size_t)n_check * D);
    for (int q = 0; q < n_check; ++q)
      for (int k = 0; k < D; ++k) idx[(size_t)q * D + k] = rng.below(n);
    Dev dv;
    double *x = nullptr, *xh = nullptr;
    int *di = nullptr, *dr = nullptr;
    int64_t* doff = nullptr;
    PTTK_TRY(dv.get(&x, n_check));
    PTTK_TRY(dv.get(&xh, n_check));
    PTTK_TRY(dv.get(&di, idx.size()));
    PTTK_TRY(dv.get(&dr, ranks.size()));
    PTTK_TRY(dv.get(&doff, off.size()));
    PTTK_TRY(eval(idx, x, dv));
    PTTK_CUDA(cudaMemcpyAsync(di, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice, s));
    PTTK_CUDA(cudaMemcpyAsync(dr, ranks.data(), sizeof(int) * ranks.size(), cudaMemcpyHostToDevice, s));
    PTTK_CUDA(cudaMemcpyAsync(doff, off.data(), sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice, s));
    int rmax = 1;
    for (int r : ranks) rmax = std::max(rmax, r);
    if (rmax > 1024) return set_error(PTTK_ENOTSUP, "greedy-cross: a rank above 1024");
    const int threads = std::max(32, ((rmax + 3) / 4 + 31) / 32 * 32);  // 4 threads' worth of entries each
    tt_eval_kernel<<<std::min(n_check, sm_count() * 8), threads, sizeof(double) * 8 * threads, s>>>(
        cores, doff, dr, D, n, di, n_check, xh); pttk::count_launch();
    PTTK_CUDA(cudaGetLastError());
    std::vector<double> a(n_check), b(n_check);
    PTTK_CUDA(cudaMemcpyAsync(a.data(), x, sizeof(double) * n_check, cudaMemcpyDeviceToHost, s));
    PTTK_CUDA(cudaMemcpyAsync(b.data(), xh, sizeof(double) * n_check, cudaMemcpyDeviceToHost, s));
    PTTK_CUDA(cudaStreamSynchronize(s));
    double num = 0.0, den = 0.0;
    for (int q = 0; q < n_check; ++q) {
      num = std::max(num, std::fabs(a[q] - b[q]));
      den = std::max(den, std::fabs(a[q]));
    }
    *err = den > 0.0 ? num / den : num;
    return PTTK_OK;
  }
};

}  // namespace
}  // namespace pttk

using namespace pttk;

extern "C" pttk_status pttk_cross_build(pttk_kernel kernel, int d, const double* src_box, const double* tgt_box,
                                        int d_theta, const double* theta_box, int n, double eps, uint64_t key,
                                        int max_sweeps, int n_check, int init_it, void* stream, pttk_tt** out,
                                        int* sweeps_out, int64_t* evals_out) {
  clear_error();
  if (!out) return set_error(PTTK_EINVAL, "NULL out");
  *out = nullptr;
  // the problem checks of the grid-entry call (boxes, kernel, d_theta, n)
  PTTK_TRY(pttk_grid_entries(kernel, d, src_box, tgt_box, d_theta, theta_box, n, nullptr, 0, PTTK_FP64, nullptr,
                             stream));
  if (!(eps > 0.0 && eps < 1.0)) return set_error(PTTK_EINVAL, "eps must lie in (0, 1)");
  if (max_sweeps < 0 || n_check < 1 || init_it < 1) return set_error(PTTK_EINVAL, "bad sweep, check or init count");
  Cross cx;
  cx.kernel = kernel;
  cx.d = d;
  cx.dth = d_theta;
  cx.D = 2 * d + d_theta;
  cx.n = n;
  cx.s = as_stream(stream);
  if (cx.D < 2) return set_error(PTTK_EINVAL, "the tensor needs at least two modes");
  for (int j = 0; j < d; ++j) {
    cx.box[j][0] = src_box[2 * j];
    cx.box[j][1] = src_box[2 * j + 1];
    cx.box[d + d_theta + j][0] = tgt_box[2 * j];
    cx.box[d + d_theta + j][1] = tgt_box[2 * j + 1];
  }
  for (int j = 0; j < d_theta; ++j) {
    cx.box[d + j][0] = theta_box[2 * j];
    cx.box[d + j][1] = theta_box[2 * j + 1];
  }
  Dev keep;
  PTTK_TRY(keep.get(&cx.d_status, 1));
  PTTK_CUDA(cudaMemsetAsync(cx.d_status, 0, sizeof(int), cx.s));
  Rng rng{key};
  std::vector<std::vector<Tup>> left, right;
  PTTK_TRY(cx.greedy_init(rng, init_it, left, right));
  const int N = cx.D;
  int sweeps = 0;
  std::vector<int> ranks;
  std::vector<int64_t> off;
  double* cores = nullptr;
  while (true) {
    Dev ck;
    PTTK_TRY(cx.cross_cores(left, right, ranks, off, &cores, keep));
    double err = 0.0;
    PTTK_TRY(cx.check_error(cores, ranks, off, rng, n_check, &err));
    if (err <= eps || sweeps >= max_sweeps) break;
    ++sweeps;
    int added = 0;
    for (int k = 1; k < N; ++k) {
      const std::vector<Tup>& L = left[k - 1];
      const std::vector<Tup>& Rn = right[k + 1];
      const int nl = (int)L.size(), nr = (int)Rn.size();
      const int rows = nl * n, cols = n * nr;
      Cross::Unfold U{&L, &Rn, n};
      std::vector<int> I, J;
      for (const Tup& l : left[k]) {
        const Tup pre(l.begin(), l.end() - 1);
        int pos = 0;
        while (pos < nl && L[pos] != pre) ++pos;
        I.push_back(pos + nl * l.back());
      }
      for (const Tup& r : right[k]) {
        const Tup suf(r.begin() + 1, r.end());
        int pos = 0;
        while (pos < nr && Rn[pos] != suf) ++pos;
        J.push_back(r[0] + n * pos);
      }
      bool found = false;
      int l = 0, t = 0;
      PTTK_TRY(cx.update_cross(U, rows, cols, I, J, rng, &found, &l, &t));
      if (!found) continue;
      Tup nl_t = L[l % nl];
      nl_t.push_back(l / nl);
      Tup nr_t{t % n};
      const Tup& suf = Rn[t / n];
      nr_t.insert(nr_t.end(), suf.begin(), suf.end());
      left[k].push_back(nl_t);
      right[k].push_back(nr_t);
      ++added;
    }
    if (added == 0) break;
  }
  int h = 0;
  PTTK_CUDA(cudaMemcpy(&h, cx.d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (h != 0) return set_error(PTTK_ECUDA, "greedy-cross: an entry index left the grid");
  // Chebyshev transform of every core (the coefficient form), then the handle
  double* tcores = nullptr;
  PTTK_TRY(keep.get(&tcores, off[N]));
  for (int k = 0; k < N; ++k) {
    const int64_t e = off[k + 1] - off[k];
    core_transform_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((e + 255) / 256, 4096)), 256, 0, cx.s>>>(
        cores + off[k], ranks[k], n, ranks[k + 1], tcores + off[k]); pttk::count_launch();
  }
  PTTK_CUDA(cudaGetLastError());
  std::vector<double> host(off[N]);
  PTTK_CUDA(cudaMemcpyAsync(host.data(), tcores, sizeof(double) * host.size(), cudaMemcpyDeviceToHost, cx.s));
  PTTK_CUDA(cudaStreamSynchronize(cx.s));
  if (sweeps_out) *sweeps_out = sweeps;
  if (evals_out) *evals_out = cx.evals;
  return pttk_tt_from_cores(kernel, d, src_box, tgt_box, d_theta, theta_box, n, ranks.data(), host.data(), out);
}

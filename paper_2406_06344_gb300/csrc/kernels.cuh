// Kernel functions of Table kern-table evaluated on the device, including a hand-written
// modified Bessel function of the second kind K_nu for the general-nu Matern kernel.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace pttk {

// Trapezoidal-rule table: s_j = cosh(t_j) - 1 = 2 sinh^2(t_j / 2) at t_j = j * KV_HMIN.
// The quadrature uses steps h_q = KV_H0 * 2^-q (q = 0..4), whose nodes are every
// (16 >> q)-th table entry.
constexpr double KV_H0 = 0.18;
constexpr double KV_HMIN = KV_H0 / 16.0;
constexpr int KV_TABLE = 1424;  // covers t <= 16

template <typename T>
struct KvEps;
template <>
struct KvEps<double> {
  static constexpr double stop = 1e-18;
};
template <>
struct KvEps<float> {
  static constexpr float stop = 1e-9f;
};

// e^x K_nu(x) for x > 0 by the trapezoidal rule applied to the integral representation
//   K_nu(x) = int_0^inf e^{-x cosh t} cosh(nu t) dt
//           = e^{-x} int_0^inf e^{-x s(t)} cosh(nu t) dt,  s(t) = cosh t - 1.
// The integrand is even, analytic and decays doubly exponentially, so the trapezoidal sum
// h [1/2 + sum_{k>=1} g(k h)] converges exponentially in 1/h (Trefethen & Weideman,
// SIAM Review 56 (2014), "The exponentially convergent trapezoidal rule"). The step is
// halved until h <= pi^2 / (x + 33 + 3 nu): the discretisation error behaves like
// exp(x cosh(t*) (1 - cos a) - 2 pi a / h) for a strip half-width a < pi/2, where t* is
// where the integrand peaks (sinh t* ~ nu / x), so the margin grows with nu. Against
// 30-digit values the scaled result is within 1.8e-15 (relative) for 0.5 <= x <= 20,
// nu in [0.5, 2.5], within 1.2e-15 for 8 <= x <= 20, nu in [3, 5], and within 2.9e-15 for
// 0.05 <= x <= 700, nu <= 5: the rounding level of the sum (a fixed margin of 60 is no
// better). A fixed margin of 38 loses accuracy for nu > 2.5 (1.2e-14 at x = 16, nu = 5).
// All terms are positive, so the sum has no
// cancellation. Summation stops once a term is below KvEps::stop of the running sum on
// the decreasing side of the integrand (x sinh t > nu), with a hard cap on nodes.
template <typename T>
__device__ __forceinline__ T kv_scaled(T nu, T x, const T* __restrict__ stab) {
  int q = 0;
  T h = T(KV_H0);
  const T hmax = T(9.869604401089358) / (x + T(33) + T(3) * nu);
  while (q < 4 && h > hmax) {
    h *= T(0.5);
    ++q;
  }
  const int stride = 16 >> q;
  const T E = exp(nu * h);
  const T Ei = T(1) / E;
  T Ek = T(1), Eik = T(1);
  T acc = T(0.5);
  for (int k = 1; k < 1024; ++k) {
    const int j = k * stride;
    T s;
    if (j < KV_TABLE) {
      s = stab[j];
    } else {
      const T sh = sinh(T(0.5) * T(k) * h);
      s = T(2) * sh * sh;
    }
    Ek *= E;
    Eik *= Ei;
    const T term = exp(-x * s) * T(0.5) * (Ek + Eik);
    acc += term;
    if (term < KvEps<T>::stop * acc && x * x * s * (s + T(2)) > nu * nu) break;
  }
  return h * acc;
}

// Fill the trapezoid table s_j = 2 sinh^2(j h_min / 2), j < KV_TABLE (cooperatively).
template <typename T>
__device__ __forceinline__ void kv_table_fill(T* stab) {
  for (int j = threadIdx.x; j < KV_TABLE; j += blockDim.x) {
    const double sh = sinh(0.5 * KV_HMIN * (double)j);
    stab[j] = (T)(2.0 * sh * sh);
  }
}

enum {
  K_GAUSS = 0,
  K_MATERN32 = 1,
  K_MATERN_NU = 2,
  K_EXPONENTIAL = 3,
  K_MATERN52 = 4,
  K_MULTIQUADRIC = 5,
  K_THIN_PLATE_SPLINE = 6,
  K_BIHARMONIC = 7,
  K_LAPLACE3D = 8,
  K_LAPLACE2D = 9,
  K_THIN_PLATE = 10
};

// kappa(r; l) of the closed-form kernels, from r^2 (l is unused by the kernels without a
// parameter, whose boxes are apart, so r > 0 there).
template <typename T>
__device__ __forceinline__ T kappa_l(int kind, T r2, T l) {
  switch (kind) {
    case K_GAUSS: return exp(-r2 / (l * l));
    case K_MATERN32: {
      const T a = T(1.7320508075688772) * sqrt(r2) / l;
      return (T(1) + a) * exp(-a);
    }
    case K_EXPONENTIAL: return exp(-sqrt(r2) / l);
    case K_MATERN52: {
      const T a = T(2.23606797749979) * sqrt(r2) / l;
      return (T(1) + a + a * a / T(3)) * exp(-a);
    }
    case K_MULTIQUADRIC: return sqrt(T(1) + r2 / (l * l));
    case K_THIN_PLATE_SPLINE: {
      const T q = r2 / (l * l);
      return q > T(0) ? q * log(q) : T(0);
    }
    case K_BIHARMONIC: return T(1) / r2;
    case K_LAPLACE3D: return T(1) / sqrt(r2);
    case K_LAPLACE2D: return T(-0.5) * log(r2);
    default: return T(0.5) * r2 * log(r2);  // K_THIN_PLATE: r^2 log r
  }
}

// Matern general nu: 2^(1-nu)/Gamma(nu) z^nu K_nu(z), z = sqrt(2 nu) r / l.
// `cnu` = 2^(1-nu)/Gamma(nu), `snu` = sqrt(2 nu) (per-node constants).
template <typename T>
__device__ __forceinline__ T kappa_matern_nu(T r2, T l, T nu, T cnu, T snu,
                                             const T* __restrict__ stab) {
  const T z = snu * sqrt(r2) / l;
  if (!(z > T(0))) return T(1);
  if (z > T(700)) return T(0);
  return cnu * exp(nu * log(z) - z) * kv_scaled<T>(nu, z, stab);
}

}  // namespace pttk

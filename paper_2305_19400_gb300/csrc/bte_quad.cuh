// bte_quad.cuh -- band equilibrium intensity by Gauss-Legendre quadrature (FP64).
#pragma once
#include "bte_internal.h"

namespace bte {

// Band quadrature.  I0_b(T) = sum_i C_i / expm1(c_i / T) (Gauss-Legendre on the
// band).  With n = 1/(e^x - 1), x = c/T:  dn/dT = n(1+n) x/T and
// d2n/dT2 = n(1+n) (x/T^2) ((1+2n) x - 2).
__device__ __forceinline__ double band_I0(const double* __restrict__ c, const double* __restrict__ C, int ng,
                                          double rT) {
  double s = 0.0;
  for (int i = 0; i < ng; ++i) s = fma(C[i], 1.0 / expm1(c[i] * rT), s);
  return s;
}

__device__ __forceinline__ void band_I0_d2(const double* __restrict__ c, const double* __restrict__ C, int ng,
                                           double rT, double& f, double& d1, double& d2) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int i = 0; i < ng; ++i) {
    const double x = c[i] * rT;
    const double n = 1.0 / expm1(x);
    const double qx = fma(n, n, n) * x;
    const double u = fma(2.0 * n, x, x) - 2.0;
    s0 = fma(C[i], n, s0);
    s1 = fma(C[i], qx, s1);
    s2 = fma(C[i] * qx, u, s2);
  }
  f = s0;
  d1 = s1 * rT;
  d2 = s2 * rT * rT;
}

}  // namespace bte

// bte_solve.cuh -- exact FP64 solve of the T_p equation for one cell by one warp.
#pragma once
#include "bte_quad.cuh"

namespace bte {

struct SolveResult {
  double Te;     // last exact evaluation point (its I0, dI0/dT, d2I0/dT2 are in Jrow)
  double delta;  // accepted step from Te: T_p = Te + delta
  int evals;     // exact band-quadrature evaluations
  int fallback;  // 1 when bisection was needed
  int bad;       // 1 when no temperature in [1, 5000] K was found
  double M[3];   // sum_b w_b (I0_b, dI0_b/dT, d2I0_b/dT2) at Te: the cell's model sums
};

// Solves sum_b w_b I0_b(T) = Ep (w = a_p unless given) from T0 by Halley steps on the exact band
// quadrature (F, F', F'' from one evaluation), bisection on [1, 5000] K as the
// fallback.  A step delta is accepted when |delta| <= trust_rel * T, where the
// second-order Taylor model at the evaluation point is accurate to the solve
// tolerance.  Each evaluation's I0, dI0/dT, d2I0/dT2 per band are written to
// Jrow ([3][nbp], may be null).  All 32 lanes of the warp must call it.
__device__ inline SolveResult exact_solve_warp(const ThermoTables& th, double Ep, double T0, double trust_rel, int maxit,
                                               double* Jrow, const double* wts = nullptr) {
  const double* wb = wts ? wts : th.a_p;
  const int lane = threadIdx.x & 31;
  const int nbp = th.nbp, ng = th.ng;
  double T = (T0 >= kTmin && T0 <= kTmax && isfinite(T0)) ? T0 : 300.0;
  double lo = kTmin, hi = kTmax, delta = 0.0;
  int mode = 0, iters = 0;  // 0 Halley, 1 bisection, 2 final
  SolveResult r{T, 0.0, 0, 0, 0, {0.0, 0.0, 0.0}};
  bool done = false;
  for (int loop = 0; loop < maxit + 224 && !done; ++loop) {
    const double rT = 1.0 / T;
    double F = 0.0, F1 = 0.0, F2 = 0.0;
    for (int b = lane; b < nbp; b += 32) {
      double f, d1, d2;
      band_I0_d2(th.node_c + b * ng, th.node_C + b * ng, ng, rT, f, d1, d2);
      if (Jrow) {
        Jrow[b] = f;
        Jrow[nbp + b] = d1;
        Jrow[2 * nbp + b] = d2;
      }
      const double ap = wb[b];
      F = fma(ap, f, F);
      F1 = fma(ap, d1, F1);
      F2 = fma(ap, d2, F2);
    }
    for (int o = 16; o > 0; o >>= 1) {
      F += __shfl_xor_sync(0xffffffffu, F, o);
      F1 += __shfl_xor_sync(0xffffffffu, F1, o);
      F2 += __shfl_xor_sync(0xffffffffu, F2, o);
    }
    r.M[0] = F;
    r.M[1] = F1;
    r.M[2] = F2;
    F -= Ep;
    ++r.evals;
    r.Te = T;
    if (mode == 0) {
      ++iters;
      bool badstep = !(isfinite(F) && isfinite(F1) && F1 > 0.0);
      double Tn = T;
      if (!badstep) {
        const double newton = -F / F1;
        const double h = F * F2 / (2.0 * F1 * F1);
        delta = fabs(h) < 0.5 ? newton / (1.0 - h) : newton;
        Tn = T + delta;
        badstep = !(Tn >= kTmin && Tn <= kTmax) || iters > maxit;
      }
      if (badstep) {
        mode = 1;
        lo = kTmin;
        hi = kTmax;
        T = 0.5 * (lo + hi);
        r.fallback = 1;
      } else if (fabs(delta) <= trust_rel * Tn) {
        done = true;
      } else {
        T = Tn;
      }
    } else if (mode == 1) {
      if (F < 0.0) lo = T; else hi = T;
      T = 0.5 * (lo + hi);
      ++iters;
      if (hi - lo <= 4e-16 * hi || iters >= maxit + 200) mode = 2;
    } else {
      delta = 0.0;
      done = true;
      if (T <= kTmin * (1.0 + 1e-9) || T >= kTmax * (1.0 - 1e-9)) r.bad = 1;
    }
  }
  if (!done) {
    r.bad = 1;
    delta = 0.0;
  }
  r.delta = delta;
  return r;
}

}  // namespace bte

// bte_solve.cuh -- exact FP64 solve of the T_p equation for one cell, by one warp or one thread-block cluster.
#pragma once
#include <cooperative_groups.h>
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

// Control of the exact solve of sum_b w_b I0_b(T) = Ep: Halley steps from T0
// on the exact band quadrature (F, F', F'' from one evaluation), bisection on
// [1, 5000] K as the fallback.  A step delta is accepted when
// |delta| <= trust_rel * T, where the second-order Taylor model at the
// evaluation point is accurate to the solve tolerance.  Shared by the warp
// and the CTA forms below, so both take the same decisions from the same sums.
struct SolveCtl {
  double T, lo, hi, delta;
  int mode, iters;  // mode 0 Halley, 1 bisection, 2 final
  bool done;
  SolveResult r;

  __device__ explicit SolveCtl(double T0)
      : T((T0 >= kTmin && T0 <= kTmax && isfinite(T0)) ? T0 : 300.0), lo(kTmin), hi(kTmax), delta(0.0), mode(0),
        iters(0), done(false), r{T, 0.0, 0, 0, 0, {0.0, 0.0, 0.0}} {}

  // One evaluation's sums at T; moves T to the next evaluation point or sets done.
  __device__ void advance(double F, double F1, double F2, double Ep, double trust_rel, int maxit) {
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

  __device__ SolveResult finish() {
    if (!done) {
      r.bad = 1;
      delta = 0.0;
    }
    r.delta = delta;
    return r;
  }
};

// Exact solve by one warp (w = a_p unless given): lanes over bands.  Each
// evaluation's I0, dI0/dT, d2I0/dT2 per band are written to Jrow ([3][nbp],
// may be null).  All 32 lanes of the warp must call it.
__device__ inline SolveResult exact_solve_warp(const ThermoTables& th, double Ep, double T0, double trust_rel, int maxit,
                                               double* Jrow, const double* wts = nullptr) {
  const double* wb = wts ? wts : th.a_p;
  const int lane = threadIdx.x & 31;
  const int nbp = th.nbp, ng = th.ng;
  SolveCtl c(T0);
  for (int loop = 0; loop < maxit + 224 && !c.done; ++loop) {
    const double rT = 1.0 / c.T;
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
    c.advance(F, F1, F2, Ep, trust_rel, maxit);
  }
  return c.finish();
}

// Shared memory (doubles) of exact_solve_cluster, per CTA.
constexpr int kCtaSolvePairs = 1024;  // (band, node) pairs per chunk
__host__ __device__ inline int cta_solve_smem_doubles(int nbp) { return 3 * kCtaSolvePairs + 6 * nbp + 4; }

// The same solve by a thread-block cluster, bit for bit the warp form's
// results.  CTA r of the C in the cluster evaluates the bands
// [r nbp / C, (r + 1) nbp / C): the costly per-node terms (expm1, the
// reciprocal, the derivative factors) are spread over its threads, and each
// band's node sum runs in node order on one thread, writing f, f', f'' to the
// CTA's own shared memory (and the cell's model row Jrow).  After one cluster
// barrier warp 0 of every CTA adds all bands through distributed shared
// memory in the warp form's order, so every CTA holds the same F, F', F'' and
// advances the same controller, and the loop ends on the same evaluation
// everywhere.  The band values alternate between two buffers over the
// cluster's successive evaluations (par counts them across calls): evaluation
// k writes buffer k % 2 after the barrier of evaluation k - 1, which every
// reader of buffer (k - 2) % 2 has passed.  One cell's evaluation thus runs
// on C SMs' FP64 units.  sm: cta_solve_smem_doubles(nbp) doubles per CTA.
// Every thread of every CTA of the cluster must call it (it synchronises the
// cluster).
__device__ inline SolveResult exact_solve_cluster(const ThermoTables& th, double Ep, double T0, double trust_rel,
                                                  int maxit, double* Jrow, double* sm, unsigned& par) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank(), nr = (int)cl.num_blocks();
  const double* wb = th.a_p;
  const int nbp = th.nbp, ng = th.ng;
  const int own0 = rank * nbp / nr, own1 = (rank + 1) * nbp / nr;  // this CTA's bands
  const int cb = kCtaSolvePairs / ng;  // bands per chunk (ng <= kMaxGauss)
  double* pn = sm;                      // [pairs] n = 1 / expm1(x)
  double* pq = pn + kCtaSolvePairs;     // [pairs] n (1 + n) x
  double* pu = pq + kCtaSolvePairs;     // [pairs] (1 + 2n) x - 2
  double* bv2 = pu + kCtaSolvePairs;    // [2][3][nbp] per band f, d1, d2 (own bands), two buffers
  double* sums = bv2 + 6 * nbp;         // [3] this CTA's copy of F, F', F''
  SolveCtl c(T0);
  for (int loop = 0; loop < maxit + 224 && !c.done; ++loop) {
    double* bv = bv2 + (size_t)(par++ & 1u) * 3 * nbp;
    const double rT = 1.0 / c.T;
    for (int b0 = own0; b0 < own1; b0 += cb) {
      const int npair = min(cb, own1 - b0) * ng;
      const double* cn = th.node_c + b0 * ng;
      for (int p = threadIdx.x; p < npair; p += blockDim.x) {
        const double x = cn[p] * rT;
        const double n = 1.0 / expm1(x);
        pn[p] = n;
        pq[p] = fma(n, n, n) * x;
        pu[p] = fma(2.0 * n, x, x) - 2.0;
      }
      __syncthreads();
      for (int k = threadIdx.x; k < npair / ng; k += blockDim.x) {
        const int b = b0 + k;
        const double* C = th.node_C + b * ng;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (int i = 0; i < ng; ++i) {
          const int p = k * ng + i;
          s0 = fma(C[i], pn[p], s0);
          s1 = fma(C[i], pq[p], s1);
          s2 = fma(C[i] * pq[p], pu[p], s2);
        }
        const double f = s0, d1 = s1 * rT, d2 = s2 * rT * rT;
        bv[b] = f;
        bv[nbp + b] = d1;
        bv[2 * nbp + b] = d2;
        if (Jrow) {
          Jrow[b] = f;
          Jrow[nbp + b] = d1;
          Jrow[2 * nbp + b] = d2;
        }
      }
      __syncthreads();
    }
    cl.sync();  // every CTA's bands are in its bv
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      double F = 0.0, F1 = 0.0, F2 = 0.0;
      for (int b = lane; b < nbp; b += 32) {
        int o = (int)(((long long)b * nr) / nbp);  // the CTA whose range holds b
        while (o + 1 < nr && (o + 1) * nbp / nr <= b) ++o;
        while (o > 0 && o * nbp / nr > b) --o;
        const double* ob = cl.map_shared_rank(bv, (unsigned)o);
        const double ap = wb[b];
        F = fma(ap, ob[b], F);
        F1 = fma(ap, ob[nbp + b], F1);
        F2 = fma(ap, ob[2 * nbp + b], F2);
      }
      for (int o = 16; o > 0; o >>= 1) {
        F += __shfl_xor_sync(0xffffffffu, F, o);
        F1 += __shfl_xor_sync(0xffffffffu, F1, o);
        F2 += __shfl_xor_sync(0xffffffffu, F2, o);
      }
      if (lane == 0) {
        sums[0] = F;
        sums[1] = F1;
        sums[2] = F2;
      }
    }
    __syncthreads();
    c.advance(sums[0], sums[1], sums[2], Ep, trust_rel, maxit);
  }
  return c.finish();
}

}  // namespace bte

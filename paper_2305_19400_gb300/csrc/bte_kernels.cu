// bte_kernels.cu -- CUDA kernels of the phonon BTE hot path (sm_103a).
//
// sweep_kernel<DIM, S>: one launch per inner iteration.  A CTA owns a run of
//   cells of one geometry; each cell is served by `lpc` lanes, lane l holding
//   V consecutive bands as one vector (FP64: 2 doubles, FP32: 4 floats, BF16:
//   4 bf16).  Each lane walks every direction d (Sec. 3.1, Eq. 5):
//     implicit  I^{k+1} = A_n I^n + A_x I_up,x^k + A_y I_up,y^k (+ A_z I_up,z^k) + A_s I0^k
//     explicit  same form with forward-Euler coefficients and I^k = I^n
//   The upwind value is the neighbour cell on the side S_d comes from, or the
//   Eq. 6 ghost at a wall (I0 of the wall face, or the cell's own value in the
//   mirrored direction).  The FP32 and BF16 modes store the deviation
//   I - I0_b(T_ref): the update is affine with coefficients summing to one, so
//   the deviation obeys the same update with I0 and wall ghosts shifted by
//   I0_b(T_ref), and rounding acts on the small deviation only.
//   The lane accumulates G_b = sum_d w_d I^{k+1}_{d,b} in registers (FP64, or a
//   compensated float pair in the reduced modes), so the reduction needs no
//   shuffles.  The epilogue reduces the cell's lanes to E_L and E_p and solves
//   the T_p equation:
//     * first on the cell's cached quadratic model of I0_b(T) around its last
//       exact evaluation point T_e (I0, dI0/dT, d2I0/dT2 per band); the model
//       root is accepted when |T - T_e| <= trust_rel*T, where the Taylor
//       remainder is below the solve tolerance;
//     * otherwise by Halley steps on the exact FP64 band quadrature, which also
//       refresh the cached model; bisection on [1, 5000] K is the fallback.
//   I0 is refreshed from the accepted model.
// The HBM stream per update is I^n read, I^{k+1} written and I^k read once
// (neighbour rows come from L2 while adjacent cells are processed together).
#include <cuda_bf16.h>

#include "bte_internal.h"

namespace bte {

namespace {

enum SolveMode { M_MODEL = 0, M_HALLEY = 1, M_BISECT = 2, M_FINAL = 3, M_ACCEPT = 4, M_DONE = 5 };

// ---------------------------------------------------------------------------
// Storage traits: V values per vector load, arithmetic type A.
template <typename S> struct Tr;

template <> struct Tr<double> {
  static constexpr int V = 2;
  using A = double;
  static __device__ __forceinline__ void ld(const double* p, A (&x)[V]) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    x[0] = v.x; x[1] = v.y;
  }
  static __device__ __forceinline__ void ld_stream(const double* p, A (&x)[V]) {
    const double2 v = __ldcs(reinterpret_cast<const double2*>(p));
    x[0] = v.x; x[1] = v.y;
  }
  static __device__ __forceinline__ void st(double* p, const A (&x)[V]) {
    __stcs(reinterpret_cast<double2*>(p), make_double2(x[0], x[1]));
  }
  static __device__ __forceinline__ double to_double(double v) { return v; }
};

template <> struct Tr<float> {
  static constexpr int V = 4;
  using A = float;
  static __device__ __forceinline__ void ld(const float* p, A (&x)[V]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
  }
  static __device__ __forceinline__ void ld_stream(const float* p, A (&x)[V]) {
    const float4 v = __ldcs(reinterpret_cast<const float4*>(p));
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
  }
  static __device__ __forceinline__ void st(float* p, const A (&x)[V]) {
    __stcs(reinterpret_cast<float4*>(p), make_float4(x[0], x[1], x[2], x[3]));
  }
  static __device__ __forceinline__ double to_double(float v) { return (double)v; }
};

template <> struct Tr<__nv_bfloat16> {
  static constexpr int V = 4;
  using A = float;
  static __device__ __forceinline__ void unpack(const uint2 v, A (&x)[V]) {
    x[0] = __uint_as_float(v.x << 16);
    x[1] = __uint_as_float(v.x & 0xffff0000u);
    x[2] = __uint_as_float(v.y << 16);
    x[3] = __uint_as_float(v.y & 0xffff0000u);
  }
  static __device__ __forceinline__ void ld(const __nv_bfloat16* p, A (&x)[V]) {
    unpack(*reinterpret_cast<const uint2*>(p), x);
  }
  static __device__ __forceinline__ void ld_stream(const __nv_bfloat16* p, A (&x)[V]) {
    unpack(__ldcs(reinterpret_cast<const uint2*>(p)), x);
  }
  static __device__ __forceinline__ void st(__nv_bfloat16* p, const A (&x)[V]) {
    const __nv_bfloat162 h0 = __floats2bfloat162_rn(x[0], x[1]);  // round to nearest even
    const __nv_bfloat162 h1 = __floats2bfloat162_rn(x[2], x[3]);
    __stcs(reinterpret_cast<uint2*>(p),
           make_uint2(*reinterpret_cast<const unsigned*>(&h0), *reinterpret_cast<const unsigned*>(&h1)));
  }
  static __device__ __forceinline__ double to_double(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
};

// V consecutive values of type A from global memory (16-byte loads).
template <typename A, int V>
__device__ __forceinline__ void ldgv(const A* p, A (&x)[V]) {
  if constexpr (sizeof(A) == 8) {
#pragma unroll
    for (int i = 0; i < V; i += 2) {
      const double2 v = __ldg(reinterpret_cast<const double2*>(p + i));
      x[i] = v.x; x[i + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < V; i += 4) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(p + i));
      x[i] = v.x; x[i + 1] = v.y; x[i + 2] = v.z; x[i + 3] = v.w;
    }
  }
}

// ---------------------------------------------------------------------------
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

// ---------------------------------------------------------------------------
// Upwind value along axis AX for one lane of cell P in direction d.  Wall data
// use compile-time side indices so DevGeom stays in registers.
template <int AX, typename S>
__device__ __forceinline__ void upwind(const S* __restrict__ Ik, const SweepArgs& a, const DevGeom& g, const DirInfo& di,
                                       long long P, int ci, int cj, int ck, long long row, int d, int b0,
                                       typename Tr<S>::A (&x)[Tr<S>::V]) {
  using T = Tr<S>;
  const int c = AX == 0 ? ci : (AX == 1 ? cj : ck);
  const int n = AX == 0 ? g.nx : (AX == 1 ? g.ny : g.nz);
  const long long stride = AX == 0 ? 1 : (AX == 1 ? (long long)g.nx : (long long)g.nx * g.ny);
  const bool from_low = (di.up >> AX) & 1;
  const int nbp = a.th.nbp;
  if (from_low ? c > 0 : c < n - 1) {
    T::ld(Ik + (P + (from_low ? -stride : stride)) * row + (long long)d * nbp + b0, x);
    return;
  }
  const int bc = from_low ? g.bc[2 * AX] : g.bc[2 * AX + 1];
  if (bc == 0) {  // isothermal wall: I0_b of the face (as a deviation in the reduced modes)
    const long long f0 = from_low ? g.face0[2 * AX] : g.face0[2 * AX + 1];
    const long long f =
        f0 + (AX == 0 ? cj + (long long)g.ny * ck : (AX == 1 ? ci + (long long)g.nx * ck : ci + (long long)g.nx * cj));
    if constexpr (sizeof(S) == 8) ldgv<double, T::V>(a.I0wall + f * nbp + b0, x);
    else ldgv<float, T::V>(a.I0wall_dev + f * nbp + b0, x);
    return;
  }
  const int r = AX == 0 ? di.rx : (AX == 1 ? di.ry : di.rz);  // symmetry wall: mirrored direction
  T::ld(Ik + P * row + (long long)r * nbp + b0, x);
}

template <int DIM, typename S>
__global__ void __launch_bounds__(256) sweep_kernel(SweepArgs a) {
  using T = Tr<S>;
  using A = typename T::A;
  constexpr int V = T::V;
  constexpr bool kDev = sizeof(S) != 8;  // reduced modes store deviations
  extern __shared__ double sm[];
  __shared__ unsigned long long cnt_evals, cnt_solves, cnt_fb, cnt_bad;
  const int lpc = a.lpc, nd = a.nd, nbp = a.th.nbp, ng = a.th.ng;
  const int slot = threadIdx.x / lpc, lane = threadIdx.x - slot * lpc;
  double* red = sm;                   // [blockDim.x][3]
  double* cst = sm + 3 * blockDim.x;  // [cells per CTA][8] solve state
  const S* __restrict__ In = reinterpret_cast<const S*>(a.In);
  const S* __restrict__ Ik = reinterpret_cast<const S*>(a.Ik);
  S* __restrict__ Io = reinterpret_cast<S*>(a.Iout);
  const A* __restrict__ coef = reinterpret_cast<const A*>(a.coef);
  const long long row = (long long)nd * nbp;
  const int b0 = V * lane;
  if (threadIdx.x == 0) { cnt_evals = 0; cnt_solves = 0; cnt_fb = 0; cnt_bad = 0; }

  for (int item = blockIdx.x; item < a.nitems; item += gridDim.x) {
    const WorkItem wi = a.items[item];
    const DevGeom g = a.geoms[wi.geom];
    const bool active = slot < wi.cell_count;
    const int lc = wi.cell_begin + (active ? slot : 0);
    const int ci = lc % g.nx, cj = (lc / g.nx) % g.ny, ck = lc / (g.nx * g.ny);
    const long long P = g.cell0 + lc;
    double G[V];
#pragma unroll
    for (int v = 0; v < V; ++v) G[v] = 0.0;

    if (active) {
      A src[V];  // I0 of the cell (deviation in the reduced modes)
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const double i0 = a.I0cell[P * nbp + b0 + v];
        src[v] = kDev ? (A)(i0 - a.I0ref[b0 + v]) : (A)i0;
      }
      A hi[V], lo[V];  // compensated float sums (reduced modes)
#pragma unroll
      for (int v = 0; v < V; ++v) { hi[v] = 0; lo[v] = 0; }
      const size_t plane = (size_t)nd * nbp;
      const A* __restrict__ cf = coef + (size_t)g.cls * 5 * plane + b0;
      const S* __restrict__ inrow = In + P * row + b0;
      S* __restrict__ outrow = Io + P * row + b0;
#pragma unroll 2
      for (int d = 0; d < nd; ++d) {
        const DirInfo di = a.dirs[d];
        const size_t co = (size_t)d * nbp;
        A An[V], Ax[V], Ay[V], As[V], vn[V], ux[V], uy[V], r[V];
        ldgv<A, V>(cf + co, An);
        ldgv<A, V>(cf + plane + co, Ax);
        ldgv<A, V>(cf + 2 * plane + co, Ay);
        ldgv<A, V>(cf + 4 * plane + co, As);
        T::ld_stream(inrow + co, vn);
        upwind<0, S>(Ik, a, g, di, P, ci, cj, ck, row, d, b0, ux);
        upwind<1, S>(Ik, a, g, di, P, ci, cj, ck, row, d, b0, uy);
#pragma unroll
        for (int v = 0; v < V; ++v) {
          r[v] = An[v] * vn[v];
          r[v] = fma(Ax[v], ux[v], r[v]);
          r[v] = fma(Ay[v], uy[v], r[v]);
        }
        if (DIM == 3) {
          A Az[V], uz[V];
          ldgv<A, V>(cf + 3 * plane + co, Az);
          upwind<2, S>(Ik, a, g, di, P, ci, cj, ck, row, d, b0, uz);
#pragma unroll
          for (int v = 0; v < V; ++v) r[v] = fma(Az[v], uz[v], r[v]);
        }
#pragma unroll
        for (int v = 0; v < V; ++v) r[v] = fma(As[v], src[v], r[v]);
        T::st(outrow + co, r);
        if constexpr (!kDev) {
          const double wd = __ldg(a.wdir + d);
#pragma unroll
          for (int v = 0; v < V; ++v) G[v] = fma(wd, (double)r[v], G[v]);
        } else {
          // the reduction sees the stored (rounded) value
          const float wd = __ldg(a.wdir32 + d);
#pragma unroll
          for (int v = 0; v < V; ++v) {
            float val = r[v];
            if constexpr (sizeof(S) == 2) val = __bfloat162float(__float2bfloat16_rn(val));
            const float p = wd * val;  // TwoSum of (hi + p)
            const float s = hi[v] + p;
            const float bb = s - hi[v];
            lo[v] += (hi[v] - (s - bb)) + (p - bb);
            hi[v] = s;
          }
        }
      }
      if constexpr (kDev) {
#pragma unroll
        for (int v = 0; v < V; ++v) G[v] = fma(a.Wtot, a.I0ref[b0 + v], (double)hi[v] + (double)lo[v]);
      }
    }

    // ---- per-cell reduction: E_L = sum_b G_b / v_b, E_p = sum_b beta_b G_b / v_b
    {
      double eL = 0.0, ep = 0.0;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const double e = G[v] * a.th.inv_v[b0 + v];
        eL += e;
        ep = fma(a.th.beta[b0 + v], e, ep);
      }
      red[3 * threadIdx.x + 0] = eL;
      red[3 * threadIdx.x + 1] = ep;
    }
    __syncthreads();
    if (lane == 0) {
      double EL = 0.0, Ep = 0.0;
      for (int l = 0; l < lpc; ++l) {
        EL += red[3 * (threadIdx.x + l) + 0];
        Ep += red[3 * (threadIdx.x + l) + 1];
      }
      double* s = cst + 8 * slot;
      s[0] = Ep;
      s[1] = active ? a.Teval[P] : 300.0;  // evaluation point of the cached model
      s[2] = kTmin;
      s[3] = kTmax;
      s[5] = 0.0;  // iterations
      s[6] = 0.0;  // accepted step from the evaluation point
      s[7] = 0.0;  // 1 when the accepted data come from a fresh exact evaluation
      int mode = M_DONE;
      if (active) {
        a.EL[P] = EL;
        if (!isfinite(EL) || !isfinite(Ep)) {
          atomicAdd(&cnt_bad, 1ULL);
        } else if (a.solve_tp) {
          mode = M_MODEL;
          atomicAdd(&cnt_solves, 1ULL);
        }
      }
      s[4] = (double)mode;
    }
    __syncthreads();

    // ---- T_p solve (lockstep over the CTA's cells) and I0 refresh.  Exact
    // evaluations go straight to the cached model J (with T_e), so J and T_e
    // always describe the same point and nothing is held in registers across
    // the barriers.
    if (a.solve_tp) {
      const int maxloop = a.maxit + 224;
      double* const Jf = a.J + (P * 3 + 0) * nbp + b0;
      double* const Jd1 = a.J + (P * 3 + 1) * nbp + b0;
      double* const Jd2 = a.J + (P * 3 + 2) * nbp + b0;
      for (int it = 0; it < maxloop; ++it) {
        double* s = cst + 8 * slot;
        const int mode = (int)s[4];
        const double Te = s[1];
        if (mode < M_ACCEPT) {
          double F = 0.0, F1 = 0.0, F2 = 0.0;
          const double rT = 1.0 / Te;
          for (int v = 0; v < V; ++v) {
            double f, d1, d2;
            if (mode == M_MODEL) {  // cached quadratic model at T_e
              f = Jf[v];
              d1 = Jd1[v];
              d2 = Jd2[v];
            } else {  // exact quadrature at T_e, which becomes the cached model
              band_I0_d2(a.th.node_c + (b0 + v) * ng, a.th.node_C + (b0 + v) * ng, ng, rT, f, d1, d2);
              Jf[v] = f;
              Jd1[v] = d1;
              Jd2[v] = d2;
            }
            const double ap = a.th.a_p[b0 + v];
            F = fma(ap, f, F);
            F1 = fma(ap, d1, F1);
            F2 = fma(ap, d2, F2);
          }
          red[3 * threadIdx.x + 0] = F;
          red[3 * threadIdx.x + 1] = F1;
          red[3 * threadIdx.x + 2] = F2;
        }
        __syncthreads();
        if (lane == 0 && mode < M_ACCEPT) {
          double F = -s[0], F1 = 0.0, F2 = 0.0;
          for (int l = 0; l < lpc; ++l) {
            F += red[3 * (threadIdx.x + l) + 0];
            F1 += red[3 * (threadIdx.x + l) + 1];
            F2 += red[3 * (threadIdx.x + l) + 2];
          }
          if (mode != M_MODEL) {
            a.Teval[P] = Te;
            atomicAdd(&cnt_evals, 1ULL);
          }
          int next = mode;
          if (mode == M_MODEL) {
            // root of F + F1 d + F2 d^2 / 2 nearest 0
            const double disc = F1 * F1 - 2.0 * F * F2;
            const double delta = (disc >= 0.0 && F1 > 0.0) ? -2.0 * F / (F1 + sqrt(disc)) : -F / F1;
            const double Tn = Te + delta;
            if (isfinite(Tn) && fabs(delta) <= a.trust_rel * Tn) {
              next = M_ACCEPT;
              s[6] = delta;
            } else {
              next = M_HALLEY;
              s[1] = (isfinite(Tn) && Tn >= kTmin && Tn <= kTmax) ? Tn : a.Tp[P];
            }
          } else if (mode == M_HALLEY) {
            s[5] += 1.0;
            bool bad = !(isfinite(F) && isfinite(F1) && F1 > 0.0);
            double Tn = Te, delta = 0.0;
            if (!bad) {
              const double newton = -F / F1;
              const double h = F * F2 / (2.0 * F1 * F1);
              delta = fabs(h) < 0.5 ? newton / (1.0 - h) : newton;
              Tn = Te + delta;
              bad = !(Tn >= kTmin && Tn <= kTmax) || s[5] > a.maxit;
            }
            if (bad) {
              next = M_BISECT;
              s[2] = kTmin;
              s[3] = kTmax;
              s[1] = 0.5 * (kTmin + kTmax);
              atomicAdd(&cnt_fb, 1ULL);
            } else if (fabs(delta) <= a.trust_rel * Tn) {
              next = M_ACCEPT;
              s[6] = delta;
            } else {
              s[1] = Tn;
            }
          } else if (mode == M_BISECT) {
            if (F < 0.0) s[2] = Te; else s[3] = Te;
            s[1] = 0.5 * (s[2] + s[3]);
            s[5] += 1.0;
            if (s[3] - s[2] <= 4e-16 * s[3] || s[5] >= a.maxit + 200) next = M_FINAL;
          } else {  // M_FINAL: exact data at the bisected temperature
            s[6] = 0.0;
            next = M_ACCEPT;
            if (Te <= kTmin * (1.0 + 1e-9) || Te >= kTmax * (1.0 - 1e-9)) atomicAdd(&cnt_bad, 1ULL);
          }
          s[4] = (double)next;
        }
        __syncthreads();
        const int m2 = (int)s[4];
        if (m2 == M_ACCEPT && mode < M_ACCEPT) {  // I0 refresh from the model at T_e
          const double dlt = s[6];
          const double hd2 = 0.5 * dlt * dlt;
          for (int v = 0; v < V; ++v) a.I0cell[P * nbp + b0 + v] = fma(Jd2[v], hd2, fma(Jd1[v], dlt, Jf[v]));
          if (lane == 0) a.Tp[P] = Te + dlt;
        }
        __syncthreads();
        if (lane == 0 && m2 == M_ACCEPT) s[4] = (double)M_DONE;
        const int pending = (lane == 0 && (int)s[4] < M_ACCEPT) ? 1 : 0;
        if (!__syncthreads_or(pending)) break;
      }
      if (lane == 0 && (int)cst[8 * slot + 4] < M_ACCEPT) atomicAdd(&cnt_bad, 1ULL);
    }
    __syncthreads();
  }
  __syncthreads();
  if (threadIdx.x == 0 && a.counters) {
    if (cnt_evals) atomicAdd(&a.counters->evals, cnt_evals);
    if (cnt_solves) atomicAdd(&a.counters->solves, cnt_solves);
    if (cnt_fb) atomicAdd(&a.counters->fallbacks, cnt_fb);
    if (cnt_bad) atomicAdd(&a.counters->nonfinite, cnt_bad);
  }
}

// ---------------------------------------------------------------------------
// Per-cell thermodynamic state at temperature T: I0cell, cached model J at T,
// T_e = T_p = T.  One CTA per cell (grid-stride); bands over threads.
__device__ void cell_state_at(double* I0cell, double* J, long long P, double T, ThermoTables th, double* row) {
  const double rT = 1.0 / T;
  for (int b = threadIdx.x; b < th.nbp; b += blockDim.x) {
    double f, d1, d2;
    band_I0_d2(th.node_c + b * th.ng, th.node_C + b * th.ng, th.ng, rT, f, d1, d2);
    row[b] = f;
    I0cell[P * th.nbp + b] = f;
    J[(P * 3 + 0) * th.nbp + b] = f;
    J[(P * 3 + 1) * th.nbp + b] = d1;
    J[(P * 3 + 2) * th.nbp + b] = d2;
  }
}

// Equilibrium initial state: I = I0_b(T_P) for every direction (stored as the
// deviation I0_b(T_P) - I0_b(T_ref) in the reduced modes).
template <typename S>
__global__ void init_cells_kernel(S* I, double* I0cell, double* J, double* Tp, double* Te, double* TL, double* EL,
                                  const double* Tcells, const double* I0ref, long long cell0, int ncells, int nd,
                                  ThermoTables th) {
  extern __shared__ double row[];  // [nbp]
  for (int c = blockIdx.x; c < ncells; c += gridDim.x) {
    const long long P = cell0 + c;
    const double T = Tcells[c];
    cell_state_at(I0cell, J, P, T, th, row);
    __syncthreads();
    const long long n = (long long)nd * th.nbp;
    for (long long e = threadIdx.x; e < n; e += blockDim.x) {
      const int b = (int)(e % th.nbp);
      const double v = sizeof(S) == 8 ? row[b] : row[b] - I0ref[b];
      if constexpr (sizeof(S) == 2) I[P * n + e] = __double2bfloat16(v);
      else I[P * n + e] = (S)v;
    }
    if (threadIdx.x == 0) {
      double e = 0.0;
      for (int b = 0; b < th.nbp; ++b) e = fma(th.a_L[b], row[b], e);
      Tp[P] = T;
      Te[P] = T;
      TL[P] = T;
      EL[P] = e;
    }
    __syncthreads();
  }
}

// Thermodynamic state from T_p after a state restore: I0cell, J, T_e.
__global__ void state_from_Tp_kernel(double* I0cell, double* J, const double* Tp, double* Te, long long ncells,
                                     ThermoTables th) {
  extern __shared__ double row[];
  for (long long P = blockIdx.x; P < ncells; P += gridDim.x) {
    cell_state_at(I0cell, J, P, Tp[P], th, row);
    if (threadIdx.x == 0) Te[P] = Tp[P];
    __syncthreads();
  }
}

// Wall ghost intensities (FP64): one thread per (face, band).
__global__ void wall_I0_kernel(double* I0wall, const double* Tf, long long nfaces, ThermoTables th) {
  const long long n = nfaces * th.nbp;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const long long f = e / th.nbp;
    const int b = (int)(e - f * th.nbp);
    I0wall[e] = band_I0(th.node_c + b * th.ng, th.node_C + b * th.ng, th.ng, 1.0 / Tf[f]);
  }
}

// Deviation ghosts for the reduced modes: I0wall - I0ref as FP32.
__global__ void wall_dev_kernel(float* out, const double* I0wall, const double* I0ref, long long n, int nbp) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    out[e] = (float)(I0wall[e] - I0ref[e % nbp]);
}

// Lattice temperature: sum_b a_L,b I0_b(T) = E_L per cell, Newton from the
// guess with bisection fallback.  One thread per cell (evaluated on request).
__global__ void solve_TL_kernel(double* TL, const double* EL, const double* Tguess, long long ncells, ThermoTables th,
                                double rtol, int maxit, DevCounters* counters) {
  for (long long P = blockIdx.x * (long long)blockDim.x + threadIdx.x; P < ncells;
       P += (long long)gridDim.x * blockDim.x) {
    const double E = EL[P];
    double T = Tguess[P];
    bool ok = false;
    if (isfinite(E) && T >= kTmin && T <= kTmax) {
      for (int it = 0; it < maxit; ++it) {
        const double rT = 1.0 / T;
        double F = -E, dF = 0.0;
        for (int b = 0; b < th.nb; ++b) {
          double f, d1, d2;
          band_I0_d2(th.node_c + b * th.ng, th.node_C + b * th.ng, th.ng, rT, f, d1, d2);
          F = fma(th.a_L[b], f, F);
          dF = fma(th.a_L[b], d1, dF);
        }
        const double dT = -F / dF;
        T += dT;
        if (!(T >= kTmin && T <= kTmax)) break;
        if (fabs(dT) <= rtol * T) { ok = true; break; }
      }
    }
    if (!ok && isfinite(E)) {
      if (counters) atomicAdd(&counters->fallbacks, 1ULL);
      double lo = kTmin, hi = kTmax;
      for (int it = 0; it < 200 && hi - lo > 4e-16 * hi; ++it) {
        const double mid = 0.5 * (lo + hi), rT = 1.0 / mid;
        double F = -E;
        for (int b = 0; b < th.nb; ++b) F = fma(th.a_L[b], band_I0(th.node_c + b * th.ng, th.node_C + b * th.ng, th.ng, rT), F);
        if (F < 0.0) lo = mid; else hi = mid;
      }
      T = 0.5 * (lo + hi);
    }
    if (!isfinite(E) && counters) atomicAdd(&counters->nonfinite, 1ULL);
    TL[P] = isfinite(E) ? T : E;
  }
}

// Deterministic block sum of one value per thread (blockDim.x a power of two <= 1024).
__device__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// Full intensity value (FP64) of element e of a padded row set.
template <typename S>
__device__ __forceinline__ double full_I(const S* I, long long e, int b, const double* I0ref) {
  if constexpr (sizeof(S) == 8) return (double)I[e];
  else return I0ref[b] + Tr<S>::to_double(I[e]);
}

// Cell heat flux q(P) = sum_b sum_d S_d I_{d,b}: one CTA per cell.
template <typename S>
__global__ void flux_cells_kernel(const S* I, const double* I0ref, double* q, const double* Sd, long long cell0,
                                  int ncells, int nd, int nbp, int dim) {
  extern __shared__ double sh[];
  for (int c = blockIdx.x; c < ncells; c += gridDim.x) {
    const long long P = cell0 + c;
    const long long base = P * (long long)nd * nbp;
    double acc[3] = {0.0, 0.0, 0.0};
    for (long long e = threadIdx.x; e < (long long)nd * nbp; e += blockDim.x) {
      const int d = (int)(e / nbp);
      const int b = (int)(e - (long long)d * nbp);
      const double v = full_I(I, base + e, b, I0ref);
      acc[0] = fma(Sd[3 * d + 0], v, acc[0]);
      acc[1] = fma(Sd[3 * d + 1], v, acc[1]);
      acc[2] = fma(Sd[3 * d + 2], v, acc[2]);
    }
    for (int ax = 0; ax < dim; ++ax) {
      const double t = block_sum(acc[ax], sh);
      if (threadIdx.x == 0) q[(long long)c * dim + ax] = t;
    }
  }
}

// Net outgoing flux through each face of one wall: one CTA per face.
template <typename S>
__global__ void flux_faces_kernel(const S* I, const double* I0ref, const double* I0wall, const DevGeom* geoms,
                                  int geom, int side, const DirInfo* dirs, const double* Sd, int nd, int nbp,
                                  double* face_out, int nfaces) {
  extern __shared__ double sh[];
  const DevGeom g = geoms[geom];
  const int ax = side / 2;
  const double nsign = (side & 1) ? 1.0 : -1.0;
  for (int f = blockIdx.x; f < nfaces; f += gridDim.x) {
    int i, j, k;
    if (side < 2) { j = f % g.ny; k = f / g.ny; i = (side & 1) ? g.nx - 1 : 0; }
    else if (side < 4) { i = f % g.nx; k = f / g.nx; j = (side & 1) ? g.ny - 1 : 0; }
    else { i = f % g.nx; j = f / g.nx; k = (side & 1) ? g.nz - 1 : 0; }
    const long long P = g.cell0 + i + (long long)g.nx * (j + (long long)g.ny * k);
    const long long base = P * (long long)nd * nbp;
    double acc = 0.0;
    for (long long e = threadIdx.x; e < (long long)nd * nbp; e += blockDim.x) {
      const int d = (int)(e / nbp);
      const int b = (int)(e - (long long)d * nbp);
      const double sn = Sd[3 * d + ax] * nsign;
      double v;
      if (sn > 0.0) v = full_I(I, base + e, b, I0ref);
      else if (g.bc[side] == 0) v = I0wall[(g.face0[side] + f) * nbp + b];
      else {
        const int r = ax == 0 ? dirs[d].rx : (ax == 1 ? dirs[d].ry : dirs[d].rz);
        v = full_I(I, base + (long long)r * nbp + b, b, I0ref);
      }
      acc = fma(sn, v, acc);
    }
    const double t = block_sum(acc, sh);
    if (threadIdx.x == 0) face_out[f] = t;
  }
}

__global__ void mean_kernel(const double* v, int n, double* out) {
  extern __shared__ double sh[];
  double acc = 0.0;
  for (int e = threadIdx.x; e < n; e += blockDim.x) acc += v[e];
  const double t = block_sum(acc, sh);
  if (threadIdx.x == 0) *out = t / (double)n;
}

// FP64 [cell][d][nb] <-> padded storage rows [cell][d][nbp] (deviation in the reduced modes).
template <typename S>
__global__ void pack_kernel(const double* src, double* dst_out, const S* Isrc, S* Idst, const double* I0ref,
                            long long ncells, int nd, int nb, int nbp, int to_padded) {
  const long long n = ncells * nd * (long long)nbp;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const long long cd = e / nbp;
    const int b = (int)(e - cd * nbp);
    if (to_padded) {
      const double v = b < nb ? (sizeof(S) == 8 ? src[cd * nb + b] : src[cd * nb + b] - I0ref[b]) : 0.0;
      if constexpr (sizeof(S) == 2) Idst[e] = __double2bfloat16(v);
      else Idst[e] = (S)v;
    } else if (b < nb) {
      dst_out[cd * nb + b] = full_I(Isrc, e, b, I0ref);
    }
  }
}

// E_L of every cell from its intensity row (used after a state restore).
template <typename S>
__global__ void energy_L_kernel(const S* I, const double* I0ref, double* EL, const double* wdir, long long ncells,
                                int nd, ThermoTables th) {
  extern __shared__ double sh[];
  for (long long P = blockIdx.x; P < ncells; P += gridDim.x) {
    const long long base = P * (long long)nd * th.nbp;
    double acc = 0.0;
    for (int b = threadIdx.x; b < th.nbp; b += blockDim.x) {
      double G = 0.0;
      for (int d = 0; d < nd; ++d) G = fma(wdir[d], full_I(I, base + (long long)d * th.nbp + b, b, I0ref), G);
      acc = fma(G, th.inv_v[b], acc);
    }
    const double t = block_sum(acc, sh);
    if (threadIdx.x == 0) EL[P] = t;
  }
}

inline int grid_for(long long n, int threads) {
  long long g = (n + threads - 1) / threads;
  if (g > 152LL * 64) g = 152LL * 64;
  return (int)(g < 1 ? 1 : g);
}

inline int cell_grid(long long ncells) { return (int)(ncells < 152 * 16 ? (ncells < 1 ? 1 : ncells) : 152 * 16); }

template <typename S>
cudaError_t sweep_dispatch(const SweepArgs& a, int dim, int threads, int grid, cudaStream_t s) {
  const int cpb = threads / a.lpc;
  const size_t smem = (3 * (size_t)threads + 8 * (size_t)cpb) * sizeof(double);
  if (dim == 3) sweep_kernel<3, S><<<grid, threads, smem, s>>>(a);
  else sweep_kernel<2, S><<<grid, threads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

int values_per_lane(int precision) { return precision == 0 ? 2 : 4; }

cudaError_t launch_sweep(int precision, const SweepArgs& a, int dim, int threads, int grid, cudaStream_t s) {
  if (precision == 0) return sweep_dispatch<double>(a, dim, threads, grid, s);
  if (precision == 1) return sweep_dispatch<float>(a, dim, threads, grid, s);
  return sweep_dispatch<__nv_bfloat16>(a, dim, threads, grid, s);
}

cudaError_t launch_init_cells(int precision, void* I, double* I0cell, double* J, double* Tp, double* Te, double* TL,
                              double* EL, const double* Tcells, const double* I0ref, long long cell0, int ncells, int nd,
                              ThermoTables th, cudaStream_t s) {
  const int grid = cell_grid(ncells);
  const size_t sm = th.nbp * sizeof(double);
  if (precision == 0)
    init_cells_kernel<double><<<grid, 256, sm, s>>>((double*)I, I0cell, J, Tp, Te, TL, EL, Tcells, I0ref, cell0, ncells, nd, th);
  else if (precision == 1)
    init_cells_kernel<float><<<grid, 256, sm, s>>>((float*)I, I0cell, J, Tp, Te, TL, EL, Tcells, I0ref, cell0, ncells, nd, th);
  else
    init_cells_kernel<__nv_bfloat16><<<grid, 256, sm, s>>>((__nv_bfloat16*)I, I0cell, J, Tp, Te, TL, EL, Tcells, I0ref,
                                                           cell0, ncells, nd, th);
  return cudaGetLastError();
}

cudaError_t launch_state_from_Tp(double* I0cell, double* J, const double* Tp, double* Te, long long ncells,
                                 ThermoTables th, cudaStream_t s) {
  state_from_Tp_kernel<<<cell_grid(ncells), 64, th.nbp * sizeof(double), s>>>(I0cell, J, Tp, Te, ncells, th);
  return cudaGetLastError();
}

cudaError_t launch_wall_I0(double* I0wall, const double* Tfaces, long long nfaces, ThermoTables th, cudaStream_t s) {
  wall_I0_kernel<<<grid_for(nfaces * th.nbp, 256), 256, 0, s>>>(I0wall, Tfaces, nfaces, th);
  return cudaGetLastError();
}

cudaError_t launch_wall_dev(float* out, const double* I0wall, const double* I0ref, long long nfaces, int nbp,
                            cudaStream_t s) {
  wall_dev_kernel<<<grid_for(nfaces * nbp, 256), 256, 0, s>>>(out, I0wall, I0ref, nfaces * nbp, nbp);
  return cudaGetLastError();
}

cudaError_t launch_solve_TL(double* TL, const double* EL, const double* Tguess, long long ncells, ThermoTables th,
                            double rtol, int maxit, DevCounters* counters, cudaStream_t s) {
  solve_TL_kernel<<<grid_for(ncells, 128), 128, 0, s>>>(TL, EL, Tguess, ncells, th, rtol, maxit, counters);
  return cudaGetLastError();
}

cudaError_t launch_flux_cells(int precision, const void* I, const double* I0ref, double* q, const double* S,
                              long long cell0, int ncells, int nd, int nbp, int dim, cudaStream_t s) {
  const int grid = cell_grid(ncells);
  const size_t sm = 256 * sizeof(double);
  if (precision == 0) flux_cells_kernel<double><<<grid, 256, sm, s>>>((const double*)I, I0ref, q, S, cell0, ncells, nd, nbp, dim);
  else if (precision == 1) flux_cells_kernel<float><<<grid, 256, sm, s>>>((const float*)I, I0ref, q, S, cell0, ncells, nd, nbp, dim);
  else flux_cells_kernel<__nv_bfloat16><<<grid, 256, sm, s>>>((const __nv_bfloat16*)I, I0ref, q, S, cell0, ncells, nd, nbp, dim);
  return cudaGetLastError();
}

cudaError_t launch_flux_faces(int precision, const void* I, const double* I0ref, const double* I0wall,
                              const DevGeom* geoms, int geom, int side, const DirInfo* dirs, const double* S, int nd,
                              int nbp, double* face_out, int nfaces, cudaStream_t s) {
  const int grid = cell_grid(nfaces);
  const size_t sm = 256 * sizeof(double);
  if (precision == 0)
    flux_faces_kernel<double><<<grid, 256, sm, s>>>((const double*)I, I0ref, I0wall, geoms, geom, side, dirs, S, nd, nbp, face_out, nfaces);
  else if (precision == 1)
    flux_faces_kernel<float><<<grid, 256, sm, s>>>((const float*)I, I0ref, I0wall, geoms, geom, side, dirs, S, nd, nbp, face_out, nfaces);
  else
    flux_faces_kernel<__nv_bfloat16><<<grid, 256, sm, s>>>((const __nv_bfloat16*)I, I0ref, I0wall, geoms, geom, side, dirs, S,
                                                           nd, nbp, face_out, nfaces);
  return cudaGetLastError();
}

cudaError_t launch_mean(const double* v, int n, double* out, cudaStream_t s) {
  mean_kernel<<<1, 256, 256 * sizeof(double), s>>>(v, n, out);
  return cudaGetLastError();
}

cudaError_t launch_pack(int precision, const double* src, double* dst_out, const void* Isrc, void* Idst,
                        const double* I0ref, long long ncells, int nd, int nb, int nbp, int to_padded, cudaStream_t s) {
  const int grid = grid_for(ncells * nd * (long long)nbp, 256);
  if (precision == 0)
    pack_kernel<double><<<grid, 256, 0, s>>>(src, dst_out, (const double*)Isrc, (double*)Idst, I0ref, ncells, nd, nb, nbp, to_padded);
  else if (precision == 1)
    pack_kernel<float><<<grid, 256, 0, s>>>(src, dst_out, (const float*)Isrc, (float*)Idst, I0ref, ncells, nd, nb, nbp, to_padded);
  else
    pack_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(src, dst_out, (const __nv_bfloat16*)Isrc, (__nv_bfloat16*)Idst, I0ref,
                                                    ncells, nd, nb, nbp, to_padded);
  return cudaGetLastError();
}

cudaError_t launch_energy_L(int precision, const void* I, const double* I0ref, double* EL, const double* wdir,
                            long long ncells, int nd, ThermoTables th, cudaStream_t s) {
  const int grid = cell_grid(ncells);
  const size_t sm = 64 * sizeof(double);
  if (precision == 0) energy_L_kernel<double><<<grid, 64, sm, s>>>((const double*)I, I0ref, EL, wdir, ncells, nd, th);
  else if (precision == 1) energy_L_kernel<float><<<grid, 64, sm, s>>>((const float*)I, I0ref, EL, wdir, ncells, nd, th);
  else energy_L_kernel<__nv_bfloat16><<<grid, 64, sm, s>>>((const __nv_bfloat16*)I, I0ref, EL, wdir, ncells, nd, th);
  return cudaGetLastError();
}

}  // namespace bte

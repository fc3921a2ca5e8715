// bte_kernels.cu -- CUDA kernels of the phonon BTE hot path (sm_103a).
//
// K1 sweep_fp64: one launch per inner iteration.  A CTA owns a run of cells of
//   one geometry; each cell is served by `lpc` lanes, lane l holding bands
//   2l, 2l+1 as one double2.  Each lane walks every direction d (Sec. 3.1,
//   Eq. 5 discretised):
//     implicit  I^{k+1} = A_n I^n + A_x I_up,x^k + A_y I_up,y^k (+ A_z I_up,z^k) + A_s I0^k
//     explicit  same form with forward-Euler coefficients and I^k = I^n
//   where the upwind value is the neighbour cell on the side S_d comes from,
//   or the Eq. 6 ghost at a wall (I0 of the wall face, or the cell's own value
//   in the mirrored direction).  The same lane accumulates
//   G_b = sum_d w_d I^{k+1}_{d,b} in registers, so the per-cell reduction of
//   the temperature update costs one FMA per update and no shuffles.  The
//   epilogue reduces the cell's lanes to E_L, E_p, solves the T_p equation by
//   warm-started Halley steps on the FP64 band quadrature and refreshes I0.
// The HBM stream per update is I^n read, I^{k+1} written and I^k read once
// (neighbour rows are re-read from L2 by the adjacent cells processed at the
// same time).
#include "bte_internal.h"

namespace bte {

namespace {

enum SolveMode { M_HALLEY = 0, M_BISECT = 1, M_FINAL = 2, M_ACCEPT = 3, M_DONE = 4 };

// I0_b(T) = sum_i C_i / expm1(c_i / T)  (Gauss-Legendre on the band).
__device__ __forceinline__ double band_I0(const double* __restrict__ c, const double* __restrict__ C, int ng,
                                          double rT) {
  double s = 0.0;
  for (int i = 0; i < ng; ++i) s = fma(C[i], 1.0 / expm1(c[i] * rT), s);
  return s;
}

// I0_b, dI0_b/dT and d2I0_b/dT2 from the same nodes.  With n = 1/(e^x - 1),
// x = c/T:  dn/dT = n(1+n) x/T,  d2n/dT2 = n(1+n) (x/T^2) ((1+2n) x - 2).
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

__device__ __forceinline__ double2 ldg2(const double* p) { return __ldg(reinterpret_cast<const double2*>(p)); }

__device__ __forceinline__ long long face_of(const DevGeom& g, int side, int i, int j, int k) {
  if (side < 2) return j + (long long)g.ny * k;
  if (side < 4) return i + (long long)g.nx * k;
  return i + (long long)g.nx * j;
}

// Upwind value along axis AX for one lane of cell P in direction d.  Wall
// data are read with compile-time side indices so DevGeom stays in registers.
template <int AX>
__device__ __forceinline__ double2 upwind(const double2* __restrict__ Ik, const double* __restrict__ I0wall,
                                          const DevGeom& g, const DirInfo& di, long long P, int ci, int cj, int ck,
                                          long long rowv, int d, int lpc, int lane) {
  const int c = AX == 0 ? ci : (AX == 1 ? cj : ck);
  const int n = AX == 0 ? g.nx : (AX == 1 ? g.ny : g.nz);
  const long long stride = AX == 0 ? 1 : (AX == 1 ? (long long)g.nx : (long long)g.nx * g.ny);
  const bool from_low = (di.up >> AX) & 1;
  if (from_low ? c > 0 : c < n - 1) return Ik[(P + (from_low ? -stride : stride)) * rowv + (long long)d * lpc + lane];
  const int bc = from_low ? g.bc[2 * AX] : g.bc[2 * AX + 1];
  if (bc == 0) {  // isothermal wall: I0_b of the face
    const long long f0 = from_low ? g.face0[2 * AX] : g.face0[2 * AX + 1];
    const long long f = f0 + (AX == 0 ? cj + (long long)g.ny * ck : (AX == 1 ? ci + (long long)g.nx * ck : ci + (long long)g.nx * cj));
    return ldg2(I0wall + f * (2LL * lpc) + 2 * lane);
  }
  const int r = AX == 0 ? di.rx : (AX == 1 ? di.ry : di.rz);  // symmetry wall: mirrored direction
  return Ik[P * rowv + (long long)r * lpc + lane];
}

template <int DIM>
__global__ void __launch_bounds__(256) sweep_fp64_kernel(SweepArgs a) {
  extern __shared__ double sm[];
  __shared__ unsigned long long cnt_evals, cnt_solves, cnt_fb, cnt_bad;
  const int lpc = a.lpc, nd = a.nd, nbp = a.th.nbp, ng = a.th.ng;
  const int slot = threadIdx.x / lpc, lane = threadIdx.x - slot * lpc;
  double* red = sm;                     // [blockDim.x][3]
  double* cst = sm + 3 * blockDim.x;    // [cpb][8] per-cell solve state
  const double2* __restrict__ In = reinterpret_cast<const double2*>(a.In);
  const double2* __restrict__ Ik = reinterpret_cast<const double2*>(a.Ik);
  double2* __restrict__ Io = reinterpret_cast<double2*>(a.Iout);
  const long long rowv = (long long)nd * lpc;
  const int b0 = 2 * lane;
  if (threadIdx.x == 0) { cnt_evals = 0; cnt_solves = 0; cnt_fb = 0; cnt_bad = 0; }

  for (int item = blockIdx.x; item < a.nitems; item += gridDim.x) {
    const WorkItem wi = a.items[item];
    const DevGeom g = a.geoms[wi.geom];
    const bool active = slot < wi.cell_count;
    const int lc = wi.cell_begin + (active ? slot : 0);
    const int ci = lc % g.nx, cj = (lc / g.nx) % g.ny, ck = lc / (g.nx * g.ny);
    const long long P = g.cell0 + lc;
    double G0 = 0.0, G1 = 0.0;

    if (active) {
      const double2 i0 = *reinterpret_cast<const double2*>(a.I0cell + P * nbp + b0);
      const double* __restrict__ cf = a.coef + (size_t)g.cls * 5 * nd * nbp + b0;
      const size_t plane = (size_t)nd * nbp;
      const double2* __restrict__ inrow = In + P * rowv + lane;
      double2* __restrict__ outrow = Io + P * rowv + lane;
#pragma unroll 2
      for (int d = 0; d < nd; ++d) {
        const DirInfo di = a.dirs[d];
        const double wd = __ldg(a.wdir + d);
        const size_t co = (size_t)d * nbp;
        const double2 An = ldg2(cf + co);
        const double2 Ax = ldg2(cf + plane + co);
        const double2 Ay = ldg2(cf + 2 * plane + co);
        const double2 As = ldg2(cf + 4 * plane + co);
        const double2 vn = inrow[(long long)d * lpc];
        const double2 ux = upwind<0>(Ik, a.I0wall, g, di, P, ci, cj, ck, rowv, d, lpc, lane);
        const double2 uy = upwind<1>(Ik, a.I0wall, g, di, P, ci, cj, ck, rowv, d, lpc, lane);
        double2 r;
        r.x = An.x * vn.x;
        r.y = An.y * vn.y;
        r.x = fma(Ax.x, ux.x, r.x);
        r.y = fma(Ax.y, ux.y, r.y);
        r.x = fma(Ay.x, uy.x, r.x);
        r.y = fma(Ay.y, uy.y, r.y);
        if (DIM == 3) {
          const double2 Az = ldg2(cf + 3 * plane + co);
          const double2 uz = upwind<2>(Ik, a.I0wall, g, di, P, ci, cj, ck, rowv, d, lpc, lane);
          r.x = fma(Az.x, uz.x, r.x);
          r.y = fma(Az.y, uz.y, r.y);
        }
        r.x = fma(As.x, i0.x, r.x);
        r.y = fma(As.y, i0.y, r.y);
        outrow[(long long)d * lpc] = r;
        G0 = fma(wd, r.x, G0);
        G1 = fma(wd, r.y, G1);
      }
    }

    // ---- per-cell reduction: E_L = sum_b G_b / v_b, E_p = sum_b beta_b G_b / v_b
    {
      const double iv0 = a.th.inv_v[b0], iv1 = a.th.inv_v[b0 + 1];
      const double e0 = G0 * iv0, e1 = G1 * iv1;
      red[3 * threadIdx.x + 0] = e0 + e1;
      red[3 * threadIdx.x + 1] = fma(a.th.beta[b0], e0, a.th.beta[b0 + 1] * e1);
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
      s[1] = active ? a.Tp[P] : 300.0;  // warm start
      s[2] = kTmin;
      s[3] = kTmax;
      s[5] = 0.0;  // iterations
      s[6] = 0.0;  // accepted step
      s[7] = 0.0;  // evaluations
      int mode = M_DONE;
      if (active) {
        a.EL[P] = EL;
        if (!isfinite(EL) || !isfinite(Ep)) {
          atomicAdd(&cnt_bad, 1ULL);
        } else if (a.solve_tp) {
          mode = M_HALLEY;
          atomicAdd(&cnt_solves, 1ULL);
        }
      }
      s[4] = (double)mode;
    }
    __syncthreads();

    // ---- T_p solve (lockstep over the CTA's cells) and I0 refresh
    if (a.solve_tp) {
      const int maxloop = a.maxit + 220;
      for (int it = 0; it < maxloop; ++it) {
        double* s = cst + 8 * slot;
        const int mode = (int)s[4];
        const double T = s[1];
        double f0 = 0.0, f1 = 0.0, p0 = 0.0, p1 = 0.0, q0 = 0.0, q1 = 0.0;
        if (mode < M_ACCEPT) {
          const double rT = 1.0 / T;
          band_I0_d2(a.th.node_c + b0 * ng, a.th.node_C + b0 * ng, ng, rT, f0, p0, q0);
          band_I0_d2(a.th.node_c + (b0 + 1) * ng, a.th.node_C + (b0 + 1) * ng, ng, rT, f1, p1, q1);
          const double ap0 = a.th.a_p[b0], ap1 = a.th.a_p[b0 + 1];
          red[3 * threadIdx.x + 0] = fma(ap0, f0, ap1 * f1);
          red[3 * threadIdx.x + 1] = fma(ap0, p0, ap1 * p1);
          red[3 * threadIdx.x + 2] = fma(ap0, q0, ap1 * q1);
        }
        __syncthreads();
        if (lane == 0 && mode < M_ACCEPT) {
          double F = -s[0], dF = 0.0, d2F = 0.0;
          for (int l = 0; l < lpc; ++l) {
            F += red[3 * (threadIdx.x + l) + 0];
            dF += red[3 * (threadIdx.x + l) + 1];
            d2F += red[3 * (threadIdx.x + l) + 2];
          }
          s[7] += 1.0;
          int next = mode;
          if (mode == M_HALLEY) {
            bool bad = !(isfinite(F) && isfinite(dF) && dF > 0.0);
            double Tn = T, delta = 0.0;
            if (!bad) {
              const double newton = -F / dF;
              const double h = F * d2F / (2.0 * dF * dF);
              delta = fabs(h) < 0.5 ? newton / (1.0 - h) : newton;
              Tn = T + delta;
              bad = !(Tn >= kTmin && Tn <= kTmax) || s[5] >= a.maxit;
            }
            if (bad) {
              next = M_BISECT;
              s[2] = kTmin;
              s[3] = kTmax;
              s[1] = 0.5 * (kTmin + kTmax);
              atomicAdd(&cnt_fb, 1ULL);
            } else if (fabs(delta) <= a.accept_rel * Tn) {
              next = M_ACCEPT;  // Taylor refresh of I0 from this evaluation point
              s[6] = delta;
            } else {
              s[1] = Tn;
              s[5] += 1.0;
            }
          } else if (mode == M_BISECT) {
            if (F < 0.0) s[2] = T; else s[3] = T;
            s[1] = 0.5 * (s[2] + s[3]);
            s[5] += 1.0;
            if (s[3] - s[2] <= 4e-16 * s[3] || s[5] >= a.maxit + 200) next = M_FINAL;
          } else {  // M_FINAL: exact I0 at the bisected temperature
            s[6] = 0.0;
            next = M_ACCEPT;
            if (T <= kTmin * (1.0 + 1e-9) || T >= kTmax * (1.0 - 1e-9)) atomicAdd(&cnt_bad, 1ULL);
          }
          s[4] = (double)next;
        }
        __syncthreads();
        const int m2 = (int)s[4];
        if (m2 == M_ACCEPT && mode < M_ACCEPT) {
          const double dlt = s[6];
          const double hd2 = 0.5 * dlt * dlt;
          double2 nI0;
          nI0.x = fma(q0, hd2, fma(p0, dlt, f0));
          nI0.y = fma(q1, hd2, fma(p1, dlt, f1));
          *reinterpret_cast<double2*>(a.I0cell + P * nbp + b0) = nI0;
          if (lane == 0) {
            a.Tp[P] = s[1] + dlt;
            atomicAdd(&cnt_evals, (unsigned long long)s[7]);
          }
        }
        __syncthreads();
        if (lane == 0 && m2 == M_ACCEPT) s[4] = (double)M_DONE;
        const int pending = (lane == 0 && (int)s[4] < M_ACCEPT) ? 1 : 0;
        if (!__syncthreads_or(pending)) break;
      }
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
// Equilibrium initial state: one CTA per cell (grid-stride).
__global__ void init_cells_kernel(double* I, double* I0cell, double* Tp, double* TL, double* EL, const double* Tcells,
                                  long long cell0, int ncells, int nd, ThermoTables th) {
  extern __shared__ double row[];  // [nbp]
  for (int c = blockIdx.x; c < ncells; c += gridDim.x) {
    const long long P = cell0 + c;
    const double T = Tcells[c];
    const double rT = 1.0 / T;
    for (int b = threadIdx.x; b < th.nbp; b += blockDim.x) {
      const double v = band_I0(th.node_c + b * th.ng, th.node_C + b * th.ng, th.ng, rT);
      row[b] = v;
      I0cell[P * th.nbp + b] = v;
    }
    __syncthreads();
    const long long n = (long long)nd * th.nbp;
    for (long long e = threadIdx.x; e < n; e += blockDim.x) I[P * n + e] = row[e % th.nbp];
    if (threadIdx.x == 0) {
      double e = 0.0;
      for (int b = 0; b < th.nbp; ++b) e = fma(th.a_L[b], row[b], e);
      Tp[P] = T;
      TL[P] = T;
      EL[P] = e;
    }
    __syncthreads();
  }
}

// Wall ghost intensities: one thread per (face, band).
__global__ void wall_I0_kernel(double* I0wall, const double* Tf, long long nfaces, ThermoTables th) {
  const long long n = nfaces * th.nbp;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const long long f = e / th.nbp;
    const int b = (int)(e - f * th.nbp);
    I0wall[e] = band_I0(th.node_c + b * th.ng, th.node_C + b * th.ng, th.ng, 1.0 / Tf[f]);
  }
}

// I0 of every cell at its T_p: one thread per (cell, band).
__global__ void I0_from_T_kernel(double* I0cell, const double* Tp, long long ncells, ThermoTables th) {
  const long long n = ncells * th.nbp;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const long long P = e / th.nbp;
    const int b = (int)(e - P * th.nbp);
    I0cell[e] = band_I0(th.node_c + b * th.ng, th.node_C + b * th.ng, th.ng, 1.0 / Tp[P]);
  }
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

// Cell heat flux q(P) = sum_b sum_d S_d I_{d,b}: one CTA per cell.
__global__ void flux_cells_kernel(const double* I, double* q, const double* S, long long cell0, int ncells, int nd,
                                  int nbp, int dim) {
  extern __shared__ double sh[];
  for (int c = blockIdx.x; c < ncells; c += gridDim.x) {
    const long long P = cell0 + c;
    const double* row = I + P * (long long)nd * nbp;
    double acc[3] = {0.0, 0.0, 0.0};
    for (long long e = threadIdx.x; e < (long long)nd * nbp; e += blockDim.x) {
      const int d = (int)(e / nbp);
      const double v = row[e];
      acc[0] = fma(S[3 * d + 0], v, acc[0]);
      acc[1] = fma(S[3 * d + 1], v, acc[1]);
      acc[2] = fma(S[3 * d + 2], v, acc[2]);
    }
    for (int ax = 0; ax < dim; ++ax) {
      const double t = block_sum(acc[ax], sh);
      if (threadIdx.x == 0) q[(long long)c * dim + ax] = t;
    }
  }
}

// Net outgoing flux through each face of one wall: one CTA per face.
__global__ void flux_faces_kernel(const double* I, const double* I0wall, const DevGeom* geoms, int geom, int side,
                                  const DirInfo* dirs, const double* S, int nd, int nbp, double* face_out, int nfaces) {
  extern __shared__ double sh[];
  const DevGeom g = geoms[geom];
  const int ax = side / 2;
  const double nsign = (side & 1) ? 1.0 : -1.0;
  for (int f = blockIdx.x; f < nfaces; f += gridDim.x) {
    // cell on the wall owning face f
    int i, j, k;
    if (side < 2) { j = f % g.ny; k = f / g.ny; i = (side & 1) ? g.nx - 1 : 0; }
    else if (side < 4) { i = f % g.nx; k = f / g.nx; j = (side & 1) ? g.ny - 1 : 0; }
    else { i = f % g.nx; j = f / g.nx; k = (side & 1) ? g.nz - 1 : 0; }
    const long long P = g.cell0 + i + (long long)g.nx * (j + (long long)g.ny * k);
    const double* row = I + P * (long long)nd * nbp;
    double acc = 0.0;
    for (long long e = threadIdx.x; e < (long long)nd * nbp; e += blockDim.x) {
      const int d = (int)(e / nbp);
      const int b = (int)(e - (long long)d * nbp);
      const double sn = S[3 * d + ax] * nsign;
      double v;
      if (sn > 0.0) v = row[e];
      else if (g.bc[side] == 0) v = I0wall[(g.face0[side] + f) * nbp + b];
      else {
        const int r = ax == 0 ? dirs[d].rx : (ax == 1 ? dirs[d].ry : dirs[d].rz);
        v = row[(long long)r * nbp + b];
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

// FP64 [cell][d][nb] <-> padded [cell][d][nbp].
__global__ void pack_kernel(const double* src, double* dst, long long ncells, int nd, int nb, int nbp, int to_padded) {
  const long long n = ncells * nd * (long long)nbp;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const long long cd = e / nbp;
    const int b = (int)(e - cd * nbp);
    if (to_padded) dst[e] = b < nb ? src[cd * nb + b] : 0.0;
    else if (b < nb) dst[cd * nb + b] = src[e];
  }
}

// E_L of every cell from its intensity row (used after a state restore).
__global__ void energy_L_kernel(const double* I, double* EL, const double* wdir, long long ncells, int nd,
                                ThermoTables th) {
  extern __shared__ double sh[];
  for (long long P = blockIdx.x; P < ncells; P += gridDim.x) {
    const double* row = I + P * (long long)nd * th.nbp;
    double acc = 0.0;
    for (int b = threadIdx.x; b < th.nbp; b += blockDim.x) {
      double G = 0.0;
      for (int d = 0; d < nd; ++d) G = fma(wdir[d], row[(long long)d * th.nbp + b], G);
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

}  // namespace

cudaError_t launch_sweep_fp64(const SweepArgs& a, int dim, int threads, int grid, cudaStream_t s) {
  const int cpb = threads / a.lpc;
  const size_t smem = (3 * (size_t)threads + 8 * (size_t)cpb) * sizeof(double);
  if (dim == 3) sweep_fp64_kernel<3><<<grid, threads, smem, s>>>(a);
  else sweep_fp64_kernel<2><<<grid, threads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_init_cells(double* I, double* I0cell, double* Tp, double* TL, double* EL, const double* Tcells,
                              long long cell0, int ncells, int nd, ThermoTables th, cudaStream_t s) {
  const int grid = ncells < 152 * 16 ? ncells : 152 * 16;
  init_cells_kernel<<<grid, 256, th.nbp * sizeof(double), s>>>(I, I0cell, Tp, TL, EL, Tcells, cell0, ncells, nd, th);
  return cudaGetLastError();
}

cudaError_t launch_wall_I0(double* I0wall, const double* Tfaces, long long nfaces, ThermoTables th, cudaStream_t s) {
  wall_I0_kernel<<<grid_for(nfaces * th.nbp, 256), 256, 0, s>>>(I0wall, Tfaces, nfaces, th);
  return cudaGetLastError();
}

cudaError_t launch_solve_TL(double* TL, const double* EL, const double* Tguess, long long ncells, ThermoTables th,
                            double rtol, int maxit, DevCounters* counters, cudaStream_t s) {
  solve_TL_kernel<<<grid_for(ncells, 128), 128, 0, s>>>(TL, EL, Tguess, ncells, th, rtol, maxit, counters);
  return cudaGetLastError();
}

cudaError_t launch_flux_cells(const double* I, double* q, const DirInfo*, const double* S, long long cell0, int ncells,
                              int nd, int nbp, int dim, cudaStream_t s) {
  const int grid = ncells < 152 * 16 ? ncells : 152 * 16;
  flux_cells_kernel<<<grid, 256, 256 * sizeof(double), s>>>(I, q, S, cell0, ncells, nd, nbp, dim);
  return cudaGetLastError();
}

cudaError_t launch_flux_faces(const double* I, const double* I0wall, const DevGeom* geoms, int geom, int side,
                              const DirInfo* dirs, const double* S, int nd, int nbp, double* face_out, int nfaces,
                              cudaStream_t s) {
  const int grid = nfaces < 152 * 16 ? nfaces : 152 * 16;
  flux_faces_kernel<<<grid, 256, 256 * sizeof(double), s>>>(I, I0wall, geoms, geom, side, dirs, S, nd, nbp, face_out,
                                                           nfaces);
  return cudaGetLastError();
}

cudaError_t launch_mean(const double* v, int n, double* out, cudaStream_t s) {
  mean_kernel<<<1, 256, 256 * sizeof(double), s>>>(v, n, out);
  return cudaGetLastError();
}

cudaError_t launch_I0_from_T(double* I0cell, const double* Tp, long long ncells, ThermoTables th, cudaStream_t s) {
  I0_from_T_kernel<<<grid_for(ncells * th.nbp, 256), 256, 0, s>>>(I0cell, Tp, ncells, th);
  return cudaGetLastError();
}

cudaError_t launch_pack_fp64(const double* src, double* dst, long long ncells, int nd, int nb, int nbp, int to_padded,
                             cudaStream_t s) {
  pack_kernel<<<grid_for(ncells * nd * (long long)nbp, 256), 256, 0, s>>>(src, dst, ncells, nd, nb, nbp, to_padded);
  return cudaGetLastError();
}

cudaError_t launch_energy_L(const double* I, double* EL, const double* wdir, long long ncells, int nd, ThermoTables th,
                            cudaStream_t s) {
  const long long grid = ncells < 152 * 16 ? ncells : 152 * 16;
  energy_L_kernel<<<(int)grid, 64, 64 * sizeof(double), s>>>(I, EL, wdir, ncells, nd, th);
  return cudaGetLastError();
}

}  // namespace bte

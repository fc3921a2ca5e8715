// bte_kernels.cu -- CUDA kernels around the sweep (sm_103a).  The sweep itself
// (upwind update, walls, per-cell reduction, cached-model T_p solve, I0
// refresh; Sec. 3.1, Eq. 4-6) lives in bte_sweep.cuh.  Here:
//   fixup_kernel        exact FP64 T_p solve (Halley on the band quadrature,
//                       bisection fallback) for the cells the model left, which
//                       also refreshes their cached model and I0;
//   solve_cells_kernel  the T_p step of a band-range handle after the caller's
//                       all-reduce of the per-cell energy partials (Sec. 3.3);
//   gs_reduce_kernel    per-cell energies (and the T_p step) after a
//                       sweep-ordered pass (bte_gs.cu);
//   init_cells / state_from_Tp / wall_I0 / wall_dev
//                       equilibrium state, cached models and Eq. 6 ghosts;
//   solve_TL_kernel     T_L on request (cached model first, exact otherwise);
//   flux_cells / flux_faces / mean / pack / energy_L
//                       heat flux, FP64 <-> storage packing, E_L after a restore.
#include <algorithm>

#include "bte_ff.cuh"
#include "bte_mlp.cuh"
#include "bte_quad.cuh"
#include "bte_solve.cuh"
#include "bte_store.cuh"

namespace bte {

namespace {

// Exact temperature solve of the cells the sweep could not settle on their
// cached model: one thread-block cluster of kFixCluster CTAs per cell
// (exact_solve_cluster spreads each evaluation's bands over the cluster's SMs;
// with a handful of such cells per step the solve's latency, not its
// throughput, is what the step waits for).  The start is the model root, or
// when there is none the previous T_p (plain mode) or the learned guess (net
// A, then surrogate Newton steps on net B, by warp 0 of each CTA: the same
// value everywhere); the exact FP64 quadrature then refines it (each
// evaluation becomes the cell's cached model) and every CTA refreshes I0 of
// the bands whose model row it wrote.
constexpr int kFixThreads = 128;
constexpr int kFixCluster = 4;

__global__ void __cluster_dims__(kFixCluster, 1, 1) __launch_bounds__(kFixThreads)
    fixup_kernel(SweepArgs a, int learned, MLPView m) {
  extern __shared__ double fsm[];  // exact_solve_cluster scratch, T0, then the learned-mode buffers
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank(), nr = (int)cl.num_blocks();
  const unsigned cid = blockIdx.x / (unsigned)nr, ncl = gridDim.x / (unsigned)nr;
  const int nbp = a.th.nbp;
  const int own0 = rank * nbp / nr, own1 = (rank + 1) * nbp / nr;  // bands whose model row this CTA writes
  double* solve_sm = fsm;
  double* t0_sm = fsm + cta_solve_smem_doubles(nbp);
  float* ybuf = reinterpret_cast<float*>(t0_sm + 2);
  float* hbuf = ybuf + 2 * nbp;
  const unsigned count = *a.fix_count;
  unsigned long long evals = 0, fb = 0, bad = 0;
  unsigned par = 0;  // evaluations of this cluster so far (the solve's buffer parity)
  for (unsigned w = cid; w < count; w += ncl) {  // the same items, in the same order, in every CTA of the cluster
    const FixItem it = a.fix[w];
    const long long P = it.P;
    // learned mode: the networks' guess starts the cells that have no usable
    // root of their cached model (a cold or far-off start); a model root, when
    // there is one, is the closer start (measured: twice the evaluations from
    // the networks' guess on the learned 3-D workload)
    const bool net = learned && !it.model;  // uniform over the cluster (one item)
    if (net) {
      if (threadIdx.x < 32) {
        const double g = mlp_guess_T(m, a.th.a_p, it.Ep, 2, ybuf, hbuf);
        if (threadIdx.x == 0) t0_sm[0] = g;
      }
      __syncthreads();
    }
    const double T0 = net ? t0_sm[0] : it.T0;
    const SolveResult r = exact_solve_cluster(a.th, it.Ep, T0, a.trust_rel, a.maxit, a.J + (P * 3) * nbp, solve_sm, par);
    evals += r.evals;
    fb += r.fallback;
    bad += r.bad;
    __syncthreads();  // this CTA's model rows, written by the solve, before its I0 refresh reads them
    // I0 refresh of the stored bands whose model rows this CTA wrote, at r.Te
    const double hd2 = 0.5 * r.delta * r.delta;
    const int s0 = max(own0 - a.th.band0, 0), s1 = min(own1 - a.th.band0, a.th.nbo);
    for (int b = s0 + (int)threadIdx.x; b < s1; b += blockDim.x) {
      const long long j = (P * 3) * nbp + a.th.band0 + b;
      a.I0cell[P * a.th.nbo + b] = b < a.th.nbr ? fma(a.J[j + 2 * nbp], hd2, fma(a.J[j + nbp], r.delta, a.J[j])) : 0.0;
    }
    if (rank == 0 && threadIdx.x == 0) {
      a.Teval[P] = r.Te;
      a.Tp[P] = r.Te + r.delta;
      a.Msum[3 * P] = r.M[0];  // the model just written to J
      a.Msum[3 * P + 1] = r.M[1];
      a.Msum[3 * P + 2] = r.M[2];
    }
    __syncthreads();  // t0_sm and the solve scratch are reused by the next item
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
  if (rank == 0 && threadIdx.x == 0 && a.counters) {
    if (evals) atomicAdd(&a.counters->evals, evals);
    if (fb) atomicAdd(&a.counters->fallbacks, fb);
    if (bad) atomicAdd(&a.counters->nonfinite, bad);
  }
}

// ---------------------------------------------------------------------------
// Per-cell thermodynamic state at temperature T: I0cell, cached model J at T
// with its T_p sums Msum, T_e = T_p = T.  One CTA per cell (grid-stride);
// bands over threads.
__device__ void cell_state_at(double* I0cell, double* J, double* Msum, long long P, double T, ThermoTables th,
                              double* row) {
  const double rT = 1.0 / T;
  for (int b = threadIdx.x; b < th.nbp; b += blockDim.x) {  // every band (the temperature model)
    double f, d1, d2;
    band_I0_d2(th.node_c + b * th.ng, th.node_C + b * th.ng, th.ng, rT, f, d1, d2);
    row[b] = f;
    J[(P * 3 + 0) * th.nbp + b] = f;
    J[(P * 3 + 1) * th.nbp + b] = d1;
    J[(P * 3 + 2) * th.nbp + b] = d2;
  }
  __syncthreads();
  for (int b = threadIdx.x; b < th.nbo; b += blockDim.x)  // stored bands
    I0cell[P * th.nbo + b] = b < th.nbr ? row[th.band0 + b] : 0.0;
  if (threadIdx.x == 0) {  // the model's sums with the T_p weights
    double m0 = 0.0, m1 = 0.0, m2 = 0.0;
    for (int b = 0; b < th.nbp; ++b) {
      const double ap = th.a_p[b];
      m0 = fma(ap, J[(P * 3 + 0) * th.nbp + b], m0);
      m1 = fma(ap, J[(P * 3 + 1) * th.nbp + b], m1);
      m2 = fma(ap, J[(P * 3 + 2) * th.nbp + b], m2);
    }
    Msum[3 * P] = m0;
    Msum[3 * P + 1] = m1;
    Msum[3 * P + 2] = m2;
  }
}

// Equilibrium initial state: I = I0_b(T_P) for every direction (stored as the
// deviation I0_b(T_P) - I0_b(T_ref) in the reduced modes).
template <typename S>
__global__ void init_cells_kernel(S* I, double* I0cell, double* J, double* Msum, double* Tp, double* Te, double* TL,
                                  double* EL, const double* Tcells, const double* I0ref, long long cell0, int ncells,
                                  int nd, ThermoTables th) {
  extern __shared__ double row[];  // [nbp]
  for (int c = blockIdx.x; c < ncells; c += gridDim.x) {
    const long long P = cell0 + c;
    const double T = Tcells[c];
    cell_state_at(I0cell, J, Msum, P, T, th, row);
    __syncthreads();
    const long long n = (long long)nd * th.nbo;
    for (long long e = threadIdx.x; e < n; e += blockDim.x) {
      const int b = (int)(e % th.nbo);  // stored band; I0ref holds the stored bands
      const double v = b < th.nbr ? (sizeof(S) == 8 ? row[th.band0 + b] : row[th.band0 + b] - I0ref[b]) : 0.0;
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
__global__ void state_from_Tp_kernel(double* I0cell, double* J, double* Msum, const double* Tp, double* Te,
                                     long long ncells, ThermoTables th) {
  extern __shared__ double row[];
  for (long long P = blockIdx.x; P < ncells; P += gridDim.x) {
    cell_state_at(I0cell, J, Msum, P, Tp[P], th, row);
    if (threadIdx.x == 0) Te[P] = Tp[P];
    __syncthreads();
  }
}

// Wall ghost intensities (FP64): one thread per (face, band).
__global__ void wall_I0_kernel(double* I0wall, const double* Tf, long long nfaces, ThermoTables th) {
  const long long n = nfaces * th.nbo;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const long long f = e / th.nbo;
    const int b = (int)(e - f * th.nbo);
    const int bg = th.band0 + b;
    I0wall[e] = b < th.nbr ? band_I0(th.node_c + bg * th.ng, th.node_C + bg * th.ng, th.ng, 1.0 / Tf[f]) : 0.0;
  }
}

// Deviation ghosts for the reduced modes: I0wall - I0ref as FP32.
__global__ void wall_dev_kernel(float* out, const double* I0wall, const double* I0ref, long long n, int nbp) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    out[e] = (float)(I0wall[e] - I0ref[e % nbp]);
}

// Lattice temperature: sum_b a_L,b I0_b(T) = E_L per cell (evaluated on
// request).  One warp per cell: the root of the cell's cached quadratic model
// of I0_b(T) around T_e (the one the T_p solve keeps) when it lies inside the
// trust radius, else Halley on the exact band quadrature from there (or from
// the guess), bisection as the fallback.
__global__ void solve_TL_kernel(double* TL, const double* EL, const double* Tguess, const double* J,
                                const double* Teval, long long ncells, ThermoTables th, double trust_rel, int maxit,
                                DevCounters* counters) {
  const int warps = blockDim.x / 32, lane = threadIdx.x & 31;
  const int nbp = th.nbp;
  for (long long P = blockIdx.x * (long long)warps + threadIdx.x / 32; P < ncells; P += (long long)gridDim.x * warps) {
    const double E = EL[P];
    if (!isfinite(E)) {
      if (lane == 0) {
        TL[P] = E;
        if (counters) atomicAdd(&counters->nonfinite, 1ULL);
      }
      continue;
    }
    double F = 0.0, F1 = 0.0, F2 = 0.0;
    for (int b = lane; b < nbp; b += 32) {
      const double w = th.a_L[b];
      F = fma(w, J[(P * 3 + 0) * nbp + b], F);
      F1 = fma(w, J[(P * 3 + 1) * nbp + b], F1);
      F2 = fma(w, J[(P * 3 + 2) * nbp + b], F2);
    }
    for (int o = 16; o > 0; o >>= 1) {
      F += __shfl_xor_sync(0xffffffffu, F, o);
      F1 += __shfl_xor_sync(0xffffffffu, F1, o);
      F2 += __shfl_xor_sync(0xffffffffu, F2, o);
    }
    F -= E;
    const double Te = Teval[P];
    const double disc = F1 * F1 - 2.0 * F * F2;
    const double delta = (disc >= 0.0 && F1 > 0.0) ? -2.0 * F / (F1 + sqrt(disc)) : -F / F1;
    const double Tn = Te + delta;
    if (isfinite(Tn) && fabs(delta) <= trust_rel * Tn) {
      if (lane == 0) TL[P] = Tn;
      continue;
    }
    const double start = (isfinite(Tn) && Tn >= kTmin && Tn <= kTmax) ? Tn : Tguess[P];
    const SolveResult r = exact_solve_warp(th, E, start, trust_rel, maxit, nullptr, th.a_L);
    if (lane == 0) {
      TL[P] = r.Te + r.delta;
      if (counters && r.fallback) atomicAdd(&counters->fallbacks, 1ULL);
      if (counters && r.bad) atomicAdd(&counters->nonfinite, 1ULL);
    }
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
      else if (g.bc[side] == 3) v = full_I(reinterpret_cast<const S*>(g.gdir[side]), (long long)f * nd * nbp + e, b, I0ref);
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
    const long long base = P * (long long)nd * th.nbo;
    double acc = 0.0;
    for (int b = threadIdx.x; b < th.nbo; b += blockDim.x) {
      double G = 0.0;
      for (int d = 0; d < nd; ++d) G = fma(wdir[d], full_I(I, base + (long long)d * th.nbo + b, b, I0ref), G);
      acc = fma(G, th.inv_v[b], acc);
    }
    const double t = block_sum(acc, sh);
    if (threadIdx.x == 0) EL[P] = t;
  }
}

// T_p step of one cell from its energies (E_L, E_p over every band), by one
// warp: the T_p equation on the cell's cached quadratic model of all bands,
// I0 refresh of the stored bands inside the trust radius, the rest to the
// fix-up list.
__device__ void solve_cell_warp(const SweepArgs& a, long long P, double EL, double Ep, int lane,
                                unsigned long long& solves, unsigned long long& badc) {
  const int nbp = a.th.nbp;
  const bool finite = isfinite(EL) && isfinite(Ep);
  if (!a.solve_tp) {  // every beta_b is zero: only E_L is kept
    if (lane == 0) {
      a.EL[P] = EL;
      if (!finite) ++badc;
    }
    return;
  }
  // the model's sums, kept with J (sum_b a_p,b J_k,b)
  double F = a.Msum[3 * P] - Ep;
  const double F1 = a.Msum[3 * P + 1], F2 = a.Msum[3 * P + 2];
  const double Te = a.Teval[P];
  const double disc = F1 * F1 - 2.0 * F * F2;
  const double delta = (disc >= 0.0 && F1 > 0.0) ? -2.0 * F / (F1 + sqrt(disc)) : -F / F1;
  const double Tn = Te + delta;
  const bool ok = finite && isfinite(Tn) && fabs(delta) <= a.trust_rel * Tn;
  if (lane == 0) {
    a.EL[P] = EL;
    if (!finite) ++badc;
    else ++solves;
    if (finite && !ok) {
      const unsigned k = atomicAdd(a.fix_count, 1u);
      FixItem fi;
      fi.P = P;
      fi.Ep = Ep;
      fi.model = (isfinite(Tn) && Tn >= kTmin && Tn <= kTmax) ? 1 : 0;
      fi.T0 = fi.model ? Tn : a.Tp[P];
      fi.pad = 0;
      a.fix[k] = fi;
    }
    if (ok) a.Tp[P] = Tn;
  }
  if (ok) {
    const double hd2 = 0.5 * delta * delta;
    for (int b = lane; b < a.th.nbo; b += 32) {
      const long long j = (P * 3) * nbp + a.th.band0 + b;
      a.I0cell[P * a.th.nbo + b] = b < a.th.nbr ? fma(a.J[j + 2 * nbp], hd2, fma(a.J[j + nbp], delta, a.J[j])) : 0.0;
    }
  }
}

__device__ void flush_counters(const SweepArgs& a, int lane, unsigned long long solves, unsigned long long badc) {
  if (lane == 0 && a.counters) {
    if (solves) atomicAdd(&a.counters->solves, solves);
    if (badc) atomicAdd(&a.counters->nonfinite, badc);
  }
}

// Temperature step of a band-range handle after the caller's all-reduce: one
// warp per cell, E_L and E_p from Epart.
__global__ void solve_cells_kernel(SweepArgs a, long long ncells) {
  const int warps = blockDim.x / 32, lane = threadIdx.x & 31;
  unsigned long long solves = 0, badc = 0;
  for (long long P = blockIdx.x * (long long)warps + threadIdx.x / 32; P < ncells; P += (long long)gridDim.x * warps)
    solve_cell_warp(a, P, a.Epart[2 * P], a.Epart[2 * P + 1], lane, solves, badc);
  flush_counters(a, lane, solves, badc);
}

// Per-cell step after a separate sweep (the sweep-ordered pass, the
// unstructured sweep): one CTA of 8 warps per cell.  Warp w sums the directions [w nd/8, (w+1) nd/8) for every stored
// band (lanes over band pairs); the 8 partials are added in warp order in
// shared memory (deterministic), then warp 0 forms
// G_b = sum_d w_d I^{k+1}_{d,b}, E_L = sum_b G_b / v_b, E_p = sum_b beta_b G_b / v_b
// and either writes them to Epart (band-range handle, for the caller's
// all-reduce) or solves T_p and refreshes I0 at once (whole handle).
// Within a warp the sums over a run of equal-weight directions are exact
// 64-bit fixed-point additions on the integer pipe (unit 2^(E-50) for the
// cell's I0 of exponent E; a value up to 32 I0 adds at most 2^55, so a run of
// 256 cannot overflow), closed by one FP64 FMA (sum x w x unit).  Values
// beyond that range (or negative, NaN) take the FP64 FMA directly.
// Reduced storage (deviations from I0_b(T_ref)): each lane sums w_d x deviation
// in FP32, flushed to FP64 every 16 directions, and G_b gets W I0_b(T_ref).
constexpr int kRedWarps = 8;

template <typename S>
__device__ __forceinline__ void reduce_dev_warp(const SweepArgs& a, const S* row, int d0, int d1, int lane,
                                                double* gpart_w) {
  const int nbo = a.th.nbo;
  for (int b0 = 2 * lane; b0 < nbo; b0 += 64) {  // two bands per lane
    double G0 = 0.0, G1 = 0.0;
    for (int d = d0; d < d1; d += 16) {  // 16 directions: loads first, then the float sums
      const int m = min(16, d1 - d);
      float x0[16], x1[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        x0[k] = x1[k] = 0.f;
        if (k < m) {
          const S* p = row + (long long)(d + k) * nbo + b0;
          x0[k] = Tr<S>::to_float(p[0]);
          x1[k] = Tr<S>::to_float(p[1]);
        }
      }
      float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const float w = k < m ? a.wdir32[d + k] : 0.f;
        acc0 = fmaf(w, x0[k], acc0);
        acc1 = fmaf(w, x1[k], acc1);
      }
      G0 += (double)acc0;
      G1 += (double)acc1;
    }
    gpart_w[b0] = G0;
    gpart_w[b0 + 1] = G1;
  }
}

template <typename S>
__global__ void __launch_bounds__(256, 4) gs_reduce_kernel(SweepArgs a, long long ncells) {
  extern __shared__ double gpart[];  // [kRedWarps][nbo]
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nbo = a.th.nbo, nd = a.nd, lpc = nbo / 2;
  const int d0 = (int)((long long)wid * nd / kRedWarps), d1 = (int)((long long)(wid + 1) * nd / kRedWarps);
  unsigned long long solves = 0, badc = 0;
  for (long long P = blockIdx.x; P < ncells; P += gridDim.x) {
    if constexpr (sizeof(S) != 8) {
      reduce_dev_warp<S>(a, reinterpret_cast<const S*>(a.Iout) + P * (long long)nd * nbo, d0, d1, lane, gpart + wid * nbo);
    } else {
    const double* row = reinterpret_cast<const double*>(a.Iout) + P * (long long)nd * nbo;
    for (int lp = lane; lp < lpc; lp += 32) {
      const int b0 = 2 * lp;
      double G[2] = {0.0, 0.0};
      unsigned long long facc[2] = {0ull, 0ull};
      long long fsc[2];
      int fe0[2];
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        const int e0 = (int)((unsigned long long)__double_as_longlong(a.I0cell[P * nbo + b0 + v]) >> 52);
        const bool on = e0 >= 200 && e0 <= 1900;
        fe0[v] = on ? e0 + 4 : -1;
        fsc[v] = on ? (long long)(e0 - 1073) * (1LL << 52) : 0;
      }
      long long wrun = d0 < d1 ? __double_as_longlong(a.wdir[d0]) : 0;
      int nrun = 0;
      auto add = [&](double2 x, int d) {
        const long long wb = __double_as_longlong(a.wdir[d]);
        if (wb != wrun || nrun == 256) {  // close the run: sum x (w x unit)
#pragma unroll
          for (int v = 0; v < 2; ++v) {
            if (facc[v] != 0ull) G[v] = fma(__ull2double_rn(facc[v]), __longlong_as_double(wrun + fsc[v]), G[v]);
            facc[v] = 0ull;
          }
          wrun = wb;
          nrun = 0;
        }
        ++nrun;
        const double xv[2] = {x.x, x.y};
        bool big = false;
#pragma unroll
        for (int v = 0; v < 2; ++v) {
          const unsigned long long rb = (unsigned long long)__double_as_longlong(xv[v]);
          const int e = (int)(rb >> 52);  // sign bit included: negative values take the FP64 path
          const unsigned long long m = ((rb & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull) << 2;
          const int sh = e == 0 ? 63 : min(fe0[v] - e, 63);  // zero (and subnormal) adds nothing
          facc[v] += sh >= 0 ? (m >> sh) : 0ull;
          big |= sh < 0;
        }
        // rare: a value beyond the fixed-point range (a warp-uniform branch, so
        // no FP64 instruction is issued in the common case)
        if (__any_sync(__activemask(), big)) {
#pragma unroll
          for (int v = 0; v < 2; ++v) {
            const int e = (int)((unsigned long long)__double_as_longlong(xv[v]) >> 52);
            if (e != 0 && fe0[v] - e < 0) G[v] = fma(a.wdir[d], xv[v], G[v]);
          }
        }
      };
      int d = d0;
      for (; d + 4 <= d1; d += 4) {
        double2 x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = __ldcs(reinterpret_cast<const double2*>(row + (long long)(d + u) * nbo + b0));
#pragma unroll
        for (int u = 0; u < 4; ++u) add(x[u], d + u);
      }
      for (; d < d1; ++d) add(__ldcs(reinterpret_cast<const double2*>(row + (long long)d * nbo + b0)), d);
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        if (facc[v] != 0ull) G[v] = fma(__ull2double_rn(facc[v]), __longlong_as_double(wrun + fsc[v]), G[v]);
        gpart[wid * nbo + b0 + v] = G[v];
      }
    }
    }
    __syncthreads();
    if (wid == 0) {
      double el = 0.0, ep = 0.0;
      for (int b = lane; b < nbo; b += 32) {
        double G = gpart[b];
        for (int w = 1; w < kRedWarps; ++w) G += gpart[w * nbo + b];
        if constexpr (sizeof(S) != 8) G = fma(a.Wtot, a.I0ref[b], G);  // the reference part, sum_d w_d I0_b(T_ref)
        const double e = G * a.th.inv_v[b];
        el += e;
        ep = fma(a.th.beta[b], e, ep);
      }
      for (int o = 16; o > 0; o >>= 1) {
        el += __shfl_xor_sync(0xffffffffu, el, o);
        ep += __shfl_xor_sync(0xffffffffu, ep, o);
      }
      if (a.partial) {
        if (lane == 0) {
          a.Epart[2 * P] = el;
          a.Epart[2 * P + 1] = ep;
        }
      } else {
        solve_cell_warp(a, P, el, ep, lane, solves, badc);
      }
    }
    __syncthreads();
  }
  if (wid == 0) flush_counters(a, lane, solves, badc);
}

// Diffuse wall ghosts of one side of one geometry: for every face, per band,
// sum over the directions leaving through the wall of |S_d,ax| I_d, divided by
// sum over the entering directions of |S_d,ax|, from the wall cell's current
// iterate, into the FP64 ghost row (and the FP32 deviation row in the reduced
// modes).  One warp per face, lanes over bands, directions in order.
template <typename S>
__global__ void diffuse_ghost_kernel(const S* I, const double* I0ref, double* I0wall, float* I0wall_dev,
                                     const DevGeom* geoms, int geom, int side, const double* Sd, int nd, int nbp,
                                     int nfaces) {
  const DevGeom g = geoms[geom];
  const int ax = side >> 1;
  const bool high = side & 1;
  const int warps = blockDim.x / 32, lane = threadIdx.x & 31;
  const long long row = (long long)nd * nbp;
  for (int f = blockIdx.x * warps + threadIdx.x / 32; f < nfaces; f += gridDim.x * warps) {
    int i, j, k;  // wall cell of face f (x sides: j + ny k, y sides: i + nx k, z sides: i + nx j)
    if (ax == 0) { i = high ? g.nx - 1 : 0; j = f % g.ny; k = f / g.ny; }
    else if (ax == 1) { j = high ? g.ny - 1 : 0; i = f % g.nx; k = f / g.nx; }
    else { k = high ? g.nz - 1 : 0; i = f % g.nx; j = f / g.nx; }
    const long long P = g.cell0 + ((long long)k * g.ny + j) * g.nx + i;
    double den = 0.0;
    for (int d = 0; d < nd; ++d) {
      const double sd = Sd[3 * d + ax];
      if (!(high ? sd > 0.0 : sd < 0.0) && sd != 0.0) den += fabs(sd);
    }
    for (int b = lane; b < nbp; b += 32) {
      double num = 0.0;
      for (int d = 0; d < nd; ++d) {
        const double sd = Sd[3 * d + ax];
        if (high ? sd > 0.0 : sd < 0.0) num += fabs(sd) * full_I(I, P * row + (long long)d * nbp + b, b, I0ref);
      }
      const double v = num / den;
      const long long e = (g.face0[side] + f) * nbp + b;
      I0wall[e] = v;
      if (I0wall_dev) I0wall_dev[e] = (float)(v - I0ref[b]);
    }
  }
}

// Partially specular side: one CTA of kPartWarps warps per wall face.  The
// diffuse value per band, D_b = sum_{out} |S_ax| I / sum_{in} |S_ax| of the
// wall cell (warps over direction ranges, added in warp order), then for
// every direction and band the ghost p I(mirror of d) + (1 - p) D_b, stored in
// the storage type (a deviation from I0_b(T_ref) in the reduced modes).
constexpr int kPartWarps = 8;

template <typename S>
__global__ void __launch_bounds__(32 * kPartWarps) partial_ghost_kernel(const S* I, const double* I0ref,
                                                                        const DevGeom* geoms, int geom, int side,
                                                                        const double* Sd, const DirInfo* dirs, int nd,
                                                                        int nbp, int nfaces, double p, S* out) {
  extern __shared__ double part[];  // [kPartWarps][nbp] partial numerators, then D [nbp]
  const DevGeom g = geoms[geom];
  const int ax = side >> 1;
  const bool high = side & 1;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long row = (long long)nd * nbp;
  const int d0 = (int)((long long)wid * nd / kPartWarps), d1 = (int)((long long)(wid + 1) * nd / kPartWarps);
  double den = 0.0;
  for (int d = 0; d < nd; ++d) {
    const double sd = Sd[3 * d + ax];
    if (!(high ? sd > 0.0 : sd < 0.0) && sd != 0.0) den += fabs(sd);
  }
  for (int f = blockIdx.x; f < nfaces; f += gridDim.x) {
    int i, j, k;  // wall cell of face f (x sides: j + ny k, y sides: i + nx k, z sides: i + nx j)
    if (ax == 0) { i = high ? g.nx - 1 : 0; j = f % g.ny; k = f / g.ny; }
    else if (ax == 1) { j = high ? g.ny - 1 : 0; i = f % g.nx; k = f / g.nx; }
    else { k = high ? g.nz - 1 : 0; i = f % g.nx; j = f / g.nx; }
    const long long P = g.cell0 + ((long long)k * g.ny + j) * g.nx + i;
    for (int b = lane; b < nbp; b += 32) {
      double num = 0.0;
      for (int d = d0; d < d1; ++d) {
        const double sd = Sd[3 * d + ax];
        if (high ? sd > 0.0 : sd < 0.0) num = fma(fabs(sd), full_I(I, P * row + (long long)d * nbp + b, b, I0ref), num);
      }
      part[wid * nbp + b] = num;
    }
    __syncthreads();
    double* D = part + kPartWarps * nbp;
    for (int b = threadIdx.x; b < nbp; b += blockDim.x) {
      double num = 0.0;
      for (int w = 0; w < kPartWarps; ++w) num += part[w * nbp + b];
      D[b] = num / den;
    }
    __syncthreads();
    for (long long e = threadIdx.x; e < row; e += blockDim.x) {
      const int d = (int)(e / nbp), b = (int)(e - (long long)d * nbp);
      const int r = ax == 0 ? dirs[d].rx : (ax == 1 ? dirs[d].ry : dirs[d].rz);
      const double v = fma(p, full_I(I, P * row + (long long)r * nbp + b, b, I0ref), (1.0 - p) * D[b]);
      if constexpr (sizeof(S) == 8) out[f * row + e] = v;
      else if constexpr (sizeof(S) == 4) out[f * row + e] = (float)(v - I0ref[b]);
      else out[f * row + e] = __double2bfloat16(v - I0ref[b]);
    }
    __syncthreads();
  }
}

inline int grid_for(long long n, int threads) {
  long long g = (n + threads - 1) / threads;
  if (g > 152LL * 64) g = 152LL * 64;
  return (int)(g < 1 ? 1 : g);
}

inline int cell_grid(long long ncells) { return (int)(ncells < 152 * 16 ? (ncells < 1 ? 1 : ncells) : 152 * 16); }

}  // namespace

int values_per_lane(int precision) { return precision == 0 ? 2 : (precision == 1 ? 4 : 8); }

cudaError_t launch_sweep(int precision, int pd, const SweepArgs& a, int dim, int threads, int grid, cudaStream_t s) {
  if (precision == 0) return launch_sweep_fp64(pd, a, dim, threads, grid, s);
  if (precision == 1) return launch_sweep_fp32(pd, a, dim, threads, grid, s);
  return launch_sweep_bf16(pd, a, dim, threads, grid, s);
}

cudaError_t launch_fixup(const SweepArgs& a, const MLPView* mlp, cudaStream_t s) {
  const size_t sm = (cta_solve_smem_doubles(a.th.nbp) + 2) * sizeof(double) +
                    (mlp ? (2 * (size_t)a.th.nbp + 4 * kHidden) * sizeof(float) : 0);
  MLPView m{};
  if (mlp) m = *mlp;
  fixup_kernel<<<2 * 152, kFixThreads, sm, s>>>(a, mlp ? 1 : 0, m);  // 76 clusters of kFixCluster CTAs
  return cudaGetLastError();
}

cudaError_t launch_diffuse_ghosts(int precision, const void* I, const double* I0ref, double* I0wall, float* I0wall_dev,
                                  const DevGeom* geoms, int geom, int side, const double* S, int nd, int nbp,
                                  int nfaces, cudaStream_t s) {
  const int grid = (int)std::min<long long>((nfaces + 3) / 4, 152LL * 16);
  if (precision == 0)
    diffuse_ghost_kernel<double><<<grid, 128, 0, s>>>((const double*)I, I0ref, I0wall, nullptr, geoms, geom, side, S, nd,
                                                      nbp, nfaces);
  else if (precision == 1)
    diffuse_ghost_kernel<float><<<grid, 128, 0, s>>>((const float*)I, I0ref, I0wall, I0wall_dev, geoms, geom, side, S, nd,
                                                     nbp, nfaces);
  else
    diffuse_ghost_kernel<__nv_bfloat16><<<grid, 128, 0, s>>>((const __nv_bfloat16*)I, I0ref, I0wall, I0wall_dev, geoms,
                                                             geom, side, S, nd, nbp, nfaces);
  return cudaGetLastError();
}

cudaError_t launch_partial_ghosts(int precision, const void* I, const double* I0ref, const DevGeom* geoms, int geom,
                                  int side, const double* S, const DirInfo* dirs, int nd, int nbp, int nfaces,
                                  double p, void* out, cudaStream_t s) {
  const int grid = (int)std::min<long long>(std::max(nfaces, 1), 152LL * 16);
  const size_t sm = (size_t)(kPartWarps + 1) * nbp * sizeof(double);
  if (precision == 0)
    partial_ghost_kernel<double><<<grid, 32 * kPartWarps, sm, s>>>((const double*)I, I0ref, geoms, geom, side, S, dirs,
                                                                   nd, nbp, nfaces, p, (double*)out);
  else if (precision == 1)
    partial_ghost_kernel<float><<<grid, 32 * kPartWarps, sm, s>>>((const float*)I, I0ref, geoms, geom, side, S, dirs, nd,
                                                                  nbp, nfaces, p, (float*)out);
  else
    partial_ghost_kernel<__nv_bfloat16><<<grid, 32 * kPartWarps, sm, s>>>((const __nv_bfloat16*)I, I0ref, geoms, geom,
                                                                          side, S, dirs, nd, nbp, nfaces, p,
                                                                          (__nv_bfloat16*)out);
  return cudaGetLastError();
}

cudaError_t launch_solve_cells(const SweepArgs& a, long long ncells, cudaStream_t s) {
  solve_cells_kernel<<<cell_grid(ncells / 4 + 1), 128, 0, s>>>(a, ncells);
  return cudaGetLastError();
}

cudaError_t launch_gs_reduce(int precision, const SweepArgs& a, long long ncells, cudaStream_t s) {
  const int grid = (int)std::min<long long>(std::max(ncells, 1LL), 152LL * 64);
  const size_t sm = (size_t)kRedWarps * a.th.nbo * sizeof(double);
  if (precision == 0) gs_reduce_kernel<double><<<grid, 32 * kRedWarps, sm, s>>>(a, ncells);
  else if (precision == 1) gs_reduce_kernel<float><<<grid, 32 * kRedWarps, sm, s>>>(a, ncells);
  else gs_reduce_kernel<__nv_bfloat16><<<grid, 32 * kRedWarps, sm, s>>>(a, ncells);
  return cudaGetLastError();
}

cudaError_t launch_init_cells(int precision, void* I, double* I0cell, double* J, double* Msum, double* Tp, double* Te,
                              double* TL, double* EL, const double* Tcells, const double* I0ref, long long cell0,
                              int ncells, int nd, ThermoTables th, cudaStream_t s) {
  const int grid = cell_grid(ncells);
  const size_t sm = th.nbp * sizeof(double);
  if (precision == 0)
    init_cells_kernel<double><<<grid, 256, sm, s>>>((double*)I, I0cell, J, Msum, Tp, Te, TL, EL, Tcells, I0ref, cell0,
                                                    ncells, nd, th);
  else if (precision == 1)
    init_cells_kernel<float><<<grid, 256, sm, s>>>((float*)I, I0cell, J, Msum, Tp, Te, TL, EL, Tcells, I0ref, cell0,
                                                   ncells, nd, th);
  else
    init_cells_kernel<__nv_bfloat16><<<grid, 256, sm, s>>>((__nv_bfloat16*)I, I0cell, J, Msum, Tp, Te, TL, EL, Tcells,
                                                           I0ref, cell0, ncells, nd, th);
  return cudaGetLastError();
}

cudaError_t launch_state_from_Tp(double* I0cell, double* J, double* Msum, const double* Tp, double* Te,
                                 long long ncells, ThermoTables th, cudaStream_t s) {
  state_from_Tp_kernel<<<cell_grid(ncells), 64, th.nbp * sizeof(double), s>>>(I0cell, J, Msum, Tp, Te, ncells,
                                                                               th);  // row: all bands
  return cudaGetLastError();
}

cudaError_t launch_wall_I0(double* I0wall, const double* Tfaces, long long nfaces, ThermoTables th, cudaStream_t s) {
  wall_I0_kernel<<<grid_for(nfaces * th.nbo, 256), 256, 0, s>>>(I0wall, Tfaces, nfaces, th);
  return cudaGetLastError();
}

cudaError_t launch_wall_dev(float* out, const double* I0wall, const double* I0ref, long long nfaces, int nbp,
                            cudaStream_t s) {
  wall_dev_kernel<<<grid_for(nfaces * nbp, 256), 256, 0, s>>>(out, I0wall, I0ref, nfaces * nbp, nbp);
  return cudaGetLastError();
}

cudaError_t launch_solve_TL(double* TL, const double* EL, const double* Tguess, const double* J, const double* Teval,
                            long long ncells, ThermoTables th, double trust_rel, int maxit, DevCounters* counters,
                            cudaStream_t s) {
  solve_TL_kernel<<<cell_grid(ncells / 4 + 1), 128, 0, s>>>(TL, EL, Tguess, J, Teval, ncells, th, trust_rel, maxit,
                                                            counters);
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

namespace {
__global__ void ff_to_doubles_kernel(ulonglong2* buf, long long npairs) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npairs; i += (long long)gridDim.x * blockDim.x) {
    const ulonglong2 v = buf[i];
    double a, b;
    ff::to_doubles(ff::P2{v.x, v.y}, a, b);
    buf[i] = make_ulonglong2((unsigned long long)__double_as_longlong(a), (unsigned long long)__double_as_longlong(b));
  }
}
}  // namespace

cudaError_t launch_ff_to_doubles(void* buf, long long npairs, cudaStream_t s) {
  if (npairs <= 0) return cudaSuccess;
  ff_to_doubles_kernel<<<grid_for(npairs, 256), 256, 0, s>>>(reinterpret_cast<ulonglong2*>(buf), npairs);
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

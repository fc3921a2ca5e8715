// bte_sweep.cuh -- the sweep kernel of one inner iteration (sm_103a).
//
// sweep_kernel<DIM, S, MINB, BM>: a CTA owns a run of cells of one geometry; each
// cell is served by a team of lpc x dteam lanes.  Lane (q, l) holds the V
// consecutive bands V*l.. as one vector (FP64: 2 doubles, FP32: 4 floats,
// BF16: 8 bf16) and walks the directions d = q, q + dteam, ...; a team step
// thus covers dteam consecutive directions of the cell's row, ~0.9 KB of
// contiguous memory per array, which is what keeps HBM streaming at full
// rate (one 16-byte vector per row per step reaches only ~70 %).  For every
// (cell, direction, band) (Sec. 3.1, Eq. 5):
//   FP64     I^{k+1} = A_n I^n + A_x I_up,x^k + A_y I_up,y^k (+ A_z I_up,z^k) + A_s I0^k
//   FP32/BF16 I^{k+1} = P I^n + Q (v_b sum_ax c_ax I_up,ax^k + beta_b I0^k)
// (implicit: point-Jacobi sweep of backward Euler; explicit: forward Euler with
// I^k = I^n).  The upwind value is the neighbour cell on the side S_d comes
// from, or the Eq. 6 ghost at a wall (I0 of the wall face, or the cell's own
// value in the mirrored direction).  FP32 and BF16 store the deviation
// I - I0_b(T_ref): the update is affine with coefficients summing to one, so
// the deviation obeys the same update with I0 and wall ghosts shifted.
// Each lane accumulates its part of G_b = sum_d w_d I^{k+1}_{d,b} in registers
// (FP64: exact fixed-point sums per run of equal-weight directions; reduced
// modes: float partials flushed to FP64).  The epilogue of an item: the band
// owners add the dteam partials per band in a fixed order and reduce their
// bands to E_L, E_p and the model sums; then one warp per cell adds those with
// a shuffle tree and solves the T_p equation on the cell's cached quadratic
// model of I0_b(T) (I0, dI0/dT, d2I0/dT2 at its last exact evaluation point
// T_e).  The model root is accepted inside the trust radius
// |T - T_e| <= trust_rel T, where the Taylor remainder is below the solve
// tolerance, and the warp refreshes the cell's I0 from it; other cells go to
// the fix-up kernel (exact FP64 band quadrature).  Five CTA barriers per item.
// Memory: I^n is read once, I^{k+1} written once, and each I^k row read from
// DRAM once (adjacent cells, processed together, re-read it from L2).  Each
// thread copies the operands of its next directions into shared memory with
// cp.async kStages-1 steps before it uses them.  MINB is the launch-bounds
// minimum of resident CTAs per SM (a register cap).  BM: FP64 storage, the
// inner-iteration form (0 I^n read, 1 B = A_n I^n also stored, 2 B read);
// reduced modes, the scheme (0 implicit, 3 explicit).
#pragma once
#include <type_traits>

#include "bte_ff.cuh"
#include "bte_store.cuh"

namespace bte {
namespace sweep {

// Per-cell addressing of one lane: its rows in I^n, I^k, I^{k+1} (band offset
// applied), the element strides to the x/y/z neighbours and which sides are
// walls, so a direction's upwind address is one select and one add.
template <typename S>
struct CellAddr {
  const S* in;
  const S* ik;
  S* out;
  S* bout;
  long long sx, sy, sz;
  int wall;      // bit 2*ax: low wall along ax, bit 2*ax+1: high wall
  int ci, cj, ck;
};

// Address of the Eq. 6 ghost of a wall side for (cell, direction): I0 of the
// face (isothermal, or a refreshed diffuse value; a deviation from I0_b(T_ref)
// in the reduced modes), the side's per-direction ghost row (partially
// specular), or the cell's own value in the mirrored direction (specular).
// off: the direction's row offset d * nbo.
template <int AX, typename S>
__device__ __forceinline__ const void* wall_ghost_src(const SweepArgs& a, const DevGeom* gp, const CellAddr<S>& c,
                                                      const int4 di, bool from_low, int b0, long long off) {
  const int nbp = a.th.nbo;
  const int side = 2 * AX + (from_low ? 0 : 1);
  const int bc = gp->bc[side];
  if (bc == 0 || bc == 3) {  // wall data stay in memory (L1): only wall cells get here
    const long long fl = AX == 0 ? c.cj + (long long)gp->ny * c.ck
                                 : (AX == 1 ? c.ci + (long long)gp->nx * c.ck : c.ci + (long long)gp->nx * c.cj);
    if (bc == 3) return reinterpret_cast<const S*>(gp->gdir[side]) + fl * ((long long)a.nd * nbp) + off + b0;
    const long long f = gp->face0[side] + fl;
    if constexpr (sizeof(S) == 8) return a.I0wall + f * nbp + b0;
    else return a.I0wall_dev + f * nbp + b0;
  }
  const int r = AX == 0 ? di.y : (AX == 1 ? di.z : di.w);
  return c.ik + (long long)r * nbp;
}

// Address of the upwind value along axis AX for direction row offset `off`.
template <int AX, typename S>
__device__ __forceinline__ const void* upwind_src(const SweepArgs& a, const DevGeom* gp, const CellAddr<S>& c,
                                                  const int4 di, long long off, int b0) {
  const bool from_low = (di.x >> AX) & 1;
  const int wbit = 2 * AX + (from_low ? 0 : 1);
  if (!((c.wall >> wbit) & 1)) {
    const long long st = AX == 0 ? c.sx : (AX == 1 ? c.sy : c.sz);
    return c.ik + (from_low ? -st : st) + off;
  }
  return wall_ghost_src<AX, S>(a, gp, c, di, from_low, b0, off);
}

// Asynchronous global -> shared copy of one lane vector (16 or 8 bytes), L2 only.
template <int BYTES>
__device__ __forceinline__ void cp_async(unsigned smem, const void* g) {
  if constexpr (BYTES == 16) asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem), "l"(g) : "memory");
  else asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Operand vector of this lane from the staging ring.
template <typename S>
__device__ __forceinline__ void ld_stage(const char* p, typename Tr<S>::A (&x)[Tr<S>::V]) {
  Tr<S>::ld(reinterpret_cast<const S*>(p), x);
}

// Shared per-direction table of the current cell-size class.
struct DirSm {
  int4 info;     // up flags, rx, ry, rz
  float4 c;      // reduced modes: c_ax = |S_d,ax| / (w_d Delta_ax)
  double w;      // w_d
  float w32;     // w_d rounded to float
  float wlo;     // w_d - w32 rounded to float (the ff form of w_d)
};

// Staging ring: per thread and stage, 16 bytes per operand.  Operands: I^n (or
// B), the upwind value per axis, and in FP64 mode the coefficients A_x, A_y
// (, A_z), A_s (A_n, needed once per step, is loaded directly).  FP64 3-D keeps
// 3 stages so that two CTAs of 224 threads still fit an SM's shared memory.
template <int DIM, typename S>
struct Ring {
  static constexpr bool kCoef = sizeof(S) == 8;
  static constexpr int kOps = 1 + DIM + (kCoef ? DIM + 1 : 0);
  static constexpr int kStages = (kCoef && DIM == 3) ? 3 : 4;
};

// Lane coordinates of a sweep CTA and the shared regions of its item epilogue.
struct ItemCtx {
  int team, cpb, slot, dg, lane, lpc, dstep, b0, wid, wl, nwarps, nbp, nbp_all, band0, nbr;
  double* gsm;  // [blockDim.x][V] per-lane band partials
  double* red;  // [cpb * lpc][2] per-band-vector E_L, E_p sums (may lie inside gsm)
  double* cst;  // [cpb][4] per-cell scratch (apart from gsm)
};

// The end of an item of a sweep CTA (every thread calls it; it holds four CTA
// barriers): G[v] is this lane's partial G_b = sum_d w_d I_{d,b} over its
// directions (in the reduced modes without the W I0_b(T_ref) term of their
// deviation storage, which is added here).
// Root nearest 0 of F + F1 d + F2 d^2 / 2, the step of the cell's cached
// temperature model: an FP32 estimate from the stable form
// -2F / (F1 + sqrt(F1^2 - 2 F F2)) (-F / F1 without a real root), then one
// Newton step in FP64 with the FP32 reciprocal of the derivative.  The
// estimate is good to about 1e-7 and the step to about 1e-14 of d (the FP32
// rounding squared), while an accepted d is below 3e-5 T.  The FP64 pipe of
// GB300 takes about 76 cycles per warp instruction: this form issues five
// FP64 operations where a square root and a division take twenty-odd, and its
// conversions run on the integer pipe (bte_ff.cuh).
__device__ __forceinline__ double model_step(double F, double F1, double F2) {
  float f, f1, f2, lo;
  ff::split(F, f, lo);
  ff::split(F1, f1, lo);
  ff::split(F2, f2, lo);
  const float disc = fmaf(f1, f1, -2.0f * f * f2);
  const float d0f = (disc >= 0.0f && f1 > 0.0f) ? -2.0f * f / (f1 + sqrtf(disc)) : -f / f1;
  const double d0 = ff::to_double(d0f, 0.0f);
  const double q = fma(fma(0.5 * F2, d0, F1), d0, F);
  float qp;
  ff::split(fma(F2, d0, F1), qp, lo);
  const double r = ff::to_double(1.0f / qp, 0.0f);
  return fma(-q, r, d0);
}

template <int V, bool kDev>
__device__ __forceinline__ void item_epilogue(const SweepArgs& a, const ItemCtx& x, const WorkItem& wi,
                                              const DevGeom* gp, const double (&G)[V], unsigned long long& cnt_solves,
                                              unsigned long long& cnt_bad) {
  // ---- per-cell reduction.  The lanes of a cell hold band partials over their
  // direction subsets; the band owners (dg == 0) add them in a fixed order to
  // G_b, then E_L = sum_b G_b / v_b and E_p = sum_b beta_b G_b / v_b per band
  // vector.  One warp per cell adds the band vectors (shuffle tree); one warp
  // then solves every cell's model (lanes over cells), and all threads refresh
  // the accepted cells' I0.  Five barriers per item: every read of gsm
  // precedes the second (so the band-vector sums may overwrite it), every
  // read of red the fourth, and every read of the per-cell scratch the next
  // item's first.
  double* gb = x.gsm;
  double* rb = x.red;
#pragma unroll
  for (int v = 0; v < V; ++v) gb[(size_t)threadIdx.x * V + v] = G[v];
  __syncthreads();
  double eL = 0.0, ep = 0.0;
  if (x.dg == 0) {
#pragma unroll
    for (int v = 0; v < V; ++v) {
      double Gb = kDev ? a.Wtot * a.I0ref[x.b0 + v] : 0.0;
      for (int q = 0; q < x.dstep; ++q) Gb += gb[(size_t)(x.slot * x.team + q * x.lpc + x.lane) * V + v];
      const double e = Gb * a.th.inv_v[x.b0 + v];
      eL += e;
      ep = fma(a.th.beta[x.b0 + v], e, ep);
    }
  }
  __syncthreads();
  if (x.dg == 0) {
    double* r2 = rb + 2 * (size_t)(x.slot * x.lpc + x.lane);
    r2[0] = eL;
    r2[1] = ep;
  }
  __syncthreads();
  double* cst = x.cst;  // [cpb][4]: E_L, E_p, model step, accepted
  for (int cs = x.wid; x.wid < x.nwarps && cs < wi.cell_count; cs += x.nwarps) {  // warp per cell: E_L, E_p
    double EL = 0.0, Ep = 0.0;
    for (int l = x.wl; l < x.lpc; l += 32) {
      const double* r2 = rb + 2 * (size_t)(cs * x.lpc + l);
      EL += r2[0];
      Ep += r2[1];
    }
    for (int o = 16; o > 0; o >>= 1) {
      EL += __shfl_xor_sync(0xffffffffu, EL, o);
      Ep += __shfl_xor_sync(0xffffffffu, Ep, o);
    }
    if (x.wl == 0) {
      cst[4 * cs] = EL;
      cst[4 * cs + 1] = Ep;
    }
  }
  __syncthreads();
  // The cells' scalar steps with lanes over cells: one warp instruction serves
  // every cell of the item (a warp per cell would spend a whole warp's FP64
  // issue slots on each cell's square root and divisions).
  if (x.wid == 0) {
    for (int cs = x.wl; cs < wi.cell_count; cs += 32) {
      const long long Pc = gp->cell0 + wi.cell_begin + cs;
      const double EL = cst[4 * cs], Ep = cst[4 * cs + 1];
      double accepted = 0.0;
      if (a.partial) {  // band-range handle: partial sums for the caller's all-reduce
        if (!a.dry) {
          a.Epart[2 * Pc] = EL;
          a.Epart[2 * Pc + 1] = Ep;
        }
      } else {
        if (!a.dry) a.EL[Pc] = EL;
        if (!isfinite(EL) || !isfinite(Ep)) {
          atomicAdd(&cnt_bad, 1ULL);
        } else if (a.solve_tp) {
          atomicAdd(&cnt_solves, 1ULL);
          // root of (F - E_p) + F1 d + F2 d^2 / 2 nearest 0; F, F1, F2: the model's
          // sums sum_b a_p,b J_k,b, kept with J
          const double Fs = a.Msum[3 * Pc] - Ep, F1s = a.Msum[3 * Pc + 1], F2s = a.Msum[3 * Pc + 2];
          const double Te = a.Teval[Pc];
          const double delta = model_step(Fs, F1s, F2s);
          const double Tn = Te + delta;
          if (isfinite(Tn) && fabs(delta) <= a.trust_rel * Tn) {
            if (!a.dry) {
              a.Tp[Pc] = Tn;
              cst[4 * cs + 2] = delta;
              accepted = 1.0;
            }
          } else if (!a.dry) {  // exact quadrature needed: hand the cell to the fix-up kernel
            const unsigned k = atomicAdd(a.fix_count, 1u);
            FixItem fi;
            fi.P = Pc;
            fi.Ep = Ep;
            fi.model = (isfinite(Tn) && Tn >= kTmin && Tn <= kTmax) ? 1 : 0;
            fi.T0 = fi.model ? Tn : a.Tp[Pc];
            fi.pad = 0;
            a.fix[k] = fi;
          }
        }
      }
      cst[4 * cs + 3] = accepted;
    }
  }
  __syncthreads();
  // I0 refresh of every band of the accepted cells from their models: threads
  // over (cell, band).  Every read of cst precedes the next item's second barrier.
  for (int e = threadIdx.x; e < wi.cell_count * x.nbp; e += blockDim.x) {
    const int cs = e / x.nbp, b = e - cs * x.nbp;
    if (cst[4 * cs + 3] == 0.0) continue;
    const long long Pc = gp->cell0 + wi.cell_begin + cs;
    const double delta = cst[4 * cs + 2], hd2 = 0.5 * delta * delta;
    const long long j = (Pc * 3) * x.nbp_all + x.band0 + b;
    a.I0cell[Pc * x.nbp + b] = b < x.nbr ? fma(a.J[j + 2 * x.nbp_all], hd2, fma(a.J[j + x.nbp_all], delta, a.J[j])) : 0.0;
  }
  }

// BM (FP64 implicit only): 0 plain; 1 also stores B = A_n I^n; 2 the In operand
// holds B, so the update is B + A_x I_x + A_y I_y (+ A_z I_z) + A_s I0 (bitwise
// the same value, one FP64 multiply fewer per update).
// TT (FP64 only): the relaxation rates depend on T (beta_exp != 0); the
// reduced modes scale beta per cell outside the step loop and need no variant.
// (The FP64 update in double-float arithmetic is sweep_ff_kernel, bte_sweep_ff.cuh.)
template <int DIM, typename S, int MINB, int BM, bool TT>
__global__ void __launch_bounds__(256, MINB) sweep_kernel(SweepArgs a) {
  using T = Tr<S>;
  using A = typename T::A;
  constexpr int V = T::V;
  constexpr bool kDev = sizeof(S) != 8;  // reduced modes store deviations
  extern __shared__ double sm[];
  __shared__ unsigned long long cnt_solves, cnt_bad;
  __shared__ int cur_cls;
  const int lpc = a.lpc, nd = a.nd, nbp = a.th.nbo, dstep = a.dteam;
  const int nbp_all = a.th.nbp, band0 = a.th.band0, nbr = a.th.nbr;
  const int team = lpc * dstep;                       // lanes per cell
  const int cpb = blockDim.x / team;
  const int slot = threadIdx.x / team, tl = threadIdx.x - slot * team;
  const int dg = tl / lpc, lane = tl - dg * lpc;      // direction offset in a step, band vector
  DirSm* dsm = reinterpret_cast<DirSm*>(sm);          // [nd]
  double* gsm = sm + (sizeof(DirSm) / 8) * nd;        // [blockDim.x][V] per-lane band partials
  double* red = gsm + (size_t)V * blockDim.x;         // [cpb * lpc][2] per-band-vector E_L, E_p sums,
                                                      // then [cpb][4] per-cell scratch
  // staging ring of the far operands: [kStages][kOps][blockDim.x] x 16 bytes
  char* ring = reinterpret_cast<char*>(
      (reinterpret_cast<uintptr_t>(red + 2 * (size_t)cpb * lpc + 4 * (size_t)cpb) + 15) & ~static_cast<uintptr_t>(15));
  const S* __restrict__ In = reinterpret_cast<const S*>(a.In);
  const S* __restrict__ Ik = reinterpret_cast<const S*>(a.Ik);
  S* __restrict__ Io = reinterpret_cast<S*>(a.Iout);
  const A* __restrict__ coef = reinterpret_cast<const A*>(a.coef);
  const long long row = (long long)nd * nbp;
  const int b0 = V * lane;
  if (threadIdx.x == 0) { cnt_solves = 0; cnt_bad = 0; cur_cls = -1; }
  const int wid = threadIdx.x >> 5, wl = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;  // full warps (a trailing partial warp takes no cell)
  A vb[V], bb[V];  // per-lane band constants (reduced modes)
#pragma unroll
  for (int v = 0; v < V; ++v) {
    vb[v] = kDev ? (A)a.vb32[b0 + v] : (A)0;
    bb[v] = kDev ? (A)a.bb32[b0 + v] : (A)0;
  }
  // reduced modes: the scheme (BM 3: explicit, BM 0: implicit) and its scalars
  // in both halves of a packed pair
  constexpr bool kExpl = kDev && BM == 3;
  const ff::x2 dt2 = ff::pack(a.dt32, a.dt32), ndt2 = ff::pack(-a.dt32, -a.dt32), rdt2 = ff::pack(a.rdt32, a.rdt32),
               one2 = ff::pack(1.0f, 1.0f);
  __syncthreads();

  for (int item = blockIdx.x; item < a.nitems; item += gridDim.x) {
    const WorkItem wi = a.items[item];
    const DevGeom* gp = a.geoms + wi.geom;
    const int gnx = gp->nx, gny = gp->ny, gcls = gp->cls;
    const int gnz = DIM == 3 ? gp->nz : 1;
    if (gcls != cur_cls) {  // (block-uniform) direction table of this cell-size class
      __syncthreads();
      for (int d = threadIdx.x; d < nd; d += blockDim.x) {
        const DirInfo di = a.dirs[d];
        DirSm e;
        e.info = make_int4(di.up, di.rx, di.ry, di.rz);
        e.c = kDev ? a.dirc[(size_t)gcls * nd + d] : make_float4(0.f, 0.f, 0.f, 0.f);
        e.w = a.wdir[d];
        e.w32 = a.wdir32[d];
        e.wlo = (float)(e.w - (double)e.w32);
        dsm[d] = e;
      }
      if (threadIdx.x == 0) cur_cls = gcls;
      __syncthreads();
    }
    const bool active = slot < wi.cell_count;
    const int lc = wi.cell_begin + (active ? slot : 0);
    const int ci = lc % gnx, cj = (lc / gnx) % gny, ck = lc / (gnx * gny);
    const long long P = gp->cell0 + lc;
    double G[V];
#pragma unroll
    for (int v = 0; v < V; ++v) G[v] = 0.0;

    if (active) {
      // temperature-dependent relaxation: beta_b(T_p) = beta_b s with
      // s = (T_p / T_ref)^p of this cell (s = 1 when tau does not depend on T)
      const bool tT = kDev ? a.beta_exp != 0.0 : TT;
      const double bsc = tT ? pow(a.Tp[P] / a.beta_Tref, a.beta_exp) : 1.0;
      if constexpr (kDev) {
        if (tT) {
#pragma unroll
          for (int v = 0; v < V; ++v) bb[v] = a.bb32[b0 + v] * (float)bsc;
        }
      }
      A src[V];  // FP64: I0 of the cell; reduced: beta_b(T_p) * (I0 - I0ref)
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const double i0 = a.I0cell[P * nbp + b0 + v];
        src[v] = kDev ? bb[v] * (A)(i0 - a.I0ref[b0 + v]) : (A)i0;
      }
      const size_t plane = (size_t)nd * nbp;
      const A* __restrict__ cf = coef + (size_t)gcls * 5 * plane + b0;
      CellAddr<S> c;
      c.in = In + P * row + b0;
      c.ik = Ik + P * row + b0;
      c.out = Io + P * row + b0;
      c.bout = BM == 1 ? reinterpret_cast<S*>(a.Bout) + P * row + b0 : nullptr;
      c.sx = row;
      c.sy = (long long)gnx * row;
      c.sz = (long long)gnx * gny * row;
      c.ci = ci; c.cj = cj; c.ck = ck;
      c.wall = (ci == 0) | ((ci == gnx - 1) << 1) | ((cj == 0) << 2) | ((cj == gny - 1) << 3) |
               (DIM == 3 ? ((ck == 0) << 4) | ((ck == gnz - 1) << 5) : 0);
      float acc[V];  // reduced modes: FP32 partial band sums, flushed to G periodically
#pragma unroll
      for (int v = 0; v < V; ++v) acc[v] = 0.f;
      int nacc = 0;
      // FP64 mode: G_b = sum_d w_d I_d.  Over a run of directions with the same
      // weight (one polar ring), each band sums I exactly in 64-bit fixed point
      // on the integer pipe: unit 2^(E - 50) for the cell's I0 of exponent E, so
      // a value up to 16 I0 adds at most 2^55 and a run of 256 cannot overflow;
      // the run then enters G with one FP64 FMA (sum x w x unit).  Values with a
      // larger exponent (or negative, NaN) take the FP64 FMA directly.  Terms
      // below 2^-10 units are dropped (at most 1/4 unit per run).
      unsigned long long facc[V];
      long long fsc[V];  // unit exponent shifted into a double's exponent field
      int fe0[V];        // largest exponent field summed in fixed point (-1: none)
      long long wrun = 0;
      int nrun = 0;
      if constexpr (!kDev) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const int e0 = (int)((unsigned long long)__double_as_longlong((double)src[v]) >> 52);  // src = I0 (>= 0)
          const bool on = e0 >= 200 && e0 <= 1900;
          facc[v] = 0ull;
          fe0[v] = on ? e0 + 4 : -1;
          fsc[v] = on ? (long long)(e0 - 1073) * (1LL << 52) : 0;
        }
      }
      // This lane's directions are d_j = dg + j*dstep.  Their operands (I^n and the
      // upwind I^k or wall ghost per axis) are copied global -> shared kStages-1
      // directions ahead with cp.async; each thread waits only for its own copies.
      constexpr int kOps = Ring<DIM, S>::kOps;
      constexpr int kStages = Ring<DIM, S>::kStages;
      constexpr int kVB = V * (int)sizeof(S);
      const int nsteps = dg < nd ? (nd - dg + dstep - 1) / dstep : 0;
      // ring slot (stage st, operand op) of this thread: 32-bit shared addresses
      const unsigned rb0 = (unsigned)__cvta_generic_to_shared(ring) + threadIdx.x * 16u;
      const unsigned ostr = blockDim.x * 16u, sstr = kOps * ostr;
      const long long sx = c.sx, sy = c.sy, sz = c.sz;
      // BF16: the step loop is compiled twice, for interior cells (no wall
      // logic at all) and for wall cells (per-axis Eq. 6 ghosts; isothermal
      // ghosts are read at use).  The other modes run one loop with a per-step
      // interior test (a second copy measured slower there).
      auto run = [&](auto interior_tag) {
      constexpr bool kInterior = decltype(interior_tag)::value;
      // stage the operands of step j into the ring slot at shared address sb
      auto issue = [&](auto checked, int j, const unsigned sb) {
        if (!decltype(checked)::value || j < nsteps) {
          const int d = dg + j * dstep;
          const int off = d * nbp;
          cp_async<kVB>(sb, c.in + off);
          if (kInterior || c.wall == 0) {  // interior cell: the upwind rows are the neighbours' (the common case)
            const int up = dsm[d].info.x;
            cp_async<kVB>(sb + ostr, c.ik + off + ((up & 1) ? -sx : sx));
            cp_async<kVB>(sb + 2 * ostr, c.ik + off + ((up & 2) ? -sy : sy));
            if (DIM == 3) cp_async<kVB>(sb + 3 * ostr, c.ik + off + ((up & 4) ? -sz : sz));
          } else {
            const int4 di = dsm[d].info;
#pragma unroll
            for (int ax = 0; ax < DIM; ++ax) {
              const void* src_p = ax == 0 ? upwind_src<0, S>(a, gp, c, di, off, b0)
                                : (ax == 1 ? upwind_src<1, S>(a, gp, c, di, off, b0) : upwind_src<2, S>(a, gp, c, di, off, b0));
              const bool iso_ghost = (sizeof(S) == 2) && ((c.wall >> (2 * ax + (((di.x >> ax) & 1) ? 0 : 1))) & 1) &&
                                     gp->bc[2 * ax + (((di.x >> ax) & 1) ? 0 : 1)] == 0;
              if (!iso_ghost) cp_async<kVB>(sb + (1 + ax) * ostr, src_p);  // BF16 iso ghosts: read at use
            }
          }
          if constexpr (Ring<DIM, S>::kCoef) {  // A_x, A_y (, A_z), A_s of this direction
#pragma unroll
            for (int k = 0; k < DIM; ++k) cp_async<16>(sb + (1 + DIM + k) * ostr, cf + (size_t)(1 + k) * plane + off);
            cp_async<16>(sb + (1 + 2 * DIM) * ostr, cf + 4 * plane + off);
          }
        }
        cp_async_commit();
      };
      // Upwind operand of axis ax from its slot.  A BF16 cell on an isothermal
      // wall reads that wall's FP32 ghost deviations (8 floats, cached wall data)
      // straight from memory instead.
      auto read_up = [&](unsigned sb, int ax, const int4 di, const int off, A (&x)[V]) {
        if constexpr (sizeof(S) == 2) {
          if constexpr (!kInterior) {
            const bool lowside = (di.x >> ax) & 1;
            const int side = 2 * ax + (lowside ? 0 : 1);
            if (((c.wall >> side) & 1) && gp->bc[side] == 0) {
              const void* g = ax == 0 ? upwind_src<0, S>(a, gp, c, di, off, b0)
                            : (ax == 1 ? upwind_src<1, S>(a, gp, c, di, off, b0) : upwind_src<2, S>(a, gp, c, di, off, b0));
              ldgv<float, V>(reinterpret_cast<const float*>(g), x);
              return;
            }
          }
        }
        T::lds(sb + (1 + ax) * ostr, x);
      };
#pragma unroll
      for (int j = 0; j < kStages - 1; ++j) issue(std::true_type{}, j, rb0 + (unsigned)j * sstr);
      auto step = [&](int j, const unsigned sb) {
        cp_async_wait<kStages - 1>();
        const int d = dg + j * dstep;
        const int off = d * nbp;
        const int4 di = dsm[d].info;
        A vn[V], ux[V], uy[V], uz[V];
        T::lds(sb, vn);
        read_up(sb, 0, di, off, ux);
        read_up(sb, 1, di, off, uy);
        if (DIM == 3) read_up(sb, 2, di, off, uz);
        A r[V];
        if constexpr (!kDev) {
          A Ax[V], Ay[V], As[V];
          Tr<double>::lds(sb + (1 + DIM) * ostr, Ax);
          Tr<double>::lds(sb + (2 + DIM) * ostr, Ay);
          Tr<double>::lds(sb + (1 + 2 * DIM) * ostr, As);
          if constexpr (BM == 2) {
#pragma unroll
            for (int v = 0; v < V; ++v) r[v] = vn[v];
          } else {
            A An[V];
            ldgv<A, V>(cf + off, An);
#pragma unroll
            for (int v = 0; v < V; ++v) r[v] = An[v] * vn[v];
            if constexpr (BM == 1) T::st(c.bout + off, r);
          }
#pragma unroll
          for (int v = 0; v < V; ++v) {
            r[v] = fma(Ax[v], ux[v], r[v]);
            r[v] = fma(Ay[v], uy[v], r[v]);
          }
          if (DIM == 3) {
            A Az[V];
            Tr<double>::lds(sb + (3 + DIM) * ostr, Az);
#pragma unroll
            for (int v = 0; v < V; ++v) r[v] = fma(Az[v], uz[v], r[v]);
          }
          if constexpr (!TT) {
#pragma unroll
            for (int v = 0; v < V; ++v) r[v] = fma(As[v], src[v], r[v]);
          } else if (a.explicit_scheme) {  // A_n -> A_n + (1 - s) A_s, A_s -> s A_s
#pragma unroll
            for (int v = 0; v < V; ++v) r[v] = fma((1.0 - bsc) * As[v], vn[v], fma(bsc * As[v], src[v], r[v]));
          } else {  // every coefficient x 1/(1 + (s - 1) A_s), A_s also x s
#pragma unroll
            for (int v = 0; v < V; ++v)
              r[v] = fma(bsc * As[v], src[v], r[v]) * __drcp_rn(fma(bsc - 1.0, As[v], 1.0));
          }
          T::st(c.out + off, r);
          const double wd = dsm[d].w;
          const long long wb = __double_as_longlong(wd);
          if (wb != wrun || nrun == 256) {  // close the run: sum x (w x unit)
#pragma unroll
            for (int v = 0; v < V; ++v) {
              if (facc[v] != 0ull) G[v] = fma(__ull2double_rn(facc[v]), __longlong_as_double(wrun + fsc[v]), G[v]);
              facc[v] = 0ull;
            }
            wrun = wb;
            nrun = 0;
          }
          ++nrun;
          bool big = false;
#pragma unroll
          for (int v = 0; v < V; ++v) {
            const unsigned long long rb = (unsigned long long)__double_as_longlong((double)r[v]);
            const int e = (int)(rb >> 52);
            const unsigned long long m = ((rb & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull) << 2;
            const int sh = e == 0 ? 63 : min(fe0[v] - e, 63);  // zero (and subnormal) adds nothing
            facc[v] += sh >= 0 ? (m >> sh) : 0ull;
            big |= sh < 0;
          }
          if (__any_sync(__activemask(), big)) {  // rare: a value beyond the fixed-point range
#pragma unroll
            for (int v = 0; v < V; ++v) {
              const int e = (int)((unsigned long long)__double_as_longlong((double)r[v]) >> 52);
              if (e != 0 && fe0[v] - e < 0) G[v] = fma(wd, (double)r[v], G[v]);
            }
          }
        } else {
          // P and Q from v_b, beta_b and sum_ax c_ax (no table loads):
          // implicit Q = 1/(1/dt + beta_b + v_b sum c), P = Q/dt; explicit P = 1 - dt(beta_b + v_b sum c), Q = dt.
          // Two bands per packed f32x2 instruction (each half rounds as the
          // scalar instruction would: the same values as band by band).
          const float4 cc = dsm[d].c;
          const ff::x2 ccw = ff::pack(cc.w, cc.w), ccx = ff::pack(cc.x, cc.x), ccy = ff::pack(cc.y, cc.y),
                       ccz = ff::pack(cc.z, cc.z);
#pragma unroll
          for (int q = 0; q < V / 2; ++q) {
            const int v = 2 * q;
            const ff::x2 vb2 = ff::pack(vb[v], vb[v + 1]);
            const ff::x2 rate = ff::fma(vb2, ccw, ff::pack(bb[v], bb[v + 1]));
            ff::x2 Pc, Qc;
            if constexpr (kExpl) {
              Qc = dt2;
              Pc = ff::fma(ndt2, rate, one2);
            } else {
              const ff::x2 den = ff::add(rdt2, rate);
              float q0, q1;
              asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(q0) : "f"(ff::lo_of(den)));
              asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(q1) : "f"(ff::hi_of(den)));
              Qc = ff::pack(q0, q1);
              Pc = ff::mul(Qc, rdt2);
            }
            ff::x2 f = ff::mul(ccx, ff::pack(ux[v], ux[v + 1]));
            f = ff::fma(ccy, ff::pack(uy[v], uy[v + 1]), f);
            if (DIM == 3) f = ff::fma(ccz, ff::pack(uz[v], uz[v + 1]), f);
            const ff::x2 t = ff::fma(vb2, f, ff::pack(src[v], src[v + 1]));
            const ff::x2 rr = ff::fma(Qc, t, ff::mul(Pc, ff::pack(vn[v], vn[v + 1])));
            r[v] = ff::lo_of(rr);
            r[v + 1] = ff::hi_of(rr);
          }
          if constexpr (sizeof(S) == 2) {
            // store the rounded values and sum exactly what was stored
            const uint4 w = make_uint4(T::pack2(r[0], r[1]), T::pack2(r[2], r[3]), T::pack2(r[4], r[5]), T::pack2(r[6], r[7]));
            __stcs(reinterpret_cast<uint4*>(c.out + off), w);
            T::unpack(w, r);
          } else {
            T::st(c.out + off, r);
          }
          const float wd = dsm[d].w32;
          const ff::x2 wd2 = ff::pack(wd, wd);
#pragma unroll
          for (int q = 0; q < V / 2; ++q) {
            const ff::x2 a2 = ff::fma(wd2, ff::pack(r[2 * q], r[2 * q + 1]), ff::pack(acc[2 * q], acc[2 * q + 1]));
            acc[2 * q] = ff::lo_of(a2);
            acc[2 * q + 1] = ff::hi_of(a2);
          }
          // FP32 partials go to FP64 every 16 directions (every 64 for BF16 storage,
          // whose 2^-8 rounding dwarfs the float sum's)
          if (++nacc == (sizeof(S) == 2 ? 64 : 16)) {
#pragma unroll
            for (int v = 0; v < V; ++v) { G[v] += (double)acc[v]; acc[v] = 0.f; }
            nacc = 0;
          }
        }
      };
      // Every step but the last kStages - 1 stages a later direction (no bounds
      // test), step j + kStages - 1 into the slot step j - 1 has just read; the
      // last steps commit an empty group, so that the wait still finds its own.
      const int nmain = nsteps - (kStages - 1);
      const unsigned slast = rb0 + (unsigned)(kStages - 1) * sstr;
      unsigned sb = rb0, sprev = slast;
      int j = 0;
      for (; j < nmain; ++j) {
        issue(std::false_type{}, j + kStages - 1, sprev);
        step(j, sb);
        sprev = sb;
        sb = sb == slast ? rb0 : sb + sstr;
      }
      for (; j < nsteps; ++j) {
        cp_async_commit();
        step(j, sb);
        sb = sb == slast ? rb0 : sb + sstr;
      }
      };
      if constexpr (sizeof(S) == 2) {
        if (c.wall == 0) run(std::true_type{});
        else run(std::false_type{});
      } else {
        run(std::false_type{});
      }
      cp_async_wait<0>();
      if constexpr (kDev) {
#pragma unroll
        for (int v = 0; v < V; ++v) G[v] += (double)acc[v];
      } else {
#pragma unroll
        for (int v = 0; v < V; ++v)
          if (facc[v] != 0ull) G[v] = fma(__ull2double_rn(facc[v]), __longlong_as_double(wrun + fsc[v]), G[v]);
      }
    }

    item_epilogue<V, kDev>(a, ItemCtx{team, cpb, slot, dg, lane, lpc, dstep, b0, wid, wl, nwarps, nbp, nbp_all, band0,
                                      nbr, gsm, red, red + 2 * (size_t)cpb * lpc},
                           wi, gp, G, cnt_solves, cnt_bad);
  }
  __syncthreads();
  if (threadIdx.x == 0 && a.counters) {
    if (cnt_solves) atomicAdd(&a.counters->solves, cnt_solves);
    if (cnt_bad) atomicAdd(&a.counters->nonfinite, cnt_bad);
  }
}

template <typename S, int MINB, int BM, bool TT>
cudaError_t launch_minb(const SweepArgs& a, int dim, int threads, int grid, cudaStream_t s) {
  const int team = a.lpc * a.dteam, cpb = threads / team;
  const size_t smem = sizeof(DirSm) * (size_t)a.nd + (size_t)Tr<S>::V * threads * sizeof(double) +
                      (2 * (size_t)cpb * a.lpc + 4 * (size_t)cpb) * sizeof(double) + 16 +
                      (size_t)(dim == 3 ? Ring<3, S>::kStages * Ring<3, S>::kOps : Ring<2, S>::kStages * Ring<2, S>::kOps) *
                          threads * 16;
  if (dim == 3) {
    const cudaError_t e = raise_dynamic_smem((const void*)sweep_kernel<3, S, MINB, BM, TT>, smem);
    if (e != cudaSuccess) return e;
    sweep_kernel<3, S, MINB, BM, TT><<<grid, threads, smem, s>>>(a);
  } else {
    const cudaError_t e = raise_dynamic_smem((const void*)sweep_kernel<2, S, MINB, BM, TT>, smem);
    if (e != cudaSuccess) return e;
    sweep_kernel<2, S, MINB, BM, TT><<<grid, threads, smem, s>>>(a);
  }
  return cudaGetLastError();
}

// variant: 1 -> at least 2 resident CTAs per SM (<= 128 registers), 2 -> 3 CTAs (<= 80 registers)
template <typename S, int BM, bool TT>
cudaError_t launch_bm(int variant, const SweepArgs& a, int dim, int threads, int grid, cudaStream_t s) {
  if (variant >= 2) return launch_minb<S, 3, BM, TT>(a, dim, threads, grid, s);
  return launch_minb<S, 2, BM, TT>(a, dim, threads, grid, s);
}

template <typename S>
cudaError_t launch(int variant, const SweepArgs& a, int dim, int threads, int grid, cudaStream_t s) {
  if constexpr (sizeof(S) == 8) {
    if (a.ff != 0) return cudaErrorInvalidValue;  // the double-float variants are sweep_ff_kernel's
    if (a.beta_exp != 0.0) {
      if (a.bmode == 1) return launch_bm<S, 1, true>(variant, a, dim, threads, grid, s);
      if (a.bmode == 2) return launch_bm<S, 2, true>(variant, a, dim, threads, grid, s);
      return launch_bm<S, 0, true>(variant, a, dim, threads, grid, s);
    }
    if (a.bmode == 1) return launch_bm<S, 1, false>(variant, a, dim, threads, grid, s);
    if (a.bmode == 2) return launch_bm<S, 2, false>(variant, a, dim, threads, grid, s);
  } else {
    if (a.bmode != 0 || a.ff != 0) return cudaErrorInvalidValue;  // the B form exists for FP64 storage only
    if (a.explicit_scheme) return launch_bm<S, 3, false>(variant, a, dim, threads, grid, s);
  }
  return launch_bm<S, 0, false>(variant, a, dim, threads, grid, s);
}

}  // namespace sweep
}  // namespace bte

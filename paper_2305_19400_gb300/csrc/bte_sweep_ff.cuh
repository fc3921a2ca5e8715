// bte_sweep_ff.cuh -- the FP64-mode Jacobi sweep in double-float arithmetic
// with factored coefficients (sm_103a).
//
// The implicit point-Jacobi update of Sec. 3.1 (Eq. 5 with backward Euler),
//   I^{k+1} = (I^n/dt + v_b sum_ax c_ax,d I_up,ax^k + beta_b I0_b^k) / (1/dt + beta_b + v_b sum_ax c_ax,d),
//   c_ax,d = |S_d,ax| / (w_d Delta_ax),
// is divided through by v_b (> 0 on every real band) and evaluated as
//   B + R (sum_ax c_ax u_ax + (beta_b / v_b) I0),  R = 1 / (1/(v_b dt) + beta_b/v_b + sum_ax c_ax,d),
// with B = (1/(v_b dt)) R I^n kept across the inner iterations of a step (BM 1
// forms and stores B, BM 2 reads it, BM 0, a step of one inner iteration,
// forms it only), in double-float arithmetic on the FP32 pipe (bte_ff.cuh):
// c_ax per direction sits in a shared table, 1/(v_b dt) and beta_b/v_b of the
// lane's two bands and (beta_b/v_b) I0_b per cell in registers, and only R per
// (direction, band) is read per step: three products and three pair sums per
// update in 2-D.  A step therefore stages four 16-byte operands (B or I^n, the
// upwind value per axis in 2-D, R) instead of the six of the five-coefficient
// form.  Shared memory per CTA is the direction table (19.2 KB for 400
// directions in 2-D, 48 bytes a direction), a 5-stage ring (35 KB) and the
// epilogue's scratch: 58 KB with the driver's reserve for a 112-thread CTA
// in 2-D, four of which share an SM, as many as its registers allow.  The tables come from the host in double-float form
// with R chosen so that R (1/(v_b dt) + beta_b/v_b + sum c_ax) = 1 holds for
// the table values to double-double accuracy, which keeps a uniform
// equilibrium in place.
//
// Work layout, staging, walls, direction sums and the item epilogue are those
// of sweep_kernel (bte_sweep.cuh); FF has the meaning described there.
#pragma once
#include <type_traits>

#include "bte_ff.cuh"
#include "bte_sweep.cuh"

namespace bte {
namespace sweep_ff {

using sweep::CellAddr;
using sweep::cp_async;
using sweep::cp_async_commit;
using sweep::cp_async_wait;
using sweep::ItemCtx;

// Shared per-direction table of the current cell-size class (16 + 16 DIM
// bytes): the coefficients already packed for the two-band operations.
template <int DIM>
struct DirFF {
  int up;          // bit a set: the upwind neighbour lies on the low side along axis a
  unsigned wkey;   // bits of w32 ^ bits of wlo: equal weights, equal keys (the runs of the direction sums)
  float w32, wlo;  // w_d as a double-float pair
  ff::x2 ch[DIM];  // c_ax,d high part in both halves, for the axes in use
  ff::x2 cl[DIM];  // c_ax,d low part in both halves
};

// L2 cache policies of the staged copies: the R table (one row per
// direction and band, read by every item of the launch) is kept
// (evict_last); B or I^n, read once per launch, leaves first (evict_first).
// The upwind rows of I^k, read again by the neighbouring cells, keep the
// default policy.
__device__ __forceinline__ unsigned long long l2_evict_last() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ unsigned long long l2_evict_first() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void cp_async_l2(unsigned smem, const void* g, unsigned long long policy) {
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(smem), "l"(g), "l"(policy)
               : "memory");
}

// Ring depth: 5 stages in 2-D and 4 in 3-D under the two-CTA register cap
// (four 112-thread CTAs of 58 KB share an SM in 2-D), 3 when three 224-thread
// CTAs share one.
template <int DIM, int MINB>
struct RingFF {
  static constexpr int kOps = 2 + DIM;  // B or I^n, upwind per axis, R
  static constexpr int kStages = MINB >= 3 ? 3 : (DIM == 2 ? 5 : 4);
};

// Threads per CTA the register cap is computed for: three resident CTAs are
// meant for the 224-thread CTAs of 55-56 bands (4 cells x 28 lanes x 2
// directions), which leaves up to 97 registers per thread.
template <int MINB>
struct MaxThreadsFF {
  static constexpr int value = MINB >= 3 ? 224 : 256;
};
// Registers per thread of MINB resident CTAs of MaxThreadsFF threads (multiples of 8).
template <int MINB>
struct MaxRegFF {
  static constexpr int value = (65536 / (MINB * MaxThreadsFF<MINB>::value)) / 8 * 8;
};

template <int DIM, int MINB, int BM, int FF>
__global__ void __launch_bounds__(MaxThreadsFF<MINB>::value) __maxnreg__(MaxRegFF<MINB>::value) sweep_ff_kernel(SweepArgs a) {
  static_assert(FF != 0, "double-float variants only");
  static_assert(BM != 2 || (FF & 1) != 0, "B is an ff pair");
  constexpr int V = 2;
  constexpr int kOps = RingFF<DIM, MINB>::kOps;
  constexpr int kStages = RingFF<DIM, MINB>::kStages;
  extern __shared__ double sm[];
  __shared__ unsigned long long cnt_solves, cnt_bad;
  __shared__ int cur_cls;
  const int lpc = a.lpc, nd = a.nd, nbp = a.th.nbo, dstep = a.dteam;
  const int nbp_all = a.th.nbp, band0 = a.th.band0, nbr = a.th.nbr;
  const int team = lpc * dstep;
  const int cpb = blockDim.x / team;
  const int slot = threadIdx.x / team, tl = threadIdx.x - slot * team;
  const int dg = tl / lpc, lane = tl - dg * lpc;
  DirFF<DIM>* dsm = reinterpret_cast<DirFF<DIM>*>(sm);
  double* gsm = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(dsm + nd) + 15) & ~static_cast<uintptr_t>(15));
  double* red = gsm;                            // the band-vector sums overwrite the read partials
  double* cst = gsm + (size_t)V * blockDim.x;   // [cpb][4] per-cell scratch
  char* ring = reinterpret_cast<char*>(
      (reinterpret_cast<uintptr_t>(cst + 4 * (size_t)cpb) + 15) & ~static_cast<uintptr_t>(15));
  const double* __restrict__ In = reinterpret_cast<const double*>(a.In);
  const double* __restrict__ Ik = reinterpret_cast<const double*>(a.Ik);
  double* __restrict__ Io = reinterpret_cast<double*>(a.Iout);
  const long long row = (long long)nd * nbp;
  const int b0 = V * lane;
  if (threadIdx.x == 0) { cnt_solves = 0; cnt_bad = 0; cur_cls = -1; }
  const int wid = threadIdx.x >> 5, wl = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  // 1/(v_b dt) and beta_b/v_b of the lane's two bands
  const ff::P2 rdtv2 = ff::ldg(a.band_ff + 2 * b0);
  const ff::P2 betav2 = ff::ldg(a.band_ff + 2 * (nbp + b0));
  __syncthreads();

  for (int item = blockIdx.x; item < a.nitems; item += gridDim.x) {
    const WorkItem wi = a.items[item];
    const DevGeom* gp = a.geoms + wi.geom;
    const int gnx = gp->nx, gny = gp->ny, gcls = gp->cls;
    const int gnz = DIM == 3 ? gp->nz : 1;
    if (gcls != cur_cls) {  // (block-uniform) direction table of this cell-size class
      __syncthreads();
      for (int d = threadIdx.x; d < nd; d += blockDim.x) {
        DirFF<DIM> e;
        e.up = a.dirs[d].up;
        e.w32 = a.wdir32[d];
        e.wlo = (float)(a.wdir[d] - (double)e.w32);
        e.wkey = __float_as_uint(e.w32) ^ __float_as_uint(e.wlo);
        const float* cc = a.dirc_ff + ((size_t)gcls * nd + d) * 6;
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
          e.ch[k] = ff::pack(cc[2 * k], cc[2 * k]);
          e.cl[k] = ff::pack(cc[2 * k + 1], cc[2 * k + 1]);
        }
        dsm[d] = e;
      }
      if (threadIdx.x == 0) cur_cls = gcls;
      __syncthreads();
    }
    const bool active = slot < wi.cell_count;
    const int lc = wi.cell_begin + (active ? slot : 0);
    const int ci = lc % gnx, cj = (lc / gnx) % gny, ck = lc / (gnx * gny);
    const long long P = gp->cell0 + lc;
    double G[V] = {0.0, 0.0};

    if (active) {
      // (beta_b / v_b) I0_b of the cell, constant over its directions
      const ff::P2 srcb =
          ff::norm(ff::mul(betav2, ff::from_doubles(a.I0cell[P * nbp + b0], a.I0cell[P * nbp + b0 + 1])));
      CellAddr<double> c;
      c.in = In + P * row + b0;
      c.ik = Ik + P * row + b0;
      c.out = Io + P * row + b0;
      c.bout = BM == 1 ? reinterpret_cast<double*>(a.Bout) + P * row + b0 : nullptr;
      c.sx = row;
      c.sy = (long long)gnx * row;
      c.sz = (long long)gnx * gny * row;
      c.ci = ci; c.cj = cj; c.ck = ck;
      c.wall = (ci == 0) | ((ci == gnx - 1) << 1) | ((cj == 0) << 2) | ((cj == gny - 1) << 3) |
               (DIM == 3 ? ((ck == 0) << 4) | ((ck == gnz - 1) << 5) : 0);
      const long long sx_ = c.sx, sy_ = c.sy, sz_ = c.sz;
      const double* __restrict__ Rrow = reinterpret_cast<const double*>(a.coef_R) + (size_t)gcls * row + b0;
      const int nsteps = dg < nd ? (nd - dg + dstep - 1) / dstep : 0;
      const unsigned rb0 = (unsigned)__cvta_generic_to_shared(ring) + threadIdx.x * 16u;
      const unsigned ostr = blockDim.x * 16u, sstr = kOps * ostr;
      const long long dst = (long long)dstep * nbp;  // elements from one step's row to the next
      // direction sums: per run of equal weights in ff, the runs into G in ff
      ff::P2 Sff = ff::zero(), Gff = ff::zero(), wff = ff::zero();
      unsigned wrun = 0xffffffffu;
      // The step loop, once for interior cells (every upwind row a neighbour's,
      // every operand an ff pair when FF & 1) and once for wall cells.
      auto run = [&](auto interior_tag) {
        constexpr bool kInt = decltype(interior_tag)::value;
        // issue side: the rows of step ji advance by dst elements per step
        const double* pin = c.in + (long long)dg * nbp;
        const double* pik = c.ik + (long long)dg * nbp;
        const double* pR = Rrow + (long long)dg * nbp;
        int ji = 0;
        const unsigned long long keep = l2_evict_last(), once = l2_evict_first();
        // stage the operands of step ji into the ring slot at shared address sbi
        auto issue = [&](auto checked, const unsigned sbi) {
          if (!decltype(checked)::value || ji < nsteps) {
            const int d = dg + ji * dstep;
            cp_async_l2(sbi, pin, once);
            if constexpr (kInt) {
              const int up = dsm[d].up;
              cp_async<16>(sbi + ostr, pik + ((up & 1) ? -sx_ : sx_));
              cp_async<16>(sbi + 2 * ostr, pik + ((up & 2) ? -sy_ : sy_));
              if (DIM == 3) cp_async<16>(sbi + 3 * ostr, pik + ((up & 4) ? -sz_ : sz_));
            } else {
              const DirInfo dinf = a.dirs[d];
              const int4 di = make_int4(dinf.up, dinf.rx, dinf.ry, dinf.rz);
              const int off = d * nbp;
              cp_async<16>(sbi + ostr, sweep::upwind_src<0, double>(a, gp, c, di, off, b0));
              cp_async<16>(sbi + 2 * ostr, sweep::upwind_src<1, double>(a, gp, c, di, off, b0));
              if (DIM == 3) cp_async<16>(sbi + 3 * ostr, sweep::upwind_src<2, double>(a, gp, c, di, off, b0));
            }
            cp_async_l2(sbi + (1 + DIM) * ostr, pR, keep);
            pin += dst;
            pik += dst;
            pR += dst;
          }
          cp_async_commit();
          ++ji;
        };
#pragma unroll
        for (int j = 0; j < kStages - 1; ++j) issue(std::true_type{}, rb0 + (unsigned)j * sstr);
        double* pout = c.out + (long long)dg * nbp;
        [[maybe_unused]] double* pbout = BM == 1 ? c.bout + (long long)dg * nbp : nullptr;  // BM 1 only
        unsigned sb = rb0;
        auto step = [&](int j) {
          cp_async_wait<kStages - 1>();
          const int d = dg + j * dstep;
          const DirFF<DIM>& e = dsm[d];
          // sum_ax c_ax u_ax; an upwind operand is an ff pair unless it is I^k in
          // doubles or an isothermal wall ghost (doubles in every variant)
          ff::P2 t;
#pragma unroll
          for (int ax = 0; ax < DIM; ++ax) {
            const unsigned ua = sb + (1 + ax) * ostr;
            ff::P2 u;
            if constexpr (kInt) {
              u = (FF & 1) ? ff::lds(ua) : ff::lds_doubles(ua);
            } else {
              const int side = 2 * ax + (((e.up >> ax) & 1) ? 0 : 1);
              const bool dbl = (FF & 1) == 0 || (((c.wall >> side) & 1) && gp->bc[side] == 0);
              u = dbl ? ff::lds_doubles(ua) : ff::lds(ua);
            }
            const ff::P2 pr = ff::mul(ff::P2{e.ch[ax], e.cl[ax]}, u);
            if (ax == 0) t = pr;
            else t = ff::add(t, pr);
          }
          const ff::P2 Rv = ff::lds(sb + (1 + DIM) * ostr);
          const ff::P2 p = ff::mul(Rv, ff::add(t, srcb));
          ff::P2 rf;
          if constexpr (BM == 2) {
            rf = ff::norm(ff::add(ff::lds(sb), p));
          } else {  // B = (R / (v_b dt)) I^n, kept for the later inner iterations when BM == 1
            const ff::P2 vin = (FF & 1) ? ff::lds(sb) : ff::lds_doubles(sb);
            const ff::P2 B = ff::norm(ff::mul(rdtv2, ff::mul(Rv, vin)));
            if constexpr (BM == 1) {
              if constexpr ((FF & 2) != 0) ff::st_stream(pbout, B);
              else ff::st_stream_doubles(pbout, B);
              pbout += dst;
            }
            rf = ff::norm(ff::add(B, p));
          }
          if constexpr ((FF & 2) != 0) ff::st_stream(pout, rf);
          else ff::st_stream_doubles(pout, rf);
          pout += dst;
          if (e.wkey != wrun) {
            ff::acc(Gff, ff::mul(wff, Sff));
            Sff = ff::zero();
            wff = ff::P2{ff::pack(e.w32, e.w32), ff::pack(e.wlo, e.wlo)};
            wrun = e.wkey;
          }
          ff::acc(Sff, rf);
        };
        // Every step but the last kStages - 1 stages a later direction (no
        // bounds test); those last ones commit an empty group, so that the
        // wait above still finds its own group complete.
        const int nmain = nsteps - (kStages - 1);
        // Step j + kStages - 1 goes into the slot step j - 1 has just read.
        const unsigned slast = rb0 + (unsigned)(kStages - 1) * sstr;
        unsigned sprev = slast;
        int j = 0;
        for (; j < nmain; ++j) {
          issue(std::false_type{}, sprev);
          step(j);
          sprev = sb;
          sb = sb == slast ? rb0 : sb + sstr;
        }
        for (; j < nsteps; ++j) {
          cp_async_commit();
          step(j);
          sb = sb == slast ? rb0 : sb + sstr;
        }
      };
      if (c.wall == 0) run(std::true_type{});
      else run(std::false_type{});
      cp_async_wait<0>();
      ff::acc(Gff, ff::mul(wff, Sff));
      ff::to_doubles(ff::norm(Gff), G[0], G[1]);
    }
    sweep::item_epilogue<V, false>(a, ItemCtx{team, cpb, slot, dg, lane, lpc, dstep, b0, wid, wl, nwarps, nbp,
                                              nbp_all, band0, nbr, gsm, red, cst},
                                   wi, gp, G, cnt_solves, cnt_bad);
  }
  __syncthreads();
  if (threadIdx.x == 0 && a.counters) {
    if (cnt_solves) atomicAdd(&a.counters->solves, cnt_solves);
    if (cnt_bad) atomicAdd(&a.counters->nonfinite, cnt_bad);
  }
}

template <int DIM, int MINB, int BM, int FF>
cudaError_t launch_shape(const SweepArgs& a, int threads, int grid, cudaStream_t s) {
  const int team = a.lpc * a.dteam, cpb = threads / team;
  const size_t smem = sizeof(DirFF<DIM>) * (size_t)a.nd + 16 + 2 * (size_t)threads * sizeof(double) +
                      4 * (size_t)cpb * sizeof(double) + 16 +
                      (size_t)RingFF<DIM, MINB>::kStages * RingFF<DIM, MINB>::kOps * threads * 16;
  const cudaError_t e = raise_dynamic_smem((const void*)sweep_ff_kernel<DIM, MINB, BM, FF>, smem);
  if (e != cudaSuccess) return e;
  sweep_ff_kernel<DIM, MINB, BM, FF><<<grid, threads, smem, s>>>(a);
  return cudaGetLastError();
}

template <int BM, int FF>
cudaError_t launch_variant(int variant, const SweepArgs& a, int dim, int threads, int grid, cudaStream_t s) {
  const bool three = variant >= 2 && threads <= MaxThreadsFF<3>::value;
  if (dim == 3) {
    if (three) return launch_shape<3, 3, BM, FF>(a, threads, grid, s);
    return launch_shape<3, 2, BM, FF>(a, threads, grid, s);
  }
  if (three) return launch_shape<2, 3, BM, FF>(a, threads, grid, s);
  return launch_shape<2, 2, BM, FF>(a, threads, grid, s);
}

// variant: 1 -> at least 2 resident CTAs per SM, 2 -> 3 CTAs (the register caps;
// CTAs of more than 224 threads take variant 1)
inline cudaError_t launch(int variant, const SweepArgs& a, int dim, int threads, int grid, cudaStream_t s) {
  if (a.beta_exp != 0.0) return cudaErrorInvalidValue;
  if (a.bmode == 0 && a.ff == 2) return launch_variant<0, 2>(variant, a, dim, threads, grid, s);
  if (a.bmode == 0 && a.ff == 3) return launch_variant<0, 3>(variant, a, dim, threads, grid, s);
  if (a.bmode == 1 && a.ff == 2) return launch_variant<1, 2>(variant, a, dim, threads, grid, s);
  if (a.bmode == 1 && a.ff == 3) return launch_variant<1, 3>(variant, a, dim, threads, grid, s);
  if (a.bmode == 2 && a.ff == 3) return launch_variant<2, 3>(variant, a, dim, threads, grid, s);
  return cudaErrorInvalidValue;
}

}  // namespace sweep_ff
}  // namespace bte

// bte_gs.cu -- sweep-ordered (Gauss-Seidel) inner iteration of the implicit
// scheme, FP64 storage.
//
// The backward-Euler equation of (cell P, direction d, band b) is the same as
// in the Jacobi sweep (Eq. 5 with the Eq. 6 ghosts):
//   I_P = A_n I^n_P + sum_ax A_ax I_up,ax + A_s I0_P        (coefficients per
//   direction, band and cell-size class, already divided by the diagonal).
// Here the cells of a direction are visited in its upwind order, so an
// interior upwind neighbour holds its value of the current pass; mirror and
// diffuse wall ghosts and I0 stay at the previous iterate I^k.  With fixed
// ghosts one pass solves the streaming part exactly.
//
// Parallel layout.  All directions whose upwind sides agree (one octant: the
// signs of S_d) share one dependency order.  A CTA owns one unit (a geometry
// and ndc directions of one octant, all stored bands) and walks the whole
// grid by itself: column tiles in upwind order (2-D: strips of gs_tx columns;
// 3-D: gs_tx x gs_ty columns), and within a tile the wavefronts
// a + b + l = t (a, b: upwind-ordered position in the tile's cross-section,
// l: position along the last axis).  The cells of one wavefront depend only
// on the previous wavefront or on earlier tiles, all written by the same CTA,
// so a CTA barrier per wavefront is the only synchronisation: no CTA waits on
// another.  Upwind values written in this pass are read with ld.global.cg
// (L2), everything else is read-only here.
#include "bte_internal.h"
#include "bte_store.cuh"

namespace bte {

namespace {

__device__ __forceinline__ double2 ldg2(const double* p) { return __ldg(reinterpret_cast<const double2*>(p)); }
__device__ __forceinline__ double2 ldcg2(const double* p) { return __ldcg(reinterpret_cast<const double2*>(p)); }
__device__ __forceinline__ void st2(double* p, double x, double y) { *reinterpret_cast<double2*>(p) = make_double2(x, y); }

// Upwind value along one axis (this thread's two bands): the neighbour's value
// of this pass, or the Eq. 6 ghost at a wall (isothermal or diffuse row, the
// side's per-direction row when partially specular, or the cell's own previous
// iterate in the mirrored direction).  face: the wall face's index on its side.
__device__ __forceinline__ double2 upwind(const SweepArgs& a, const DevGeom* gp, const double* Io, const double* Ik,
                                          int side, bool interior, long long base, long long step, long long Prow,
                                          int rdir, long long face, int nbp, int b0) {
  if (interior) return ldcg2(Io + base + step);
  if (gp->bc[side] == 0) return ldg2(a.I0wall + (gp->face0[side] + face) * nbp + b0);
  if (gp->bc[side] == 3)
    return ldg2(reinterpret_cast<const double*>(gp->gdir[side]) + face * ((long long)a.nd * nbp) + (base - Prow));
  return ldg2(Ik + Prow + (long long)rdir * nbp + b0);
}

// The walk of one unit: column tiles in upwind order, wavefronts a + b + l = t
// within a tile, one CTA barrier per wavefront; update(i, j, k) for every cell
// of this thread's cell slots.  Every thread of the CTA runs the same loops.
template <int DIM, typename F>
__device__ __forceinline__ void walk(const SweepArgs& a, int nx, int ny, int nz, bool act, int grp, int ngrp, bool ax_,
                                     bool ay_, bool az_, F&& update) {
  if constexpr (DIM == 2) {
    for (int u0 = 0; u0 < nx; u0 += a.gs_tx) {  // strips of columns, upwind first
      const int w = min(a.gs_tx, nx - u0);
      for (int t = 0; t < w + ny - 1; ++t) {
        const int lo = max(0, t - (ny - 1)), hi = min(w - 1, t);
        if (act)
          for (int s = lo + grp; s <= hi; s += ngrp) {
            const int ux = u0 + s, uy = t - s;
            update(ax_ ? ux : nx - 1 - ux, ay_ ? uy : ny - 1 - uy, 0);
          }
        __syncthreads();
      }
    }
  } else {
    for (int v0 = 0; v0 < ny; v0 += a.gs_ty)
      for (int u0 = 0; u0 < nx; u0 += a.gs_tx) {  // column tiles, upwind first
        const int wx = min(a.gs_tx, nx - u0), wy = min(a.gs_ty, ny - v0);
        for (int t = 0; t < wx + wy + nz - 2; ++t) {
          if (act)
            for (int s = grp; s < wx * wy; s += ngrp) {
              const int p = s % wx, q = s / wx, l = t - p - q;
              if (l < 0 || l >= nz) continue;
              const int ux = u0 + p, uy = v0 + q;
              update(ax_ ? ux : nx - 1 - ux, ay_ ? uy : ny - 1 - uy, az_ ? l : nz - 1 - l);
            }
          __syncthreads();
        }
      }
  }
}

// BM: 0 In is I^n; 1 In is I^n and B = A_n I^n is also stored; 2 In holds B.
// TT: beta_b(T) = beta_b s per cell, s from a.bscale.
template <int DIM, int BM, bool TT>
__global__ void __launch_bounds__(256, 3) gs_sweep_kernel(SweepArgs a) {
  const int nbp = a.th.nbo, nd = a.nd;
  const int lpc = nbp / 2;  // lanes per (cell, direction) row, two bands each
  const int team = lpc * a.gs_ndc;
  const int ngrp = blockDim.x / team;  // cell slots per wavefront pass
  const int grp = threadIdx.x / team;
  const int tl = threadIdx.x - grp * team;
  const int dc = tl / lpc, lane = tl - dc * lpc;
  const int b0 = 2 * lane;
  const long long row = (long long)nd * nbp;
  const size_t plane = (size_t)nd * nbp;
  const double* __restrict__ In = reinterpret_cast<const double*>(a.In);
  const double* __restrict__ Ik = reinterpret_cast<const double*>(a.Ik);
  double* Io = reinterpret_cast<double*>(a.Iout);
  double* Bo = reinterpret_cast<double*>(a.Bout);
  const double* coef = reinterpret_cast<const double*>(a.coef);

  for (int u = blockIdx.x; u < a.gs_nunits; u += gridDim.x) {
    const GsUnit un = a.gs_units[u];
    const DevGeom* gp = a.geoms + un.geom;
    const int nx = gp->nx, ny = gp->ny, nz = DIM == 3 ? gp->nz : 1;
    const bool act = grp < ngrp && dc < un.ndc;
    const int d = a.gs_dirs[un.dir0 + (act ? dc : 0)];
    const DirInfo di = a.dirs[d];
    const bool ax_ = di.up & 1, ay_ = (di.up >> 1) & 1, az_ = (di.up >> 2) & 1;  // ascending along the axis
    // this thread's coefficients (direction d, bands b0, b0 + 1)
    const double* cf = coef + (size_t)gp->cls * 5 * plane + (size_t)d * nbp + b0;
    const double2 An = ldg2(cf), Ax = ldg2(cf + plane), Ay = ldg2(cf + 2 * plane);
    const double2 Az = DIM == 3 ? ldg2(cf + 3 * plane) : make_double2(0.0, 0.0);
    const double2 As = ldg2(cf + 4 * plane);
    const long long off = (long long)d * nbp + b0;
    const long long sx = row, sy = (long long)nx * row, sz = (long long)nx * ny * row;

    auto update = [&](int i, int j, int k) {
      const long long lc = ((long long)k * ny + j) * nx + i;
      const long long P = gp->cell0 + lc;
      const long long Prow = P * row;
      const long long base = Prow + off;
      const double2 vn = ldg2(In + base);
      const double2 src = ldg2(a.I0cell + P * nbp + b0);
      const double2 ux = upwind(a, gp, Io, Ik, ax_ ? 0 : 1, ax_ ? i > 0 : i < nx - 1, base, ax_ ? -sx : sx, Prow,
                                di.rx, (long long)j + (long long)ny * k, nbp, b0);
      const double2 uy = upwind(a, gp, Io, Ik, ay_ ? 2 : 3, ay_ ? j > 0 : j < ny - 1, base, ay_ ? -sy : sy, Prow,
                                di.ry, (long long)i + (long long)nx * k, nbp, b0);
      double2 uz = make_double2(0.0, 0.0);
      if (DIM == 3)
        uz = upwind(a, gp, Io, Ik, az_ ? 4 : 5, az_ ? k > 0 : k < nz - 1, base, az_ ? -sz : sz, Prow, di.rz,
                    (long long)i + (long long)nx * j, nbp, b0);
      double rx, ry;
      if (BM == 2) {
        rx = vn.x;
        ry = vn.y;
      } else {
        rx = An.x * vn.x;
        ry = An.y * vn.y;
        if (BM == 1) st2(Bo + base, rx, ry);
      }
      rx = fma(Ax.x, ux.x, rx);
      ry = fma(Ax.y, ux.y, ry);
      rx = fma(Ay.x, uy.x, rx);
      ry = fma(Ay.y, uy.y, ry);
      if (DIM == 3) {
        rx = fma(Az.x, uz.x, rx);
        ry = fma(Az.y, uz.y, ry);
      }
      if constexpr (!TT) {
        rx = fma(As.x, src.x, rx);
        ry = fma(As.y, src.y, ry);
      } else {  // every coefficient x 1/(1 + (s - 1) A_s), A_s also x s
        const double s = a.bscale[P];
        rx = fma(s * As.x, src.x, rx) * __drcp_rn(fma(s - 1.0, As.x, 1.0));
        ry = fma(s * As.y, src.y, ry) * __drcp_rn(fma(s - 1.0, As.y, 1.0));
      }
      st2(Io + base, rx, ry);
    };

    walk<DIM>(a, nx, ny, nz, act, grp, ngrp, ax_, ay_, az_, update);
  }
}

// Reduced storage (FP32 / BF16 deviations from I0_b(T_ref), update in FP32):
// the same walk and equation on deviations,
//   dev' = P dev^n + Q [v_b sum_ax c_ax dev_up + beta_b (I0 - I0ref)],
//   Q = 1 / (1/dt + beta_b + v_b sum_ax c_ax), P = Q / dt,
// with beta_b scaled per cell when tau depends on T.  A lane holds V bands
// (16 bytes of storage); wall ghosts are the float deviation rows (isothermal,
// diffuse), the side's per-direction rows (partially specular) or the cell's
// own previous iterate mirrored.
template <typename S, int DIM>
__global__ void __launch_bounds__(256, 3) gs_sweep_dev_kernel(SweepArgs a) {
  using T = Tr<S>;
  constexpr int V = T::V;
  const int nbp = a.th.nbo, nd = a.nd;
  const int lpc = nbp / V;
  const int team = lpc * a.gs_ndc;
  const int ngrp = blockDim.x / team;
  const int grp = threadIdx.x / team;
  const int tl = threadIdx.x - grp * team;
  const int dc = tl / lpc, lane = tl - dc * lpc;
  const int b0 = V * lane;
  const long long row = (long long)nd * nbp;
  const S* __restrict__ In = reinterpret_cast<const S*>(a.In);
  const S* __restrict__ Ik = reinterpret_cast<const S*>(a.Ik);
  S* Io = reinterpret_cast<S*>(a.Iout);
  const bool tT = a.beta_exp != 0.0;
  float vb[V], bb[V], i0r[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    vb[v] = a.vb32[b0 + v];
    bb[v] = a.bb32[b0 + v];
    i0r[v] = (float)a.I0ref[b0 + v];
  }
  for (int u = blockIdx.x; u < a.gs_nunits; u += gridDim.x) {
    const GsUnit un = a.gs_units[u];
    const DevGeom* gp = a.geoms + un.geom;
    const int nx = gp->nx, ny = gp->ny, nz = DIM == 3 ? gp->nz : 1;
    const bool act = grp < ngrp && dc < un.ndc;
    const int d = a.gs_dirs[un.dir0 + (act ? dc : 0)];
    const DirInfo di = a.dirs[d];
    const bool ax_ = di.up & 1, ay_ = (di.up >> 1) & 1, az_ = (di.up >> 2) & 1;
    const float4 cc = a.dirc[(size_t)gp->cls * nd + d];  // c_x, c_y, c_z, sum
    const long long off = (long long)d * nbp + b0;
    const long long sx = row, sy = (long long)nx * row, sz = (long long)nx * ny * row;
    // upwind deviations along one axis: this pass's neighbour, or the wall ghost
    auto upwind_dev = [&](int side, bool interior, long long base, long long step, long long Prow, int rdir,
                          long long face, float (&x)[V]) {
      if (interior) {
        const S* p = Io + base + step;
        if constexpr (sizeof(S) == 4) {
          const float4 v = __ldcg(reinterpret_cast<const float4*>(p));
          x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
        } else {
          T::unpack(__ldcg(reinterpret_cast<const uint4*>(p)), x);
        }
      } else if (gp->bc[side] == 0) {
        ldgv<float, V>(a.I0wall_dev + (gp->face0[side] + face) * nbp + b0, x);
      } else if (gp->bc[side] == 3) {
        T::ld(reinterpret_cast<const S*>(gp->gdir[side]) + face * row + (base - Prow), x);
      } else {
        T::ld(Ik + Prow + (long long)rdir * nbp + b0, x);
      }
    };
    auto update = [&](int i, int j, int k) {
      const long long P = gp->cell0 + ((long long)k * ny + j) * nx + i;
      const long long Prow = P * row;
      const long long base = Prow + off;
      float in[V], ux[V], uy[V], uz[V];
      T::ld(In + base, in);
      upwind_dev(ax_ ? 0 : 1, ax_ ? i > 0 : i < nx - 1, base, ax_ ? -sx : sx, Prow, di.rx,
                 (long long)j + (long long)ny * k, ux);
      upwind_dev(ay_ ? 2 : 3, ay_ ? j > 0 : j < ny - 1, base, ay_ ? -sy : sy, Prow, di.ry,
                 (long long)i + (long long)nx * k, uy);
      if (DIM == 3)
        upwind_dev(az_ ? 4 : 5, az_ ? k > 0 : k < nz - 1, base, az_ ? -sz : sz, Prow, di.rz,
                   (long long)i + (long long)nx * j, uz);
      const float sc = tT ? (float)a.bscale[P] : 1.f;
      float r[V];
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const float be = bb[v] * sc;
        const float src = be * ((float)a.I0cell[P * nbp + b0 + v] - i0r[v]);
        float Q;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(Q) : "f"(a.rdt32 + fmaf(vb[v], cc.w, be)));
        float f = cc.x * ux[v];
        f = fmaf(cc.y, uy[v], f);
        if (DIM == 3) f = fmaf(cc.z, uz[v], f);
        r[v] = fmaf(Q, fmaf(vb[v], f, src), Q * a.rdt32 * in[v]);
      }
      T::st(Io + base, r);
    };
    walk<DIM>(a, nx, ny, nz, act, grp, ngrp, ax_, ay_, az_, update);
  }
}

template <int DIM, int BM>
cudaError_t launch_dim_bm(const SweepArgs& a, int threads, int grid, cudaStream_t s) {
  if (a.beta_exp != 0.0) gs_sweep_kernel<DIM, BM, true><<<grid, threads, 0, s>>>(a);
  else gs_sweep_kernel<DIM, BM, false><<<grid, threads, 0, s>>>(a);
  return cudaGetLastError();
}

template <int DIM>
cudaError_t launch_dim(const SweepArgs& a, int threads, int grid, cudaStream_t s) {
  if (a.bmode == 1) return launch_dim_bm<DIM, 1>(a, threads, grid, s);
  if (a.bmode == 2) return launch_dim_bm<DIM, 2>(a, threads, grid, s);
  return launch_dim_bm<DIM, 0>(a, threads, grid, s);
}

__global__ void beta_scale_kernel(double* out, const double* Tp, double Tref, double p, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = pow(Tp[i] / Tref, p);
}

}  // namespace

// threads: a multiple of lpc * gs_ndc, at most 256; one CTA per unit.
cudaError_t launch_gs_sweep(int precision, const SweepArgs& a, int dim, int threads, cudaStream_t s) {
  if (a.gs_nunits <= 0) return cudaSuccess;
  const int grid = a.gs_nunits;
  if (precision == 1) {
    if (dim == 3) gs_sweep_dev_kernel<float, 3><<<grid, threads, 0, s>>>(a);
    else gs_sweep_dev_kernel<float, 2><<<grid, threads, 0, s>>>(a);
    return cudaGetLastError();
  }
  if (precision == 2) {
    if (dim == 3) gs_sweep_dev_kernel<__nv_bfloat16, 3><<<grid, threads, 0, s>>>(a);
    else gs_sweep_dev_kernel<__nv_bfloat16, 2><<<grid, threads, 0, s>>>(a);
    return cudaGetLastError();
  }
  return dim == 3 ? launch_dim<3>(a, threads, grid, s) : launch_dim<2>(a, threads, grid, s);
}

cudaError_t launch_beta_scale(double* out, const double* Tp, double Tref, double p, long long ncells, cudaStream_t s) {
  const int grid = (int)std::min<long long>((ncells + 255) / 256, 4096);
  beta_scale_kernel<<<grid > 0 ? grid : 1, 256, 0, s>>>(out, Tp, Tref, p, ncells);
  return cudaGetLastError();
}

}  // namespace bte

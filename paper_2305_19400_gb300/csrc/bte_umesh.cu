// bte_umesh.cu -- the hot path on unstructured meshes (include/bte_umesh.h):
// the face-sum form of Eq. 5 on a face list, then the per-cell reduction,
// T_p solve and I0 refresh shared with the sweep-ordered scheme
// (gs_reduce_kernel) and the exact fix-up (fixup_kernel).  FP64 storage.
//
// Device layout (cudaMalloc per array):
//   I buffers   3 x [cell][dir][nbp]
//   cell faces  CSR: cf_ptr[cell], per entry the upwind code (neighbour cell,
//               or -1 - boundary face index) and g[entry][dir] =
//               (S_d . n A)/(w_d V) with n out of the cell; gout[cell][dir] =
//               sum of the positive g (outflow)
//   boundary    per boundary face: kind (ghost row, mirror, or p x mirror +
//               ghost row), mirror axis, specularity p, ghost rows
//               [bface][nbp] (isothermal I0, refreshed diffuse values, scaled
//               by 1 - p on partially specular faces)
//   R           [cell][dir][nbp] implicit reciprocal diagonal 1/(1/dt + beta_b +
//               v_b gout), rebuilt when dt changes (one division per element
//               instead of one per update)
// Sweep kernel: a team of lpc x dteam lanes per cell (lane: two bands, team
// step: dteam directions), every face of the cell per direction.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/bte_umesh.h"
#include "bte_internal.h"
#include "bte_store.cuh"
#include "bte_tables.h"

using namespace bte;

namespace {

constexpr int kMaxCellFaces = 64;

struct UArgs {
  const double* In;        // I^n, or B = (I^n/dt) R (implicit, BM = 2)
  double* Bout;            // BM = 1: receives B
  const double* Ik;
  double* Iout;
  const double* I0cell;
  const double* ghost;     // [bface][nbp]
  const int* cf_ptr;       // [nc + 1]
  const long long* cf_up;  // [entries] neighbour cell, or -1 - bface
  const double* g;         // [entries][nd]
  const double* gout;      // [nc][nd]
  const int* bf_mirror;    // [bface] 0: ghost row, 1: mirror, 2: p x mirror + ghost row
  const int* bf_axis;      // [bface]
  const double* bf_spec;   // [bface] specularity p of kind-2 faces
  const int* refl;         // [3][nd]
  const double* R;         // [nc][nd][nbp] implicit: 1 / (1/dt + beta_b + v_b gout)
  const double* vb;        // [nbp] v_b (0 on padding)
  const double* bb;        // [nbp] beta_b (0 on padding)
  double dt, rdt;
  long long nc;
  int nd, nbp, lpc, dteam;
  // reduced storage (deviations from I0_b(T_ref)): buffers in the storage type,
  // R and the ghost deviations as float
  const void* Ind;
  const void* Ikd;
  void* Ioutd;
  void* Boutd;
  const float* Rf;
  const float* ghost_dev;
  const double* I0ref;
  const float* g32;        // [entries][nd] g as float (reduced storage)
  const double* bscale;    // TT: [nc] s = (T_p / T_ref)^p, beta_b(T_p) = beta_b s
};

// V consecutive floats (16-byte loads).
template <int V>
__device__ __forceinline__ void ldf(const float* p, float (&x)[V]) {
#pragma unroll
  for (int i = 0; i < V; i += 4) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p + i));
    x[i] = v.x; x[i + 1] = v.y; x[i + 2] = v.z; x[i + 3] = v.w;
  }
}

// Reduced-storage form of umesh_sweep_kernel: I = I0_b(T_ref) + deviation, the
// deviation stored in S (FP32 or BF16) and updated in FP32 with the same
// equation (both direction sets are point-symmetric, so a closed cell's inflow
// and outflow sums of |g| are equal and the reference part cancels):
// implicit R [v sum |g| dev_up + beta (I0 - I0ref)] + (dev^n/dt) R, explicit
// dev + dt [beta (I0 - I0ref - dev) - v (gout dev - sum |g| dev_up)].
// A lane holds V bands (16 bytes of storage).  The kernel is bound by the
// latency of the face gathers, so it is capped at 6 CTAs of 252 threads per SM
// (more warps in flight; measured faster than 3-5 CTAs despite small spills).
template <typename S, bool EXPL, int BM, bool TT>
__global__ void __launch_bounds__(256, 6) umesh_sweep_dev_kernel(UArgs a) {
  using T = Tr<S>;
  constexpr int V = T::V;
  const int team = a.lpc * a.dteam;
  const int cpb = blockDim.x / team;
  const int slot = threadIdx.x / team, tl = threadIdx.x - slot * team;
  const int dg = tl / a.lpc, lane = tl - dg * a.lpc;
  const int b0 = V * lane;
  if (slot >= cpb) return;  // no barrier or shuffle below
  const long long row = (long long)a.nd * a.nbp;
  const S* In = reinterpret_cast<const S*>(a.Ind);
  const S* Isrc = EXPL ? In : reinterpret_cast<const S*>(a.Ikd);
  S* Io = reinterpret_cast<S*>(a.Ioutd);
  S* Bo = reinterpret_cast<S*>(a.Boutd);
  const float dt = (float)a.dt, rdt = (float)a.rdt;
  float vb[V], bb[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    vb[v] = (float)a.vb[b0 + v];
    bb[v] = (float)a.bb[b0 + v];
  }
  for (long long P = (long long)blockIdx.x * cpb + slot; P < a.nc; P += (long long)gridDim.x * cpb) {
    const int e0 = a.cf_ptr[P], e1 = a.cf_ptr[P + 1];
    float bs[V], sm1[V];  // beta_b(T_p) = beta_b s; (s - 1) beta_b
    const double sc = TT ? a.bscale[P] : 1.0;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      bs[v] = TT ? (float)(sc * (double)bb[v]) : bb[v];
      sm1[v] = TT ? (float)((sc - 1.0) * (double)bb[v]) : 0.f;
    }
    float src[V];  // beta_b(T_p) (I0 - I0ref)
#pragma unroll
    for (int v = 0; v < V; ++v) src[v] = bs[v] * (float)(a.I0cell[P * a.nbp + b0 + v] - a.I0ref[b0 + v]);
    for (int d = dg; d < a.nd; d += a.dteam) {
      const long long off = P * row + (long long)d * a.nbp + b0;
      float in[V], f[V];
      T::ld(In + off, in);
#pragma unroll
      for (int v = 0; v < V; ++v) f[v] = 0.f;
      for (int e = e0; e < e1; ++e) {
        const float ge = a.g32[(long long)e * a.nd + d];
        if (__float_as_int(ge) < 0) {  // inflow: the sign bit, tested on the integer pipe
          const long long up = a.cf_up[e];
          const float gf = -ge;
          if (up >= 0) {
            float u[V];
            T::ld(Isrc + up * row + (long long)d * a.nbp + b0, u);
#pragma unroll
            for (int v = 0; v < V; ++v) f[v] = fmaf(gf, u[v], f[v]);
          } else {
            // ghost row (isothermal, diffuse, or (1 - p) x diffuse) and/or the
            // mirrored value (weight p on a partially specular face), one row
            // live at a time
            const long long bf = -1 - up;
            const int mk = a.bf_mirror[bf];
            float wm = gf;
            if (mk != 1) {
              float u[V];
              ldf<V>(a.ghost_dev + bf * a.nbp + b0, u);
#pragma unroll
              for (int v = 0; v < V; ++v) f[v] = fmaf(gf, u[v], f[v]);
              wm = mk == 2 ? gf * (float)a.bf_spec[bf] : 0.f;
            }
            if (mk != 0) {
              float u[V];
              T::ld(Isrc + P * row + (long long)a.refl[a.bf_axis[bf] * a.nd + d] * a.nbp + b0, u);
#pragma unroll
              for (int v = 0; v < V; ++v) f[v] = fmaf(wm, u[v], f[v]);
            }
          }
        }
      }
      float r[V];
      if (EXPL) {
        const float go = (float)a.gout[P * a.nd + d];
#pragma unroll
        for (int v = 0; v < V; ++v) r[v] = fmaf(dt, fmaf(-bs[v], in[v], src[v]) - vb[v] * fmaf(go, in[v], -f[v]), in[v]);
      } else {
        float R[V], B[V];
        ldf<V>(a.Rf + off, R);
#pragma unroll
        for (int v = 0; v < V; ++v) B[v] = BM == 2 ? in[v] : in[v] * rdt * R[v];
        if (BM == 1) T::st(Bo + off, B);
#pragma unroll
        for (int v = 0; v < V; ++v) r[v] = fmaf(R[v], fmaf(vb[v], f[v], src[v]), B[v]);
        if constexpr (TT) {  // R_s = R / (1 + (s - 1) beta R): the cached R is at s = 1
#pragma unroll
          for (int v = 0; v < V; ++v) r[v] *= __frcp_rn(fmaf(sm1[v], R[v], 1.f));
        }
      }
      T::st(Io + off, r);
    }
  }
}

__device__ __forceinline__ double2 ld2(const double* p) { return __ldg(reinterpret_cast<const double2*>(p)); }

// EXPL: explicit scheme.  BM (implicit): 0 In is I^n; 1 In is I^n and B =
// (I^n/dt) R is stored; 2 In holds B (the same in every inner iteration of a
// step), so the update is R (beta I0 + v sum |g| I_up) + B.  Capped at 5 CTAs
// of 256 threads per SM (48 registers, a few bytes of spill outside the face
// loop): uncapped it takes 58 registers and 4 CTAs, measured 7 % slower.
template <bool EXPL, int BM, bool TT>
__global__ void __launch_bounds__(256, 5) umesh_sweep_kernel(UArgs a) {
  const int team = a.lpc * a.dteam;
  const int cpb = blockDim.x / team;
  const int slot = threadIdx.x / team, tl = threadIdx.x - slot * team;
  const int dg = tl / a.lpc, lane = tl - dg * a.lpc;
  const int b0 = 2 * lane;
  if (slot >= cpb) return;  // no barrier below
  const long long row = (long long)a.nd * a.nbp;
  const double v0 = a.vb[b0], v1 = a.vb[b0 + 1], be0 = a.bb[b0], be1 = a.bb[b0 + 1];
  for (long long P = (long long)blockIdx.x * cpb + slot; P < a.nc; P += (long long)gridDim.x * cpb) {
    const int e0 = a.cf_ptr[P], e1 = a.cf_ptr[P + 1];
    const double2 i0 = ld2(a.I0cell + P * a.nbp + b0);
    // beta_b(T_p) = beta_b s (s = 1 unless TT) and (s - 1) beta_b
    const double sc = TT ? a.bscale[P] : 1.0;
    const double bs0 = TT ? sc * be0 : be0, bs1 = TT ? sc * be1 : be1;
    const double sm0 = TT ? (sc - 1.0) * be0 : 0.0, sm1 = TT ? (sc - 1.0) * be1 : 0.0;
    const double bi0 = bs0 * i0.x, bi1 = bs1 * i0.y;
    for (int d = dg; d < a.nd; d += a.dteam) {
      const long long off = P * row + (long long)d * a.nbp + b0;
      const double2 in = ld2(a.In + off);
      const double* Isrc = EXPL ? a.In : a.Ik;
      double f0 = 0.0, f1 = 0.0;  // sum over inflow faces of |g| I_up
      for (int e = e0; e < e1; ++e) {
        const double ge = a.g[(long long)e * a.nd + d];
        if (__double_as_longlong(ge) < 0) {  // inflow: the sign bit, tested on the integer pipe
          const long long up = a.cf_up[e];
          if (up >= 0) {
            const double2 u = ld2(Isrc + up * row + (long long)d * a.nbp + b0);
            f0 = fma(-ge, u.x, f0);
            f1 = fma(-ge, u.y, f1);
          } else {
            // ghost row (isothermal, diffuse, or (1 - p) x diffuse) and/or the
            // mirrored value (weight p on a partially specular face)
            const long long bf = -1 - up;
            const int mk = a.bf_mirror[bf];
            double wm = -ge;
            if (mk != 1) {
              const double2 u = ld2(a.ghost + bf * a.nbp + b0);
              f0 = fma(-ge, u.x, f0);
              f1 = fma(-ge, u.y, f1);
              wm = mk == 2 ? -ge * a.bf_spec[bf] : 0.0;
            }
            if (mk != 0) {
              const double2 u = ld2(Isrc + P * row + (long long)a.refl[a.bf_axis[bf] * a.nd + d] * a.nbp + b0);
              f0 = fma(wm, u.x, f0);
              f1 = fma(wm, u.y, f1);
            }
          }
        }
      }
      double r0, r1;
      if (EXPL) {  // I + dt [beta (I0 - I) - v (gout I - sum |g| I_up)]
        const double go = a.gout[P * a.nd + d];
        r0 = fma(a.dt, fma(bs0, i0.x - in.x, -v0 * fma(go, in.x, -f0)), in.x);
        r1 = fma(a.dt, fma(bs1, i0.y - in.y, -v1 * fma(go, in.y, -f1)), in.y);
      } else {  // R [beta I0 + v sum |g| I_up] + (I^n/dt) R, R = 1 / [1/dt + beta + v gout]
        const double2 rr = ld2(a.R + off);
        double B0 = in.x, B1 = in.y;
        if (BM != 2) {
          B0 = in.x * a.rdt * rr.x;
          B1 = in.y * a.rdt * rr.y;
          if (BM == 1) *reinterpret_cast<double2*>(a.Bout + off) = make_double2(B0, B1);
        }
        r0 = fma(rr.x, fma(v0, f0, bi0), B0);
        r1 = fma(rr.y, fma(v1, f1, bi1), B1);
        if constexpr (TT) {  // R_s = R / (1 + (s - 1) beta R): the cached R is at s = 1
          r0 *= __drcp_rn(fma(sm0, rr.x, 1.0));
          r1 *= __drcp_rn(fma(sm1, rr.y, 1.0));
        }
      }
      *reinterpret_cast<double2*>(a.Iout + off) = make_double2(r0, r1);
    }
  }
}

// R[P][d][b] = 1 / (1/dt + beta_b + v_b gout[P][d]): the implicit update's
// reciprocal diagonal, fixed while dt is (one thread per element).
template <typename R_t>
__global__ void umesh_rcp_kernel(const double* gout, const double* vb, const double* bb, double rdt, long long nc,
                                 int nd, int nbp, R_t* R) {
  const long long n = nc * nd * nbp;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i % nbp);
    R[i] = (R_t)(1.0 / fma(vb[b], gout[i / nbp], rdt + bb[b]));
  }
}

// g[entry][d] = sign (S_d . nA_f) / (w_d V_P); one thread per (entry, direction).
__global__ void umesh_geom_kernel(const long long* ent_face, const int* ent_sign, const long long* ent_cell,
                                  const double* nA, const double* vol, const double* S, const double* w, int nd,
                                  long long nent, double* g) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nent * nd;
       i += (long long)gridDim.x * blockDim.x) {
    const long long e = i / nd;
    const int d = (int)(i - e * nd);
    const double* n = nA + 3 * ent_face[e];
    const double sn = S[3 * d] * n[0] + S[3 * d + 1] * n[1] + S[3 * d + 2] * n[2];
    g[i] = ent_sign[e] * sn / (w[d] * vol[ent_cell[e]]);
  }
}

__global__ void to_float_kernel(const double* x, long long n, float* y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

// gout[P][d] = sum over the cell's entries (in order) of the positive g.
__global__ void umesh_gout_kernel(const int* cf_ptr, const double* g, int nd, long long nc, double* gout) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nc * nd; i += (long long)gridDim.x * blockDim.x) {
    const long long P = i / nd;
    const int d = (int)(i - P * nd);
    double s = 0.0;
    for (int e = cf_ptr[P]; e < cf_ptr[P + 1]; ++e) {
      const double ge = g[(long long)e * nd + d];
      if (ge > 0.0) s += ge;
    }
    gout[i] = s;
  }
}

// Diffuse ghosts: for each listed boundary face, per band,
// sum_{S.n > 0} (S.n) I / sum_{S.n < 0} |S.n| of the owner cell.  One CTA of
// kDiffWarps warps per face: warp w sums the directions [w nd/W, (w+1) nd/W)
// (lanes over bands); the partial sums are added in warp order.  Reduced
// storage sums the stored deviations and writes the ghost deviation (the
// reference part passes through the ratio: the sets are point-symmetric).
// On a partially specular face the row receives (1 - p) x the diffuse value
// (the sweep adds p x the mirrored value).
constexpr int kDiffWarps = 8;

template <typename St>
__global__ void __launch_bounds__(32 * kDiffWarps) umesh_diffuse_kernel(const St* I, const long long* bfs, int nlist,
                                                                        const long long* bface, const long long* owner,
                                                                        const double* nA, const double* S, int nd,
                                                                        int nbp, const double* spec, double* ghost,
                                                                        float* ghost_dev) {
  extern __shared__ double part[];  // [kDiffWarps][2][nbp]
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int d0 = (int)((long long)wid * nd / kDiffWarps), d1 = (int)((long long)(wid + 1) * nd / kDiffWarps);
  for (int k = blockIdx.x; k < nlist; k += gridDim.x) {
    const long long bf = bfs[k], f = bface[bf], P = owner[f];
    const double* n = nA + 3 * f;
    const St* row = I + P * (long long)nd * nbp;
    for (int b = lane; b < nbp; b += 32) {
      double num = 0.0, den = 0.0;
#pragma unroll 4
      for (int e = d0; e < d1; ++e) {
        const double sn = S[3 * e] * n[0] + S[3 * e + 1] * n[1] + S[3 * e + 2] * n[2];
        if (sn > 0.0) num = fma(sn, Tr<St>::to_double(row[(long long)e * nbp + b]), num);
        else den -= sn;
      }
      part[(wid * 2) * nbp + b] = num;
      part[(wid * 2 + 1) * nbp + b] = den;
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbp; b += blockDim.x) {
      double num = 0.0, den = 0.0;
      for (int w = 0; w < kDiffWarps; ++w) {
        num += part[(w * 2) * nbp + b];
        den += part[(w * 2 + 1) * nbp + b];
      }
      const double v = (1.0 - spec[bf]) * (den > 0.0 ? num / den : 0.0);
      if constexpr (sizeof(St) == 8) ghost[bf * nbp + b] = v;
      else ghost_dev[bf * nbp + b] = (float)v;
    }
    __syncthreads();
  }
}

// Net heat flow out through each boundary face: one warp per face.
template <typename St>
__global__ void umesh_face_flux_kernel(const St* I, const double* I0ref, const double* ghost, const float* ghost_dev,
                                       const long long* bface, long long nbf, const long long* owner, const double* nA,
                                       const int* bf_mirror, const int* bf_axis, const double* bf_spec,
                                       const int* refl, const double* S, int nd, int nbp, int nb, double* Qb) {
  const int warps = blockDim.x / 32, lane = threadIdx.x & 31;
  for (long long bf = blockIdx.x * (long long)warps + threadIdx.x / 32; bf < nbf; bf += (long long)gridDim.x * warps) {
    const long long f = bface[bf], P = owner[f];
    const double* n = nA + 3 * f;
    const long long base = P * (long long)nd * nbp;
    double s = 0.0;
    for (int d = 0; d < nd; ++d) {
      const double sn = S[3 * d] * n[0] + S[3 * d + 1] * n[1] + S[3 * d + 2] * n[2];
      for (int b = lane; b < nb; b += 32) {
        double v;
        const int mk = bf_mirror[bf];
        if (sn > 0.0) {
          v = full_I(I, base + (long long)d * nbp + b, b, I0ref);
        } else if (mk == 1) {
          v = full_I(I, base + (long long)refl[bf_axis[bf] * nd + d] * nbp + b, b, I0ref);
        } else {  // the ghost row, plus p x the mirrored value on a partially specular face
          if constexpr (sizeof(St) == 8) v = ghost[bf * nbp + b];
          else v = I0ref[b] * (mk == 2 ? 1.0 - bf_spec[bf] : 1.0) + (double)ghost_dev[bf * nbp + b];
          if (mk == 2) v += bf_spec[bf] * full_I(I, base + (long long)refl[bf_axis[bf] * nd + d] * nbp + b, b, I0ref);
        }
        s = fma(sn, v, s);
      }
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) Qb[bf] = s;
  }
}

// One sweep launch: storage precision, scheme, B mode (0 plain, 1 store B, 2
// read B) and TT (per-cell relaxation scale).
template <bool TT>
cudaError_t launch_umesh_sweep(int prec, bool expl, int bm, const UArgs& a, int grid, int threads, cudaStream_t s) {
  if (prec == BTE_FP64) {
    if (expl) umesh_sweep_kernel<true, 0, TT><<<grid, threads, 0, s>>>(a);
    else if (bm == 1) umesh_sweep_kernel<false, 1, TT><<<grid, threads, 0, s>>>(a);
    else if (bm == 2) umesh_sweep_kernel<false, 2, TT><<<grid, threads, 0, s>>>(a);
    else umesh_sweep_kernel<false, 0, TT><<<grid, threads, 0, s>>>(a);
  } else if (prec == BTE_FP32) {
    if (expl) umesh_sweep_dev_kernel<float, true, 0, TT><<<grid, threads, 0, s>>>(a);
    else if (bm == 1) umesh_sweep_dev_kernel<float, false, 1, TT><<<grid, threads, 0, s>>>(a);
    else if (bm == 2) umesh_sweep_dev_kernel<float, false, 2, TT><<<grid, threads, 0, s>>>(a);
    else umesh_sweep_dev_kernel<float, false, 0, TT><<<grid, threads, 0, s>>>(a);
  } else {
    if (expl) umesh_sweep_dev_kernel<__nv_bfloat16, true, 0, TT><<<grid, threads, 0, s>>>(a);
    else if (bm == 1) umesh_sweep_dev_kernel<__nv_bfloat16, false, 1, TT><<<grid, threads, 0, s>>>(a);
    else if (bm == 2) umesh_sweep_dev_kernel<__nv_bfloat16, false, 2, TT><<<grid, threads, 0, s>>>(a);
    else umesh_sweep_dev_kernel<__nv_bfloat16, false, 0, TT><<<grid, threads, 0, s>>>(a);
  }
  return cudaGetLastError();
}

thread_local std::string g_umesh_err;

int grid_for(long long n, int per_block) {
  return (int)std::max<long long>(1, std::min<long long>((n + per_block - 1) / per_block, 152LL * 32));
}

}  // namespace

struct bte_umesh_ctx {
  std::string err;
  cudaStream_t stream = nullptr;
  bte_opts opts{};
  int dim = 2;
  long long nc = 0, nf = 0;
  std::vector<double> vol, nA;
  std::vector<long long> owner, nbr;
  std::vector<int> tag;
  // boundary faces
  std::vector<long long> bface;  // face id of each boundary face
  std::vector<int> bf_tag, bf_type, bf_axis, bf_ok_axis;
  std::vector<int> bf_geo_axis;  // axis of the face normal; bf_axis is it, or 3 / 4 on rotational faces
  std::vector<double> fc;        // [nf][3] face centres (empty when the mesh gave none)
  double rot_alpha = 0.0;        // wedge angle of the rotational faces (0: none set)
  std::vector<double> bf_T, bf_p;  // isothermal temperature / specularity
  std::vector<int> tags;          // distinct boundary tags
  std::vector<char> tag_set;      // per entry of tags
  // directions
  int nd = 0;
  std::vector<double> S, w;
  std::vector<int> refl;  // [5][nd]: mirror across x, y, z; rotation about z by -alpha, by +alpha
  double Wtot = 0.0;
  // bands
  bool bands_set = false, solve_tp = false;
  int nb = 0, nbp = 0, ng = 16;
  std::vector<double> wlo, whi, vg, beta, deg;
  // device
  std::vector<void*> allocs;
  bool mem_ready = false, init_done = false, TL_valid = false;
  double* I[3] = {nullptr, nullptr, nullptr};
  int cur = 0;
  double *I0cell = nullptr, *J = nullptr, *Teval = nullptr, *Tp = nullptr, *TL = nullptr, *EL = nullptr;
  double* Msum = nullptr;  // [cell][3] the T_p model's sums, kept with J
  double *ghost = nullptr, *g = nullptr, *gout = nullptr, *S_d = nullptr, *w_d = nullptr, *nA_d = nullptr;
  double *vb_d = nullptr, *bb_d = nullptr, *bfT_d = nullptr, *scratch = nullptr, *Qb = nullptr, *qbuf = nullptr;
  double* bf_spec_d = nullptr;  // [bface] specularity of partially specular faces, 0 elsewhere
  double* bscale = nullptr;     // [nc] relaxation scale (T_p / T_ref)^beta_T_exp
  double* R = nullptr;     // implicit reciprocal diagonal for R_dt (FP64 storage)
  float* Rf = nullptr;     //   the same as float (reduced storage)
  double R_dt = -1.0;
  int prec = BTE_FP64;     // storage of I: FP64, or FP32 / BF16 deviations from I0_b(T_ref)
  double* I0ref = nullptr; // [nbp] I0_b(T_ref)
  float* ghost_dev = nullptr;  // [bface][nbp] ghost deviations (reduced storage)
  float* w32_d = nullptr;  // [nd] direction weights as float
  float* g32 = nullptr;    // [entries][nd] g as float (reduced storage)
  double *node_c = nullptr, *node_C = nullptr, *a_p = nullptr, *a_L = nullptr, *inv_v = nullptr, *beta_d = nullptr;
  int *cf_ptr = nullptr, *bf_mirror_d = nullptr, *bf_axis_d = nullptr, *refl_d = nullptr;
  long long *cf_up = nullptr, *bface_d = nullptr, *owner_d = nullptr, *diff_d = nullptr;
  int ndiff = 0;
  FixItem* fix = nullptr;
  unsigned* fix_count = nullptr;
  DevCounters* counters = nullptr;
  int lpc = 0, dteam = 1;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

int ufail(bte_umesh_ctx* u, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (u) u->err = buf; else g_umesh_err = buf;
  return code;
}

#define UTRY(u, call)                                                                         \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return ufail(u, BTE_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
int dalloc(bte_umesh_ctx* u, T** p, size_t n) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
  if (e != cudaSuccess) return ufail(u, BTE_E_NOMEM, "cudaMalloc(%zu bytes): %s", n * sizeof(T), cudaGetErrorString(e));
  u->allocs.push_back(q);
  *p = (T*)q;
  return BTE_OK;
}

template <typename T>
int upload(bte_umesh_ctx* u, T* dst, const T* src, size_t n) {
  UTRY(u, cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyHostToDevice, u->stream));
  return BTE_OK;
}

ThermoTables uthermo(const bte_umesh_ctx* u) {
  ThermoTables t;
  t.node_c = u->node_c;
  t.node_C = u->node_C;
  t.a_p = u->a_p;
  t.a_L = u->a_L;
  t.inv_v = u->inv_v;
  t.beta = u->beta_d;
  t.ng = u->ng;
  t.nbp = t.nbo = u->nbp;
  t.nb = t.nbr = u->nb;
  t.band0 = 0;
  return t;
}

// SweepArgs for the per-cell step and the fix-up (the fields those kernels read).
SweepArgs cell_args(bte_umesh_ctx* u, double* Inew) {
  SweepArgs a{};
  a.Iout = Inew;
  a.I0cell = u->I0cell;
  a.Tp = u->Tp;
  a.Teval = u->Teval;
  a.J = u->J;
  a.Msum = u->Msum;
  a.EL = u->EL;
  a.wdir = u->w_d;
  a.nd = u->nd;
  a.solve_tp = u->solve_tp ? 1 : 0;
  a.trust_rel = std::cbrt(u->opts.newton_rtol / 4.0);
  a.maxit = u->opts.newton_maxit;
  a.counters = u->counters;
  a.fix = u->fix;
  a.fix_count = u->fix_count;
  a.partial = 0;
  a.I0ref = u->I0ref;
  a.Wtot = u->Wtot;
  a.wdir32 = u->w32_d;
  a.th = uthermo(u);
  return a;
}

// Device arrays, tables and the cell -> face lists (after the band table).
int ensure_mem(bte_umesh_ctx* u) {
  if (u->mem_ready) return BTE_OK;
  int rc;
  const long long nc = u->nc, nd = u->nd, nbp = u->nbp, nbf = (long long)u->bface.size();
  const size_t eb = u->prec == BTE_FP64 ? 8 : (u->prec == BTE_FP32 ? 4 : 2);
  for (int i = 0; i < 3; ++i) {
    char* q = nullptr;
    if ((rc = dalloc(u, &q, (size_t)(nc * nd * nbp) * eb))) return rc;
    u->I[i] = reinterpret_cast<double*>(q);
  }
  if (u->prec == BTE_FP64) {
    if ((rc = dalloc(u, &u->R, (size_t)(nc * nd * nbp)))) return rc;
  } else if ((rc = dalloc(u, &u->Rf, (size_t)(nc * nd * nbp)))) {
    return rc;
  }
  if ((rc = dalloc(u, &u->I0ref, nbp)) || (rc = dalloc(u, &u->ghost_dev, nbf * nbp)) || (rc = dalloc(u, &u->w32_d, nd)))
    return rc;
  if ((rc = dalloc(u, &u->I0cell, nc * nbp)) || (rc = dalloc(u, &u->J, nc * 3 * nbp)) || (rc = dalloc(u, &u->Msum, nc * 3)) ||
      (rc = dalloc(u, &u->Teval, nc)) || (rc = dalloc(u, &u->Tp, nc)) || (rc = dalloc(u, &u->TL, nc)) ||
      (rc = dalloc(u, &u->EL, nc)) || (rc = dalloc(u, &u->ghost, nbf * nbp)) || (rc = dalloc(u, &u->bfT_d, nbf)) ||
      (rc = dalloc(u, &u->S_d, nd * 3)) || (rc = dalloc(u, &u->w_d, nd)) || (rc = dalloc(u, &u->nA_d, u->nf * 3)) ||
      (rc = dalloc(u, &u->vb_d, nbp)) || (rc = dalloc(u, &u->bb_d, nbp)) || (rc = dalloc(u, &u->scratch, nc)) ||
      (rc = dalloc(u, &u->Qb, nbf)) || (rc = dalloc(u, &u->qbuf, nc * 3)) || (rc = dalloc(u, &u->bf_mirror_d, nbf)) || (rc = dalloc(u, &u->bf_axis_d, nbf)) || (rc = dalloc(u, &u->bf_spec_d, nbf)) || (rc = dalloc(u, &u->bscale, nc)) ||
      (rc = dalloc(u, &u->refl_d, 5 * nd)) || (rc = dalloc(u, &u->bface_d, nbf)) || (rc = dalloc(u, &u->owner_d, u->nf)) ||
      (rc = dalloc(u, &u->diff_d, nbf)) || (rc = dalloc(u, &u->fix, nc)) || (rc = dalloc(u, &u->fix_count, 4)) ||
      (rc = dalloc(u, &u->counters, 1)) || (rc = dalloc(u, &u->node_c, nbp * u->ng)) ||
      (rc = dalloc(u, &u->node_C, nbp * u->ng)) || (rc = dalloc(u, &u->a_p, nbp)) || (rc = dalloc(u, &u->a_L, nbp)) ||
      (rc = dalloc(u, &u->inv_v, nbp)) || (rc = dalloc(u, &u->beta_d, nbp)) || (rc = dalloc(u, &u->cf_ptr, nc + 1)))
    return rc;
  // cell -> face entries
  std::vector<int> ptr(nc + 1, 0);
  for (long long f = 0; f < u->nf; ++f) {
    ptr[u->owner[f] + 1]++;
    if (u->nbr[f] >= 0) ptr[u->nbr[f] + 1]++;
  }
  for (long long P = 0; P < nc; ++P) {
    if (ptr[P + 1] > kMaxCellFaces) return ufail(u, BTE_E_ARG, "cell %lld has more than %d faces", P, kMaxCellFaces);
    ptr[P + 1] += ptr[P];
  }
  const long long nent = ptr[nc];
  std::vector<long long> ent_face(nent), ent_cell(nent), ent_up(nent);
  std::vector<int> ent_sign(nent), fill(nc, 0);
  std::vector<long long> bf_of_face(u->nf, -1);
  for (long long k = 0; k < nbf; ++k) bf_of_face[u->bface[k]] = k;
  for (long long f = 0; f < u->nf; ++f) {
    const long long Pa = u->owner[f], Pb = u->nbr[f];
    long long e = ptr[Pa] + fill[Pa]++;
    ent_face[e] = f; ent_cell[e] = Pa; ent_sign[e] = 1;
    ent_up[e] = Pb >= 0 ? Pb : -1 - bf_of_face[f];
    if (Pb >= 0) {
      e = ptr[Pb] + fill[Pb]++;
      ent_face[e] = f; ent_cell[e] = Pb; ent_sign[e] = -1; ent_up[e] = Pa;
    }
  }
  long long *ef_d = nullptr, *ec_d = nullptr;
  int* es_d = nullptr;
  if ((rc = dalloc(u, &u->cf_up, nent)) || (rc = dalloc(u, &u->g, nent * nd)) || (rc = dalloc(u, &u->gout, nc * nd)) ||
      (rc = dalloc(u, &ef_d, nent)) || (rc = dalloc(u, &ec_d, nent)) || (rc = dalloc(u, &es_d, nent)))
    return rc;
  cudaStream_t s = u->stream;
  double* vol_d = nullptr;
  if ((rc = dalloc(u, &vol_d, nc))) return rc;
  if ((rc = upload(u, u->cf_ptr, ptr.data(), nc + 1)) || (rc = upload(u, u->cf_up, ent_up.data(), nent)) ||
      (rc = upload(u, ef_d, ent_face.data(), nent)) || (rc = upload(u, ec_d, ent_cell.data(), nent)) ||
      (rc = upload(u, es_d, ent_sign.data(), nent)) || (rc = upload(u, vol_d, u->vol.data(), nc)) ||
      (rc = upload(u, u->nA_d, u->nA.data(), u->nf * 3)) || (rc = upload(u, u->S_d, u->S.data(), nd * 3)) ||
      (rc = upload(u, u->w_d, u->w.data(), nd)) || (rc = upload(u, u->refl_d, u->refl.data(), 5 * nd)) ||
      (rc = upload(u, u->bface_d, u->bface.data(), nbf)) || (rc = upload(u, u->owner_d, u->owner.data(), u->nf)))
    return rc;
  umesh_geom_kernel<<<grid_for(nent * nd, 256), 256, 0, s>>>(ef_d, es_d, ec_d, u->nA_d, vol_d, u->S_d, u->w_d, (int)nd,
                                                             nent, u->g);
  UTRY(u, cudaGetLastError());
  umesh_gout_kernel<<<grid_for(nc * nd, 256), 256, 0, s>>>(u->cf_ptr, u->g, (int)nd, nc, u->gout);
  UTRY(u, cudaGetLastError());
  if (u->prec != BTE_FP64) {
    if ((rc = dalloc(u, &u->g32, nent * nd))) return rc;
    to_float_kernel<<<grid_for(nent * nd, 256), 256, 0, s>>>(u->g, nent * nd, u->g32);
    UTRY(u, cudaGetLastError());
  }
  // band tables
  std::vector<double> nC, nCC, ap, aL, iv, be;
  build_thermo(u->nb, u->nbp, u->ng, u->wlo.data(), u->whi.data(), u->vg.data(), u->beta.data(), u->deg.data(), u->Wtot,
               nC, nCC, ap, aL, iv, be);
  std::vector<double> vbp(nbp, 0.0), bbp(nbp, 0.0);
  for (int b = 0; b < u->nb; ++b) { vbp[b] = u->vg[b]; bbp[b] = u->beta[b]; }
  if ((rc = upload(u, u->node_c, nC.data(), nC.size())) || (rc = upload(u, u->node_C, nCC.data(), nCC.size())) ||
      (rc = upload(u, u->a_p, ap.data(), ap.size())) || (rc = upload(u, u->a_L, aL.data(), aL.size())) ||
      (rc = upload(u, u->inv_v, iv.data(), iv.size())) || (rc = upload(u, u->beta_d, be.data(), be.size())) ||
      (rc = upload(u, u->vb_d, vbp.data(), nbp)) || (rc = upload(u, u->bb_d, bbp.data(), nbp)))
    return rc;
  for (int i = 0; i < 3; ++i) UTRY(u, cudaMemsetAsync(u->I[i], 0, (size_t)(nc * nd * nbp) * eb, s));
  UTRY(u, cudaMemsetAsync(u->ghost, 0, (size_t)std::max(nbf * nbp, 1LL) * 8, s));
  UTRY(u, cudaMemsetAsync(u->ghost_dev, 0, (size_t)std::max(nbf * nbp, 1LL) * 4, s));
  {
    std::vector<float> w32(u->w.begin(), u->w.end());
    if ((rc = upload(u, u->w32_d, w32.data(), nd))) return rc;
    // I0_b(T_ref): the reference the reduced storage keeps deviations from
    const double tref = u->opts.T_ref;
    if ((rc = upload(u, u->scratch, &tref, 1))) return rc;
    UTRY(u, launch_wall_I0(u->I0ref, u->scratch, 1, uthermo(u), s));
  }
  UTRY(u, cudaMemsetAsync(u->counters, 0, sizeof(DevCounters), s));
  UTRY(u, cudaMemsetAsync(u->fix_count, 0, 4, s));
  UTRY(u, cudaStreamSynchronize(s));
  u->lpc = u->nbp / values_per_lane(u->prec);
  u->dteam = std::max(1, std::min(256 / u->lpc, u->nd));
  u->mem_ready = true;
  return BTE_OK;
}

// map[d] = e with S_e = R_z(phi) S_d (rotation about the z axis), matched to
// 1e-9 of |S_d|; false when some direction has no image in the set.
bool rotation_map(const std::vector<double>& S, int nd, double phi, int* map) {
  const double c = std::cos(phi), s = std::sin(phi);
  for (int d = 0; d < nd; ++d) {
    const double* v = &S[3 * d];
    const double r[3] = {c * v[0] - s * v[1], s * v[0] + c * v[1], v[2]};
    const double tol = 1e-9 * std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    map[d] = -1;
    for (int e = 0; e < nd && map[d] < 0; ++e) {
      const double* q = &S[3 * e];
      const double dx = q[0] - r[0], dy = q[1] - r[1], dz = q[2] - r[2];
      if (std::sqrt(dx * dx + dy * dy + dz * dz) <= tol) map[d] = e;
    }
    if (map[d] < 0) return false;
  }
  return true;
}

// Ghost rows of the boundary faces: isothermal I0_b(T_face) and the mirror /
// ghost selector of each face (after every tag has a condition).
int upload_bc(bte_umesh_ctx* u) {
  const long long nbf = (long long)u->bface.size();
  std::vector<int> mirror(nbf), diff;
  std::vector<long long> diffl;
  std::vector<double> T(nbf), spec(nbf, 0.0);
  for (long long k = 0; k < nbf; ++k) {
    const int t = u->bf_type[k];
    mirror[k] = (t == BTE_BC_SPECULAR || t == BTE_BC_ROTATIONAL) ? 1 : (t == BTE_BC_PARTIAL ? 2 : 0);
    T[k] = t == BTE_BC_ISOTHERMAL ? u->bf_T[k] : u->opts.T_ref;
    if (t == BTE_BC_PARTIAL) spec[k] = u->bf_p[k];
    if (t == BTE_BC_DIFFUSE || t == BTE_BC_PARTIAL) diffl.push_back(k);
  }
  int rc;
  if ((rc = upload(u, u->bf_mirror_d, mirror.data(), nbf)) || (rc = upload(u, u->bf_axis_d, u->bf_axis.data(), nbf)) ||
      (rc = upload(u, u->refl_d, u->refl.data(), 5 * (size_t)u->nd)) ||
      (rc = upload(u, u->bf_spec_d, spec.data(), nbf)) ||
      (rc = upload(u, u->bfT_d, T.data(), nbf)) || (rc = upload(u, u->diff_d, diffl.data(), diffl.size())))
    return rc;
  u->ndiff = (int)diffl.size();
  if (nbf > 0) UTRY(u, launch_wall_I0(u->ghost, u->bfT_d, nbf, uthermo(u), u->stream));
  if (nbf > 0 && u->prec != BTE_FP64) UTRY(u, launch_wall_dev(u->ghost_dev, u->ghost, u->I0ref, nbf, u->nbp, u->stream));
  UTRY(u, cudaStreamSynchronize(u->stream));
  return BTE_OK;
}

cudaError_t refresh_diffuse(bte_umesh_ctx* u, const void* I) {
  if (u->ndiff == 0) return cudaSuccess;
  const int grid = (int)std::min<long long>(u->ndiff, 152LL * 16);
  const size_t sm = (size_t)kDiffWarps * 2 * u->nbp * sizeof(double);
  if (u->prec == BTE_FP64)
    umesh_diffuse_kernel<double><<<grid, 32 * kDiffWarps, sm, u->stream>>>(
        (const double*)I, u->diff_d, u->ndiff, u->bface_d, u->owner_d, u->nA_d, u->S_d, u->nd, u->nbp, u->bf_spec_d,
        u->ghost, nullptr);
  else if (u->prec == BTE_FP32)
    umesh_diffuse_kernel<float><<<grid, 32 * kDiffWarps, sm, u->stream>>>(
        (const float*)I, u->diff_d, u->ndiff, u->bface_d, u->owner_d, u->nA_d, u->S_d, u->nd, u->nbp, u->bf_spec_d,
        nullptr, u->ghost_dev);
  else
    umesh_diffuse_kernel<__nv_bfloat16><<<grid, 32 * kDiffWarps, sm, u->stream>>>(
        (const __nv_bfloat16*)I, u->diff_d, u->ndiff, u->bface_d, u->owner_d, u->nA_d, u->S_d, u->nd, u->nbp,
        u->bf_spec_d, nullptr, u->ghost_dev);
  return cudaGetLastError();
}

int ensure_TL(bte_umesh_ctx* u) {
  if (u->TL_valid) return BTE_OK;
  UTRY(u, launch_solve_TL(u->TL, u->EL, u->solve_tp ? u->Tp : u->TL, u->J, u->Teval, u->nc, uthermo(u),
                          std::cbrt(u->opts.newton_rtol / 4.0), u->opts.newton_maxit, u->counters, u->stream));
  u->TL_valid = true;
  return BTE_OK;
}

}  // namespace

extern "C" {

int bte_umesh_create(const bte_umesh_desc* m, const bte_opts* opts, bte_umesh* out) {
  if (!out) return ufail(nullptr, BTE_E_ARG, "out is NULL");
  *out = nullptr;
  if (!m || !m->volume || !m->owner || !m->neighbor || !m->nA || !m->tag)
    return ufail(nullptr, BTE_E_ARG, "mesh description or one of its arrays is NULL");
  if (m->dim != 2 && m->dim != 3) return ufail(nullptr, BTE_E_ARG, "dim must be 2 or 3");
  if (m->ncells < 1 || m->nfaces < 1 || m->ncells > (1LL << 31) - 2)
    return ufail(nullptr, BTE_E_ARG, "need ncells >= 1 (< 2^31) and nfaces >= 1");
  bte_opts o;
  bte_default_opts(&o);
  if (opts) o = *opts;
  if (o.precision != BTE_FP64 && o.precision != BTE_FP32 && o.precision != BTE_BF16)
    return ufail(nullptr, BTE_E_ARG, "unknown precision %d", o.precision);
  if (o.learned) return ufail(nullptr, BTE_E_ARG, "learned mode is not offered here");
  if (!(std::fabs(o.beta_T_exp) <= 16.0)) return ufail(nullptr, BTE_E_ARG, "beta_T_exp must lie in [-16, 16]");
  if (o.n_gauss < 1 || o.n_gauss > kMaxGauss) return ufail(nullptr, BTE_E_ARG, "n_gauss must be in [1, %d]", kMaxGauss);
  for (long long P = 0; P < m->ncells; ++P)
    if (!(std::isfinite(m->volume[P]) && m->volume[P] > 0)) return ufail(nullptr, BTE_E_ARG, "cell %lld: volume must be > 0", P);
  for (long long f = 0; f < m->nfaces; ++f) {
    if (m->owner[f] < 0 || m->owner[f] >= m->ncells) return ufail(nullptr, BTE_E_ARG, "face %lld: bad owner", f);
    if (m->neighbor[f] < -1 || m->neighbor[f] >= m->ncells || m->neighbor[f] == m->owner[f])
      return ufail(nullptr, BTE_E_ARG, "face %lld: bad neighbour", f);
    for (int c = 0; c < 3; ++c)
      if (!std::isfinite(m->nA[3 * f + c])) return ufail(nullptr, BTE_E_ARG, "face %lld: area vector not finite", f);
    if (m->dim == 2 && m->nA[3 * f + 2] != 0.0) return ufail(nullptr, BTE_E_ARG, "face %lld: 2-D area vectors need z = 0", f);
    if (m->neighbor[f] < 0 && m->tag[f] < 0) return ufail(nullptr, BTE_E_ARG, "boundary face %lld: tag must be >= 0", f);
  }
  auto* u = new bte_umesh_ctx();
  u->opts = o;
  u->prec = o.precision;
  u->stream = (cudaStream_t)o.cuda_stream;
  u->dim = m->dim;
  u->nc = m->ncells;
  u->nf = m->nfaces;
  u->vol.assign(m->volume, m->volume + m->ncells);
  u->owner.assign(m->owner, m->owner + m->nfaces);
  u->nbr.assign(m->neighbor, m->neighbor + m->nfaces);
  u->nA.assign(m->nA, m->nA + 3 * m->nfaces);
  u->tag.assign(m->tag, m->tag + m->nfaces);
  for (long long f = 0; f < u->nf; ++f) {
    if (u->nbr[f] >= 0) continue;
    u->bface.push_back(f);
    u->bf_tag.push_back(u->tag[f]);
    u->bf_type.push_back(-1);
    u->bf_T.push_back(0.0);
    u->bf_p.push_back(0.0);
    const double* a = &u->nA[3 * f];
    int ax = 0;
    for (int c = 1; c < 3; ++c)
      if (std::fabs(a[c]) > std::fabs(a[ax])) ax = c;
    const double off = std::sqrt(a[(ax + 1) % 3] * a[(ax + 1) % 3] + a[(ax + 2) % 3] * a[(ax + 2) % 3]);
    u->bf_axis.push_back(ax);
    u->bf_geo_axis.push_back(ax);
    u->bf_ok_axis.push_back(off <= 1e-12 * std::fabs(a[ax]) ? 1 : 0);
    if (std::find(u->tags.begin(), u->tags.end(), u->tag[f]) == u->tags.end()) u->tags.push_back(u->tag[f]);
  }
  u->tag_set.assign(u->tags.size(), 0);
  int rc = o.dir_kind == BTE_DIRS_INPLANE ? build_dirs_inplane(o.n_inplane, u->S, u->w, u->refl)
         : o.dir_kind == BTE_DIRS_POLAR_AZIM ? build_dirs_polar_azim(o.n_polar, o.n_azim, u->S, u->w, u->refl)
         : BTE_E_ARG;
  if (rc != 0) {
    delete u;
    return ufail(nullptr, BTE_E_ARG, "bad direction set");
  }
  u->nd = (int)u->w.size();
  u->refl.resize(5 * (size_t)u->nd);
  for (int d = 0; d < u->nd; ++d) u->refl[3 * u->nd + d] = u->refl[4 * u->nd + d] = d;  // until a rotation is set
  if (m->fc) u->fc.assign(m->fc, m->fc + 3 * m->nfaces);
  if (u->nd > 2048) {
    delete u;
    return ufail(nullptr, BTE_E_ARG, "at most 2048 directions");
  }
  u->Wtot = 0.0;
  for (double x : u->w) u->Wtot += x;
  u->ng = o.n_gauss;
  cudaEventCreate(&u->ev0);
  cudaEventCreate(&u->ev1);
  *out = u;
  return BTE_OK;
}

int bte_umesh_set_bands(bte_umesh u, int nb, const double* wlo, const double* whi, const double* vg, const double* beta,
                        const double* deg) {
  if (!u) return BTE_E_ARG;
  if (u->bands_set) return ufail(u, BTE_E_STATE, "bands are already set");
  if (nb < 1 || nb > kMaxBands || !wlo || !whi || !vg || !beta || !deg)
    return ufail(u, BTE_E_ARG, "need 1 <= nb <= %d and five band arrays", kMaxBands);
  for (int b = 0; b < nb; ++b) {
    if (!(std::isfinite(wlo[b]) && std::isfinite(whi[b]) && wlo[b] >= 0 && whi[b] > wlo[b]))
      return ufail(u, BTE_E_ARG, "band %d: need 0 <= omega_lo < omega_hi", b);
    if (!(std::isfinite(vg[b]) && vg[b] > 0)) return ufail(u, BTE_E_ARG, "band %d: vg must be > 0", b);
    if (!(std::isfinite(beta[b]) && beta[b] >= 0)) return ufail(u, BTE_E_ARG, "band %d: beta must be >= 0", b);
    if (!(std::isfinite(deg[b]) && deg[b] > 0)) return ufail(u, BTE_E_ARG, "band %d: degeneracy must be > 0", b);
  }
  u->nb = nb;
  u->nbp = (nb + 7) / 8 * 8;
  u->wlo.assign(wlo, wlo + nb);
  u->whi.assign(whi, whi + nb);
  u->vg.assign(vg, vg + nb);
  u->beta.assign(beta, beta + nb);
  u->deg.assign(deg, deg + nb);
  u->solve_tp = false;
  for (int b = 0; b < nb; ++b) u->solve_tp |= beta[b] > 0;
  u->bands_set = true;
  return ensure_mem(u);
}

int bte_umesh_set_bc(bte_umesh u, int tag, int type, const double* T_faces, double T_uniform) {
  if (!u) return BTE_E_ARG;
  if (!u->mem_ready) return ufail(u, BTE_E_STATE, "bte_umesh_set_bands must come first");
  const auto it = std::find(u->tags.begin(), u->tags.end(), tag);
  if (it == u->tags.end()) return ufail(u, BTE_E_ARG, "no boundary face has tag %d", tag);
  if (type != BTE_BC_ISOTHERMAL && type != BTE_BC_SPECULAR && type != BTE_BC_DIFFUSE && type != BTE_BC_PARTIAL &&
      type != BTE_BC_ROTATIONAL)
    return ufail(u, BTE_E_ARG, "unknown boundary type %d", type);
  std::vector<int> rot(2 * (size_t)u->nd);
  if (type == BTE_BC_ROTATIONAL) {
    const double alpha = T_uniform;
    if (u->fc.empty()) return ufail(u, BTE_E_ARG, "tag %d: rotational faces need the face centres (fc) of the mesh", tag);
    if (!(std::isfinite(alpha) && alpha > 0.0 && alpha < kPi))
      return ufail(u, BTE_E_ARG, "tag %d: the wedge angle must lie in (0, pi)", tag);
    if (u->rot_alpha != 0.0 && u->rot_alpha != alpha)
      return ufail(u, BTE_E_ARG, "tag %d: every rotational tag takes the same wedge angle (%g set before)", tag,
                   u->rot_alpha);
    if (!rotation_map(u->S, u->nd, -alpha, rot.data()) || !rotation_map(u->S, u->nd, alpha, rot.data() + u->nd))
      return ufail(u, BTE_E_ARG, "tag %d: a rotation by %g rad does not map the direction set onto itself", tag, alpha);
  }
  for (size_t k = 0; k < u->bface.size(); ++k) {
    if (u->bf_tag[k] != tag) continue;
    if (type == BTE_BC_ROTATIONAL) {  // a plane through the z axis
      const double* a = &u->nA[3 * u->bface[k]];
      const double* c = &u->fc[3 * u->bface[k]];
      const double an = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
      const double cr = std::sqrt(c[0] * c[0] + c[1] * c[1]);
      if (!(cr > 0.0) || std::fabs(a[2]) > 1e-12 * an || std::fabs(a[0] * c[0] + a[1] * c[1]) > 1e-9 * an * cr)
        return ufail(u, BTE_E_ARG, "tag %d: face %lld is not a plane through the z axis", tag, u->bface[k]);
    }
    if ((type == BTE_BC_SPECULAR || type == BTE_BC_PARTIAL) && !u->bf_ok_axis[k])
      return ufail(u, BTE_E_ARG, "tag %d: face %lld is not normal to an axis (a mirror needs that)", tag, u->bface[k]);
    if (type == BTE_BC_PARTIAL) {
      const double p = T_faces ? T_faces[u->bface[k]] : T_uniform;
      if (!(p >= 0.0 && p <= 1.0)) return ufail(u, BTE_E_ARG, "tag %d: specularity must lie in [0, 1]", tag);
    }
    if (type == BTE_BC_ISOTHERMAL) {
      const double T = T_faces ? T_faces[u->bface[k]] : T_uniform;
      if (!(std::isfinite(T) && T >= kTmin && T <= kTmax))
        return ufail(u, BTE_E_ARG, "tag %d: face temperatures must lie in [1, 5000] K", tag);
    }
  }
  for (size_t k = 0; k < u->bface.size(); ++k) {
    if (u->bf_tag[k] != tag) continue;
    u->bf_type[k] = type;
    u->bf_T[k] = type == BTE_BC_ISOTHERMAL ? (T_faces ? T_faces[u->bface[k]] : T_uniform) : 0.0;
    u->bf_p[k] = type == BTE_BC_PARTIAL ? (T_faces ? T_faces[u->bface[k]] : T_uniform) : 0.0;
    u->bf_axis[k] = u->bf_geo_axis[k];
    if (type == BTE_BC_ROTATIONAL) {  // outward along +e_theta: the far side, ghost rotated back by -alpha (row 3)
      const double* a = &u->nA[3 * u->bface[k]];
      const double* c = &u->fc[3 * u->bface[k]];
      u->bf_axis[k] = (-c[1] * a[0] + c[0] * a[1]) > 0.0 ? 3 : 4;
    }
  }
  if (type == BTE_BC_ROTATIONAL) {
    u->rot_alpha = T_uniform;
    std::copy(rot.begin(), rot.end(), u->refl.begin() + 3 * (size_t)u->nd);
  }
  u->tag_set[it - u->tags.begin()] = 1;
  for (char c : u->tag_set)
    if (!c) return BTE_OK;
  return upload_bc(u);
}

int bte_umesh_set_initial(bte_umesh u, const double* T_cells, double T_uniform) {
  if (!u) return BTE_E_ARG;
  if (!u->mem_ready) return ufail(u, BTE_E_STATE, "bte_umesh_set_bands must come first");
  std::vector<double> T(u->nc);
  for (long long P = 0; P < u->nc; ++P) {
    T[P] = T_cells ? T_cells[P] : T_uniform;
    if (!(std::isfinite(T[P]) && T[P] >= kTmin && T[P] <= kTmax))
      return ufail(u, BTE_E_ARG, "cell %lld: temperature must lie in [1, 5000] K", P);
  }
  int rc = upload(u, u->scratch, T.data(), u->nc);
  if (rc) return rc;
  u->cur = 0;
  UTRY(u, launch_init_cells(u->prec, u->I[0], u->I0cell, u->J, u->Msum, u->Tp, u->Teval, u->TL, u->EL, u->scratch, u->I0ref, 0,
                            (int)u->nc, u->nd, uthermo(u), u->stream));
  UTRY(u, cudaStreamSynchronize(u->stream));
  u->init_done = true;
  u->TL_valid = true;
  return BTE_OK;
}

int bte_umesh_step(bte_umesh u, double dt, int nsteps, int ninner, int scheme, bte_stats* stats) {
  if (!u) return BTE_E_ARG;
  if (!u->init_done) return ufail(u, BTE_E_STATE, "bte_umesh_set_initial must come first");
  for (char c : u->tag_set)
    if (!c) return ufail(u, BTE_E_STATE, "every boundary tag needs bte_umesh_set_bc");
  if (!(dt > 0 && std::isfinite(dt))) return ufail(u, BTE_E_ARG, "dt must be > 0");
  if (nsteps < 0) return ufail(u, BTE_E_ARG, "nsteps must be >= 0");
  if (scheme != BTE_IMPLICIT_JACOBI && scheme != BTE_EXPLICIT) return ufail(u, BTE_E_ARG, "unknown scheme %d", scheme);
  if (scheme == BTE_EXPLICIT) ninner = 1;
  if (ninner < 1) return ufail(u, BTE_E_ARG, "ninner must be >= 1");
  cudaStream_t s = u->stream;
  if (scheme != BTE_EXPLICIT && u->R_dt != dt) {
    const int gr = grid_for(u->nc * u->nd * u->nbp, 256);
    if (u->prec == BTE_FP64)
      umesh_rcp_kernel<double><<<gr, 256, 0, s>>>(u->gout, u->vb_d, u->bb_d, 1.0 / dt, u->nc, u->nd, u->nbp, u->R);
    else
      umesh_rcp_kernel<float><<<gr, 256, 0, s>>>(u->gout, u->vb_d, u->bb_d, 1.0 / dt, u->nc, u->nd, u->nbp, u->Rf);
    UTRY(u, cudaGetLastError());
    u->R_dt = dt;
  }
  if (stats) {
    UTRY(u, cudaMemsetAsync(u->counters, 0, sizeof(DevCounters), s));
    UTRY(u, cudaEventRecord(u->ev0, s));
  }
  UArgs a{};
  a.R = u->R;
  a.Rf = u->Rf;
  a.g32 = u->g32;
  a.ghost_dev = u->ghost_dev;
  a.I0ref = u->I0ref;
  a.I0cell = u->I0cell;
  a.ghost = u->ghost;
  a.cf_ptr = u->cf_ptr;
  a.cf_up = u->cf_up;
  a.g = u->g;
  a.gout = u->gout;
  a.bf_mirror = u->bf_mirror_d;
  a.bf_axis = u->bf_axis_d;
  a.bf_spec = u->bf_spec_d;
  a.refl = u->refl_d;
  a.vb = u->vb_d;
  a.bb = u->bb_d;
  a.dt = dt;
  a.rdt = 1.0 / dt;
  a.nc = u->nc;
  a.nd = u->nd;
  a.nbp = u->nbp;
  a.lpc = u->lpc;
  a.dteam = u->dteam;
  const int threads = (256 / (u->lpc * u->dteam)) * u->lpc * u->dteam;
  const int cpb = threads / (u->lpc * u->dteam);
  const int grid = (int)std::min<long long>((u->nc + cpb - 1) / cpb, 65535);
  int launches = 0;
  // implicit steps of two or more inner iterations keep B = (I^n/dt) R in the
  // third buffer: iteration 0 reads I^n and writes I^1 and B; iteration k reads
  // B and I^k and overwrites the buffer I^n (or I^{k-2}) was in
  const bool use_b = scheme != BTE_EXPLICIT && ninner >= 2;
  const bool tt = u->opts.beta_T_exp != 0.0 && u->solve_tp;  // tau(T); with every beta_b = 0 there is no relaxation
  a.bscale = tt ? u->bscale : nullptr;
  for (int st = 0; st < nsteps; ++st) {
    const int n = u->cur;
    int k = n, z = -1;
    for (int it = 0; it < ninner; ++it) {
      int o = 0, bm = 0;
      if (use_b && it == 0) {
        while (o == n) ++o;
        z = 0;
        while (z == n || z == o) ++z;
        a.In = u->I[n];
        a.Bout = u->I[z];
        bm = 1;
      } else if (use_b) {
        while (o == z || o == k) ++o;
        a.In = u->I[z];
        bm = 2;
      } else {
        while (o == n || o == k) ++o;
        a.In = u->I[n];
      }
      a.Ik = u->I[k];
      a.Iout = u->I[o];
      a.Ind = a.In;
      a.Ikd = a.Ik;
      a.Ioutd = a.Iout;
      a.Boutd = a.Bout;
      UTRY(u, cudaMemsetAsync(u->fix_count, 0, 4, s));
      UTRY(u, refresh_diffuse(u, a.Ik));
      if (tt) {  // beta_b(T_p) of the current T_p, as the oracle takes it
        UTRY(u, launch_beta_scale(u->bscale, u->Tp, u->opts.T_ref, u->opts.beta_T_exp, u->nc, s));
        UTRY(u, launch_umesh_sweep<true>(u->prec, scheme == BTE_EXPLICIT, bm, a, grid, threads, s));
      } else {
        UTRY(u, launch_umesh_sweep<false>(u->prec, scheme == BTE_EXPLICIT, bm, a, grid, threads, s));
      }
      SweepArgs c = cell_args(u, a.Iout);
      UTRY(u, launch_gs_reduce(u->prec, c, u->nc, s));
      if (u->solve_tp) UTRY(u, launch_fixup(c, nullptr, s));
      launches += 2 + (u->solve_tp ? 1 : 0) + (u->ndiff ? 1 : 0) + (tt ? 1 : 0);
      k = o;
    }
    u->cur = k;
  }
  if (nsteps > 0) u->TL_valid = false;
  if (stats) {
    UTRY(u, cudaEventRecord(u->ev1, s));
    UTRY(u, cudaEventSynchronize(u->ev1));
    DevCounters c;
    UTRY(u, cudaMemcpy(&c, u->counters, sizeof c, cudaMemcpyDeviceToHost));
    float ms = 0.f;
    UTRY(u, cudaEventElapsedTime(&ms, u->ev0, u->ev1));
    stats->updates = u->nc * u->nd * (long long)u->nb * ninner * nsteps;
    stats->solve_evals = (long long)c.evals;
    stats->solves = (long long)c.solves;
    stats->fallbacks = (long long)c.fallbacks;
    stats->nonfinite = (long long)c.nonfinite;
    stats->launches = launches;
    stats->gpu_ms = ms;
    if (c.nonfinite) return ufail(u, BTE_E_NONFINITE, "%llu cells had a non-finite energy or no temperature in [1, 5000] K",
                                  (unsigned long long)c.nonfinite);
    if (c.fallbacks) return BTE_W_FALLBACK;
  }
  return BTE_OK;
}

int bte_umesh_get_T(bte_umesh u, int which, double* out, int on_device) {
  if (!u || !out) return u ? ufail(u, BTE_E_ARG, "out is NULL") : BTE_E_ARG;
  if (!u->init_done) return ufail(u, BTE_E_STATE, "no state");
  if (which != BTE_T_PSEUDO && which != BTE_T_LATTICE) return ufail(u, BTE_E_ARG, "bad which");
  const double* src = u->Tp;
  if (which == BTE_T_LATTICE) {
    int rc = ensure_TL(u);
    if (rc) return rc;
    src = u->TL;
  }
  if (which == BTE_T_PSEUDO && !u->solve_tp) {  // every beta_b = 0: T_p is T_L
    int rc = ensure_TL(u);
    if (rc) return rc;
    src = u->TL;
  }
  UTRY(u, cudaMemcpyAsync(out, src, u->nc * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, u->stream));
  UTRY(u, cudaStreamSynchronize(u->stream));
  return BTE_OK;
}

int bte_umesh_get_intensity(bte_umesh u, double* out) {
  if (!u || !out) return u ? ufail(u, BTE_E_ARG, "out is NULL") : BTE_E_ARG;
  if (!u->init_done) return ufail(u, BTE_E_STATE, "no state");
  if (u->prec == BTE_FP64) {
    UTRY(u, cudaMemcpy2DAsync(out, (size_t)u->nb * 8, u->I[u->cur], (size_t)u->nbp * 8, (size_t)u->nb * 8,
                              (size_t)(u->nc * u->nd), cudaMemcpyDeviceToHost, u->stream));
    UTRY(u, cudaStreamSynchronize(u->stream));
    return BTE_OK;
  }
  // reduced storage: full FP64 values (I0_b(T_ref) + deviation) through a temporary device buffer
  double* tmp = nullptr;
  const size_t n = (size_t)(u->nc * u->nd) * u->nb;
  cudaError_t e = cudaMalloc(&tmp, n * 8);
  if (e != cudaSuccess) return ufail(u, BTE_E_NOMEM, "cudaMalloc(%zu bytes): %s", n * 8, cudaGetErrorString(e));
  e = launch_pack(u->prec, nullptr, tmp, u->I[u->cur], nullptr, u->I0ref, u->nc, u->nd, u->nb, u->nbp, 0, u->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, tmp, n * 8, cudaMemcpyDeviceToHost, u->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(u->stream);
  cudaFree(tmp);
  if (e != cudaSuccess) return ufail(u, BTE_E_CUDA, "reading the intensities: %s", cudaGetErrorString(e));
  return BTE_OK;
}

int bte_umesh_set_intensity(bte_umesh u, const double* in, const double* Tp_cells) {
  if (!u) return BTE_E_ARG;
  if (!in || !Tp_cells) return ufail(u, BTE_E_ARG, "in and Tp_cells are required");
  if (!u->init_done) return ufail(u, BTE_E_STATE, "bte_umesh_set_initial must come first");
  for (long long P = 0; P < u->nc; ++P)
    if (!(std::isfinite(Tp_cells[P]) && Tp_cells[P] >= kTmin && Tp_cells[P] <= kTmax))
      return ufail(u, BTE_E_ARG, "cell %lld: T_p must lie in [1, 5000] K", P);
  cudaStream_t s = u->stream;
  const size_t n = (size_t)(u->nc * u->nd) * u->nb;
  double* tmp = nullptr;
  cudaError_t e = cudaMalloc(&tmp, n * 8);
  if (e != cudaSuccess) return ufail(u, BTE_E_NOMEM, "cudaMalloc(%zu bytes): %s", n * 8, cudaGetErrorString(e));
  e = cudaMemcpyAsync(tmp, in, n * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = launch_pack(u->prec, tmp, nullptr, nullptr, u->I[u->cur], u->I0ref, u->nc, u->nd, u->nb, u->nbp, 1, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(u->Tp, Tp_cells, u->nc * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = launch_state_from_Tp(u->I0cell, u->J, u->Msum, u->Tp, u->Teval, u->nc, uthermo(u), s);
  if (e == cudaSuccess) e = launch_energy_L(u->prec, u->I[u->cur], u->I0ref, u->EL, u->w_d, u->nc, u->nd, uthermo(u), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(tmp);
  if (e != cudaSuccess) return ufail(u, BTE_E_CUDA, "restoring the state: %s", cudaGetErrorString(e));
  u->TL_valid = false;
  return BTE_OK;
}

int bte_umesh_get_flux(bte_umesh u, double* q, double* Q) {
  if (!u) return BTE_E_ARG;
  if (!u->init_done) return ufail(u, BTE_E_STATE, "no state");
  cudaStream_t s = u->stream;
  const double* I = u->I[u->cur];
  if (q) {
    UTRY(u, launch_flux_cells(u->prec, I, u->I0ref, u->qbuf, u->S_d, 0, (int)u->nc, u->nd, u->nbp, 3, s));
    UTRY(u, cudaMemcpyAsync(q, u->qbuf, (size_t)u->nc * 3 * 8, cudaMemcpyDeviceToHost, s));
    UTRY(u, cudaStreamSynchronize(s));
  }
  if (Q) {
    const long long nbf = (long long)u->bface.size();
    UTRY(u, refresh_diffuse(u, I));
    if (nbf > 0) {
      const int gr = grid_for(nbf, 4);
      if (u->prec == BTE_FP64)
        umesh_face_flux_kernel<double><<<gr, 128, 0, s>>>((const double*)I, u->I0ref, u->ghost, u->ghost_dev, u->bface_d,
                                                          nbf, u->owner_d, u->nA_d, u->bf_mirror_d, u->bf_axis_d, u->bf_spec_d,
                                                          u->refl_d, u->S_d, u->nd, u->nbp, u->nb, u->Qb);
      else if (u->prec == BTE_FP32)
        umesh_face_flux_kernel<float><<<gr, 128, 0, s>>>((const float*)I, u->I0ref, u->ghost, u->ghost_dev, u->bface_d,
                                                         nbf, u->owner_d, u->nA_d, u->bf_mirror_d, u->bf_axis_d, u->bf_spec_d,
                                                         u->refl_d, u->S_d, u->nd, u->nbp, u->nb, u->Qb);
      else
        umesh_face_flux_kernel<__nv_bfloat16><<<gr, 128, 0, s>>>((const __nv_bfloat16*)I, u->I0ref, u->ghost,
                                                                 u->ghost_dev, u->bface_d, nbf, u->owner_d, u->nA_d,
                                                                 u->bf_mirror_d, u->bf_axis_d, u->bf_spec_d, u->refl_d, u->S_d, u->nd,
                                                                 u->nbp, u->nb, u->Qb);
      UTRY(u, cudaGetLastError());
    }
    std::vector<double> Qb(nbf);
    if (nbf > 0) UTRY(u, cudaMemcpyAsync(Qb.data(), u->Qb, nbf * 8, cudaMemcpyDeviceToHost, s));
    UTRY(u, cudaStreamSynchronize(s));
    for (long long f = 0; f < u->nf; ++f) Q[f] = 0.0;
    for (long long k = 0; k < nbf; ++k) Q[u->bface[k]] = Qb[k];
  }
  return BTE_OK;
}

const char* bte_umesh_last_error(bte_umesh u) { return u ? u->err.c_str() : g_umesh_err.c_str(); }

void bte_umesh_destroy(bte_umesh u) {
  if (!u) return;
  if (u->stream) cudaStreamSynchronize(u->stream);
  for (void* p : u->allocs) cudaFree(p);
  if (u->ev0) cudaEventDestroy(u->ev0);
  if (u->ev1) cudaEventDestroy(u->ev1);
  delete u;
}

}  // extern "C"

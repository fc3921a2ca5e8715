// bte_tables.cpp -- host-side tables of the library (built once per handle,
// uploaded to the workspace).
//
//  * direction sets (Sec. 3.1): in-plane N or polar x azimuthal control
//    angles; S_d is the integral of the unit vector over the control angle,
//    w_d its solid angle.  The sets are built from one octant/quadrant and
//    mirrored, so the wall reflections of Eq. 6 map a direction onto one whose
//    weight and tangential components are bitwise equal and whose normal
//    component is exactly negated; this keeps the specular wall flux balance
//    exact in floating point.
//  * Gauss-Legendre nodes (Newton on the Legendre recurrence),
//  * per-band node tables for I0_b(T) (Debye-type band, Bose-Einstein),
//  * the sweep coefficients of the implicit and explicit updates.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <vector>

#include "bte_internal.h"
#include "bte_tables.h"

namespace bte {

void gauss_legendre(int n, double* x, double* w) {
  const int m = (n + 1) / 2;
  for (int i = 0; i < m; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    double pp = 0.0;
    for (int it = 0; it < 60; ++it) {
      double p1 = 1.0, p2 = 0.0;
      for (int k = 1; k <= n; ++k) {
        const double p3 = p2;
        p2 = p1;
        p1 = ((2.0 * k - 1.0) * z * p2 - (k - 1.0) * p3) / k;
      }
      pp = n * (z * p1 - p2) / (z * z - 1.0);
      const double dz = p1 / pp;
      z -= dz;
      if (std::fabs(dz) < 1e-17) break;
    }
    double p1 = 1.0, p2 = 0.0;
    for (int k = 1; k <= n; ++k) {
      const double p3 = p2;
      p2 = p1;
      p1 = ((2.0 * k - 1.0) * z * p2 - (k - 1.0) * p3) / k;
    }
    pp = n * (z * p1 - p2) / (z * z - 1.0);
    const double wi = 2.0 / ((1.0 - z * z) * pp * pp);
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = wi;
    w[n - 1 - i] = wi;
  }
  if (n % 2) x[n / 2] = 0.0;
}

int build_dirs_inplane(int n, std::vector<double>& S, std::vector<double>& w, std::vector<int>& refl) {
  if (n < 4 || n % 4) return -1;
  S.assign(3 * n, 0.0);
  w.assign(n, 4.0 * kPi / n);
  refl.assign(3 * n, 0);
  const int q = n / 4;
  // first quadrant, then mirror: phi_d = (d + 1/2) 2 pi / n
  for (int d = 0; d < q; ++d) {
    const double phi = (d + 0.5) * 2.0 * kPi / n;
    const double cx = w[d] * std::cos(phi), cy = w[d] * std::sin(phi);
    const int d2 = n / 2 - 1 - d;  // pi - phi
    const int d3 = n / 2 + d;      // pi + phi
    const int d4 = n - 1 - d;      // -phi
    S[3 * d + 0] = cx;   S[3 * d + 1] = cy;
    S[3 * d2 + 0] = -cx; S[3 * d2 + 1] = cy;
    S[3 * d3 + 0] = -cx; S[3 * d3 + 1] = -cy;
    S[3 * d4 + 0] = cx;  S[3 * d4 + 1] = -cy;
  }
  for (int d = 0; d < n; ++d) {
    refl[0 * n + d] = ((n / 2 - 1 - d) % n + n) % n;
    refl[1 * n + d] = n - 1 - d;
    refl[2 * n + d] = d;
  }
  return 0;
}

int build_dirs_polar_azim(int nt, int np, std::vector<double>& S, std::vector<double>& w, std::vector<int>& refl) {
  if (nt < 2 || nt % 2 || np < 4 || np % 4) return -1;
  const int n = nt * np;
  S.assign(3 * n, 0.0);
  w.assign(n, 0.0);
  refl.assign(3 * n, 0);
  const double dth = kPi / nt, dph = 2.0 * kPi / np;
  for (int i = 0; i < nt / 2; ++i) {  // upper hemisphere, mirrored to the lower one
    const double t1 = i * dth, t2 = (i + 1) * dth;
    const double J = 0.5 * (t2 - t1) - 0.25 * (std::sin(2.0 * t2) - std::sin(2.0 * t1));
    const double wt = dph * (std::cos(t1) - std::cos(t2));
    const double sz = 0.5 * dph * (std::sin(t2) * std::sin(t2) - std::sin(t1) * std::sin(t1));
    for (int j = 0; j < np / 4; ++j) {  // first azimuthal quadrant, mirrored to the others
      const double p1 = j * dph, p2 = (j + 1) * dph;
      const double sx = J * (std::sin(p2) - std::sin(p1));
      const double sy = J * (std::cos(p1) - std::cos(p2));
      const int js[4] = {j, np / 2 - 1 - j, np / 2 + j, np - 1 - j};
      const double fx[4] = {1, -1, -1, 1}, fy[4] = {1, 1, -1, -1};
      for (int h = 0; h < 2; ++h) {
        const int ii = h ? nt - 1 - i : i;
        for (int qd = 0; qd < 4; ++qd) {
          const int d = ii * np + js[qd];
          w[d] = wt;
          S[3 * d + 0] = fx[qd] * sx;
          S[3 * d + 1] = fy[qd] * sy;
          S[3 * d + 2] = h ? -sz : sz;
        }
      }
    }
  }
  for (int i = 0; i < nt; ++i)
    for (int j = 0; j < np; ++j) {
      const int d = i * np + j;
      refl[0 * n + d] = i * np + ((np / 2 - 1 - j) % np + np) % np;
      refl[1 * n + d] = i * np + (np - 1 - j);
      refl[2 * n + d] = (nt - 1 - i) * np + j;
    }
  return 0;
}

void build_thermo(int nb, int nbp, int ng, const double* wlo, const double* whi, const double* vg, const double* beta,
                  const double* deg, double Wtot, std::vector<double>& node_c, std::vector<double>& node_C,
                  std::vector<double>& a_p, std::vector<double>& a_L, std::vector<double>& inv_v,
                  std::vector<double>& beta_p) {
  double gx[kMaxGauss], gw[kMaxGauss];
  gauss_legendre(ng, gx, gw);
  node_c.assign((size_t)nbp * ng, 1000.0);  // padding: finite, contributes C = 0
  node_C.assign((size_t)nbp * ng, 0.0);
  a_p.assign(nbp, 0.0);
  a_L.assign(nbp, 0.0);
  inv_v.assign(nbp, 0.0);
  beta_p.assign(nbp, 0.0);
  for (int b = 0; b < nb; ++b) {
    const double half = 0.5 * (whi[b] - wlo[b]), mid = 0.5 * (whi[b] + wlo[b]);
    const double pref = deg[b] * kHbar / (8.0 * kPi * kPi * kPi * vg[b] * vg[b]) * half;
    for (int i = 0; i < ng; ++i) {
      const double om = mid + half * gx[i];
      node_c[(size_t)b * ng + i] = kHbar * om / kBoltz;
      node_C[(size_t)b * ng + i] = pref * gw[i] * om * om * om;
    }
    inv_v[b] = 1.0 / vg[b];
    a_L[b] = Wtot / vg[b];
    a_p[b] = Wtot * beta[b] / vg[b];
    beta_p[b] = beta[b];
  }
}

// Sweep coefficients for one cell-size class: [5][nd][nbp] = A_n, A_x, A_y, A_z, A_s.
void build_coef(int dim, const double delta[3], int nd, const double* S, const double* w, int nb, int nbp,
                const double* vg, const double* beta, double dt, int explicit_scheme, double* out) {
  const size_t plane = (size_t)nd * nbp;
  for (size_t e = 0; e < 5 * plane; ++e) out[e] = 0.0;
  for (int d = 0; d < nd; ++d) {
    double c[3] = {0.0, 0.0, 0.0};
    for (int ax = 0; ax < dim; ++ax) c[ax] = std::fabs(S[3 * d + ax]) / (w[d] * delta[ax]);
    const double csum = c[0] + c[1] + c[2];
    for (int b = 0; b < nb; ++b) {
      const size_t o = (size_t)d * nbp + b;
      if (explicit_scheme) {
        out[o] = 1.0 - dt * (beta[b] + vg[b] * csum);
        for (int ax = 0; ax < 3; ++ax) out[(1 + ax) * plane + o] = dt * vg[b] * c[ax];
        out[4 * plane + o] = dt * beta[b];
      } else {
        const double inv = 1.0 / (1.0 / dt + beta[b] + vg[b] * csum);
        out[o] = inv / dt;
        for (int ax = 0; ax < 3; ++ax) out[(1 + ax) * plane + o] = vg[b] * c[ax] * inv;
        out[4 * plane + o] = beta[b] * inv;
      }
    }
  }
}

namespace {
// Double-double values (hi + lo) for the factored tables.
struct DD {
  double hi, lo;
};
DD dd_of(float h, float l) {  // exact: a float pair is a double-double
  const double a = h, b = l;
  const double s = a + b;
  return {s, b - (s - a)};
}
DD dd_add(DD x, DD y) {
  const double s = x.hi + y.hi;
  const double bv = s - x.hi;
  const double e = (x.hi - (s - bv)) + (y.hi - bv) + x.lo + y.lo;
  const double r = s + e;
  return {r, e - (r - s)};
}
DD dd_mul(DD x, DD y) {
  const double p = x.hi * y.hi;
  const double e = std::fma(x.hi, y.hi, -p) + (std::fma(x.hi, y.lo, 0.0) + std::fma(x.lo, y.hi, 0.0));
  const double r = p + e;
  return {r, e - (r - p)};
}
DD dd_recip(DD d) {  // one Newton step from the double reciprocal
  const double r0 = 1.0 / d.hi;
  const double p = d.hi * r0;
  const double e = ((1.0 - p) - std::fma(d.hi, r0, -p)) - d.lo * r0;
  const double r = r0 + r0 * e;
  return {r, (r0 - r) + r0 * e};
}
void ff_of(double x, float& h, float& l) {
  h = (float)x;
  l = (float)(x - (double)h);
}
void ff_of_dd(DD x, float& h, float& l) {
  h = (float)x.hi;
  l = (float)((x.hi - (double)h) + x.lo);
}
}  // namespace

void build_ff_factored(int dim, const double delta[3], int nd, const double* S, const double* w, int nb, int nbp,
                       const double* vg, const double* beta, double dt, float* R, float* dirc, float* band) {
  for (size_t e = 0; e < 4 * (size_t)nbp; ++e) band[e] = 0.0f;
  std::vector<DD> rv_dd(nb), bv_dd(nb);
  for (int b = 0; b < nb; ++b) {  // pair layout: element b of an [nbp] array at float (b - b%2)*2 + b%2 (+2 for l)
    float h, l;
    const size_t o = (size_t)(b - (b & 1)) * 2 + (b & 1);
    ff_of(1.0 / (vg[b] * dt), h, l);  // 1 / (v_b dt)
    band[o] = h;
    band[o + 2] = l;
    rv_dd[b] = dd_of(h, l);
    ff_of(beta[b] / vg[b], h, l);  // beta_b / v_b
    band[2 * (size_t)nbp + o] = h;
    band[2 * (size_t)nbp + o + 2] = l;
    bv_dd[b] = dd_of(h, l);
  }
  for (size_t e = 0; e < 2 * (size_t)nd * nbp; ++e) R[e] = 0.0f;
  for (int d = 0; d < nd; ++d) {
    DD csum{0.0, 0.0};
    for (int ax = 0; ax < 3; ++ax) {
      const double c = ax < dim ? std::fabs(S[3 * d + ax]) / (w[d] * delta[ax]) : 0.0;
      float h, l;
      ff_of(c, h, l);
      dirc[(size_t)d * 6 + 2 * ax] = h;
      dirc[(size_t)d * 6 + 2 * ax + 1] = l;
      csum = dd_add(csum, dd_of(h, l));
    }
    for (int b = 0; b < nb; ++b) {
      const DD D = dd_add(dd_add(rv_dd[b], bv_dd[b]), csum);
      float h, l;
      ff_of_dd(dd_recip(D), h, l);
      const size_t o = ((size_t)d * nbp + b - (b & 1)) * 2 + (b & 1);
      R[o] = h;
      R[o + 2] = l;
    }
  }
}

// Reduced-precision form of the same update: I' = P I^n + Q (v_b sum_ax c_ax I_up + beta_b I0),
// P and Q per (d, b) as float, c_ax = |S_d,ax|/(w_d Delta_ax) per direction.
//   implicit: Q = 1/(1/dt + beta_b + v_b sum c), P = Q/dt;  explicit: P = 1 - dt(beta_b + v_b sum c), Q = dt.
void build_pq(int dim, const double delta[3], int nd, const double* S, const double* w, int nb, int nbp,
              const double* vg, const double* beta, double dt, int explicit_scheme, float* P, float* Q, float* dirc) {
  for (size_t e = 0; e < (size_t)nd * nbp; ++e) P[e] = Q[e] = 0.0f;
  for (int d = 0; d < nd; ++d) {
    double c[3] = {0.0, 0.0, 0.0};
    for (int ax = 0; ax < dim; ++ax) c[ax] = std::fabs(S[3 * d + ax]) / (w[d] * delta[ax]);
    dirc[4 * d + 0] = (float)c[0];
    dirc[4 * d + 1] = (float)c[1];
    dirc[4 * d + 2] = (float)c[2];
    dirc[4 * d + 3] = (float)(c[0] + c[1] + c[2]);
    const double csum = c[0] + c[1] + c[2];
    for (int b = 0; b < nb; ++b) {
      const size_t o = (size_t)d * nbp + b;
      if (explicit_scheme) {
        P[o] = (float)(1.0 - dt * (beta[b] + vg[b] * csum));
        Q[o] = (float)dt;
      } else {
        const double inv = 1.0 / (1.0 / dt + beta[b] + vg[b] * csum);
        P[o] = (float)(inv / dt);
        Q[o] = (float)inv;
      }
    }
  }
}

}  // namespace bte

// bte_tables.h -- host table builders (bte_tables.cpp).
#pragma once
#include <vector>

namespace bte {

void gauss_legendre(int n, double* x, double* w);
int build_dirs_inplane(int n, std::vector<double>& S, std::vector<double>& w, std::vector<int>& refl);
int build_dirs_polar_azim(int nt, int np, std::vector<double>& S, std::vector<double>& w, std::vector<int>& refl);
void build_thermo(int nb, int nbp, int ng, const double* wlo, const double* whi, const double* vg, const double* beta,
                  const double* deg, double Wtot, std::vector<double>& node_c, std::vector<double>& node_C,
                  std::vector<double>& a_p, std::vector<double>& a_L, std::vector<double>& inv_v,
                  std::vector<double>& beta_p);
void build_coef(int dim, const double delta[3], int nd, const double* S, const double* w, int nb, int nbp,
                const double* vg, const double* beta, double dt, int explicit_scheme, double* out);

// Tables of the factored double-float sweep (bte_sweep_ff.cuh) for one class,
// the implicit update divided through by v_b (v_b > 0 on every real band):
// I' = B + R (sum_ax c_ax,d u_ax + (beta_b / v_b) I0),  B = (1 / (v_b dt)) R I^n,
// R = 1 / (1 / (v_b dt) + beta_b / v_b + sum_ax c_ax,d).
// dirc[nd][3][2] c_ax,d = |S_d,ax|/(w_d Delta_ax) as double-float pairs (h, l);
// band[2][nbp] 1/(v_b dt) and beta_b/v_b and R[nd][nbp] in the pair layout of
// bte_ff.cuh (per two bands h_b, h_b+1, l_b, l_b+1; padding bands 0).  R is the
// double-float pair nearest the reciprocal of a denominator formed exactly
// (double-double) from the stored pairs themselves, so that a uniform field is
// a fixed point of the update to the pairs' resolution.
void build_ff_factored(int dim, const double delta[3], int nd, const double* S, const double* w, int nb, int nbp,
                       const double* vg, const double* beta, double dt, float* R, float* dirc, float* band);

void build_pq(int dim, const double delta[3], int nd, const double* S, const double* w, int nb, int nbp,
              const double* vg, const double* beta, double dt, int explicit_scheme, float* P, float* Q, float* dirc);

}  // namespace bte

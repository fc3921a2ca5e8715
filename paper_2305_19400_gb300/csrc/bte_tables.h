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

void build_pq(int dim, const double delta[3], int nd, const double* S, const double* w, int nb, int nbp,
              const double* vg, const double* beta, double dt, int explicit_scheme, float* P, float* Q, float* dirc);

}  // namespace bte

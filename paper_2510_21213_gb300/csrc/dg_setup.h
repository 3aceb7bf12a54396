// Host-side setup helpers (FP64): quadrature, Lagrange traces, 1-D SIPDG
// tables, level hierarchy pieces, Chebyshev bounds, dense coarse inverse and
// the Gaussian-sum 1/r table.
#pragma once

#include <vector>

#include "dg_internal.h"

namespace dg {

struct GaussSum {
  std::vector<double> c, a;  // 1/r ~ sum_k c_k exp(-a_k r^2)
  double rmin = 0, rmax = 0, relerr = 0;
};

void gauss_legendre(int n, double* x, double* w);
void lagrange(const double* nodes, int m, double x, double* L, double* dL);
double penalty(int p, double h, int form, double eps);
void build_axis(AxisOp& A, int n, int p, double lo, double hi, double sigma);
// sigma (per axis) overrides the penalty of (p, h) when not null
void build_level(LevelOp& L, const int n[3], int p, const double lo[3], const double hi[3], int pform, double eps,
                 const double* sigma = nullptr);
std::vector<double> axis_matrix(const AxisOp& A, const LevelOp& L);
double sym_max_eig(std::vector<double> S, int n);
double level_lambda_max(const LevelOp& L);
void sym_eig(std::vector<double> S, int n, std::vector<double>& lam, std::vector<double>& V);
std::vector<double> schwarz_tables(const LevelOp& L);
void build_transfer(TransferOp& T, const LevelOp& fine, const LevelOp& coarse);
bool spd_inverse(std::vector<double>& A, int n);
std::vector<double> level_dense(const LevelOp& L);
GaussSum make_gauss_sum(double rmin, double rmax, double tol, bool tabulated = true);

}  // namespace dg

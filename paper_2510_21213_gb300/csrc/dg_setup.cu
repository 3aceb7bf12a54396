// Setup (step S0): Gauss-Legendre rule, Lagrange traces, 1-D SIPDG tables per
// level (Sec. 3.4 eq. sip_bilinear, Sec. 3.5 eq. pen_poly, Nitsche boundary
// faces), the hp level hierarchy and its transfers (Sec. 6.4), Chebyshev
// bounds, the coarsest-level inverse and the Gaussian-sum tables used for the
// Dirichlet data (Sec. 5.2, Sec. 6.3). Host FP64 throughout.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "dg_setup.h"
#include "dg_gauss_tables.h"

namespace dg {

// ---------------------------------------------------------------------------
// 1-D numerics
// ---------------------------------------------------------------------------
// Gauss-Legendre nodes (ascending) and weights on [-1, 1] by Newton's method on
// P_n, evaluated with the three-term recurrence (k+1) P_{k+1} = (2k+1) z P_k - k P_{k-1}.
void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 200; ++it) {
      double pk = 1.0, pkm1 = 0.0;
      for (int k = 0; k < n; ++k) {
        const double pkp1 = ((2.0 * k + 1.0) * z * pk - k * pkm1) / (k + 1.0);
        pkm1 = pk;
        pk = pkp1;
      }
      dp = n * (z * pk - pkm1) / (z * z - 1.0);
      const double dz = pk / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-17) break;
    }
    {
      double pk = 1.0, pkm1 = 0.0;
      for (int k = 0; k < n; ++k) {
        const double pkp1 = ((2.0 * k + 1.0) * z * pk - k * pkm1) / (k + 1.0);
        pkm1 = pk;
        pk = pkp1;
      }
      dp = n * (z * pk - pkm1) / (z * z - 1.0);
    }
    x[n - 1 - i] = z;
    x[i] = -z;
    const double wi = 2.0 / ((1.0 - z * z) * dp * dp);
    w[i] = wi;
    w[n - 1 - i] = wi;
  }
  if (n % 2 == 1) x[n / 2] = 0.0;
}

// Lagrange basis on `nodes` (m points): values L[i] and derivatives dL[i] at x.
void lagrange(const double* nodes, int m, double x, double* L, double* dL) {
  for (int i = 0; i < m; ++i) {
    double v = 1.0;
    for (int j = 0; j < m; ++j)
      if (j != i) v *= (x - nodes[j]) / (nodes[i] - nodes[j]);
    L[i] = v;
    double der = 0.0;
    for (int j = 0; j < m; ++j) {
      if (j == i) continue;
      double t = 1.0 / (nodes[i] - nodes[j]);
      for (int l = 0; l < m; ++l)
        if (l != i && l != j) t *= (x - nodes[l]) / (nodes[i] - nodes[l]);
      der += t;
    }
    dL[i] = der;
  }
}

double penalty(int p, double h, int form, double eps) {
  const double c2 = (double)(p + 1) * (p + 1);
  return form == 1 ? c2 / (eps * h * h) : c2 / (eps * h);
}

// 1-D tables of one axis (see AxisOp). Rows are test functions l_a, columns
// trial functions l_i, both on the element; faces use the jump/average of
// Sec. 3.1 with n^- = +1, n^+ = -1.
void build_axis(AxisOp& A, int n, int p, double lo, double hi, double sigma) {
  const int n1 = p + 1;
  double xi[MAXN1], w[MAXN1];
  gauss_legendre(n1, xi, w);
  std::memset(&A, 0, sizeof(A));
  A.n = n;
  A.lo = lo;
  A.hi = hi;
  A.h = (hi - lo) / n;
  A.sigma = sigma;
  const double h = A.h;
  double D[MAXN1][MAXN1], L[MAXN1], dL[MAXN1];
  for (int q = 0; q < n1; ++q) {
    lagrange(xi, n1, xi[q], L, dL);
    for (int i = 0; i < n1; ++i) D[q][i] = dL[i];
  }
  double lm[MAXN1], dlm[MAXN1], lp[MAXN1], dlp[MAXN1];
  lagrange(xi, n1, -1.0, lm, dlm);
  lagrange(xi, n1, 1.0, lp, dlp);
  for (int ty = 0; ty < 4; ++ty) {
    const bool lb = ty & 1, rb = ty & 2;
    for (int a = 0; a < n1; ++a)
      for (int i = 0; i < n1; ++i) {
        double v = 0.0;
        for (int q = 0; q < n1; ++q) v += w[q] * D[q][a] * D[q][i];
        v *= 2.0 / h;  // int l_a' l_i' dx
        if (lb)  // Nitsche, outward normal -1
          v += (2.0 / h) * lm[i] * dlm[a] + (2.0 / h) * dlm[i] * lm[a] + sigma * lm[i] * lm[a];
        else  // interior face, element on the + side
          v += (1.0 / h) * lm[i] * dlm[a] + (1.0 / h) * dlm[i] * lm[a] + sigma * lm[i] * lm[a];
        if (rb)  // Nitsche, outward normal +1
          v += -(2.0 / h) * lp[i] * dlp[a] - (2.0 / h) * dlp[i] * lp[a] + sigma * lp[i] * lp[a];
        else  // interior face, element on the - side
          v += -(1.0 / h) * lp[i] * dlp[a] - (1.0 / h) * dlp[i] * lp[a] + sigma * lp[i] * lp[a];
        A.Kd[ty][a * n1 + i] = v;
      }
  }
  for (int a = 0; a < n1; ++a) {
    A.cLv[a] = -(1.0 / h) * dlm[a] - sigma * lm[a];
    A.cLd[a] = (1.0 / h) * lm[a];
    A.cRv[a] = (1.0 / h) * dlp[a] - sigma * lp[a];
    A.cRd[a] = -(1.0 / h) * lp[a];
    A.m[a] = w[a] * h / 2.0;
    A.lift[0][a] = sigma * lm[a] + (2.0 / h) * dlm[a];
    A.lift[1][a] = sigma * lp[a] - (2.0 / h) * dlp[a];
  }
}

void build_level(LevelOp& L, const int n[3], int p, const double lo[3], const double hi[3], int pform, double eps,
                 const double* sigma) {
  std::memset(&L, 0, sizeof(L));
  const int n1 = p + 1;
  for (int d = 0; d < 3; ++d) L.n[d] = n[d];
  L.p = p;
  L.n1 = n1;
  L.E = n[0] * n[1] * n[2];
  L.Nq = (long long)L.E * n1 * n1 * n1;
  double xi[MAXN1], w[MAXN1];
  gauss_legendre(n1, xi, w);
  lagrange(xi, n1, -1.0, L.tl, L.dl);
  lagrange(xi, n1, 1.0, L.tr, L.dr);
  for (int d = 0; d < 3; ++d) {
    const double h = (hi[d] - lo[d]) / n[d];
    build_axis(L.ax[d], n[d], p, lo[d], hi[d], sigma ? sigma[d] : penalty(p, h, pform, eps));
  }
}

// Dense global 1-D matrix of one axis from its tables.
std::vector<double> axis_matrix(const AxisOp& A, const LevelOp& L) {
  const int n1 = L.n1, n = A.n, Ld = n * n1;
  std::vector<double> M((size_t)Ld * Ld, 0.0);
  for (int e = 0; e < n; ++e) {
    const int ty = (e == 0 ? 1 : 0) | (e == n - 1 ? 2 : 0);
    for (int a = 0; a < n1; ++a) {
      const int r = e * n1 + a;
      for (int i = 0; i < n1; ++i) {
        M[(size_t)r * Ld + e * n1 + i] = A.Kd[ty][a * n1 + i];
        if (e > 0) M[(size_t)r * Ld + (e - 1) * n1 + i] = A.cLv[a] * L.tr[i] + A.cLd[a] * L.dr[i];
        if (e < n - 1) M[(size_t)r * Ld + (e + 1) * n1 + i] = A.cRv[a] * L.tl[i] + A.cRd[a] * L.dl[i];
      }
    }
  }
  return M;
}

// Largest eigenvalue of a symmetric matrix (cyclic Jacobi rotations).
double sym_max_eig(std::vector<double> S, int n) {
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < n; ++i) {
      diag += S[(size_t)i * n + i] * S[(size_t)i * n + i];
      for (int j = i + 1; j < n; ++j) off += S[(size_t)i * n + j] * S[(size_t)i * n + j];
    }
    if (off <= 1e-30 * diag) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = S[(size_t)p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double app = S[(size_t)p * n + p], aqq = S[(size_t)q * n + q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {
          const double skp = S[(size_t)k * n + p], skq = S[(size_t)k * n + q];
          S[(size_t)k * n + p] = c * skp - s * skq;
          S[(size_t)k * n + q] = s * skp + c * skq;
        }
        for (int k = 0; k < n; ++k) {
          const double spk = S[(size_t)p * n + k], sqk = S[(size_t)q * n + k];
          S[(size_t)p * n + k] = c * spk - s * sqk;
          S[(size_t)q * n + k] = s * spk + c * sqk;
        }
      }
  }
  double mx = -1e300;
  for (int i = 0; i < n; ++i) mx = std::max(mx, S[(size_t)i * n + i]);
  return mx;
}

// Full eigen-decomposition of a symmetric matrix by cyclic Jacobi rotations:
// S = V diag(lam) V^T, V[i*n + k] = component i of eigenvector k.
void sym_eig(std::vector<double> S, int n, std::vector<double>& lam, std::vector<double>& V) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 80; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < n; ++i) {
      diag += S[(size_t)i * n + i] * S[(size_t)i * n + i];
      for (int j = i + 1; j < n; ++j) off += S[(size_t)i * n + j] * S[(size_t)i * n + j];
    }
    if (off <= 1e-32 * diag) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = S[(size_t)p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double app = S[(size_t)p * n + p], aqq = S[(size_t)q * n + q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < n; ++k) {
          const double skp = S[(size_t)k * n + p], skq = S[(size_t)k * n + q];
          S[(size_t)k * n + p] = c * skp - sn * skq;
          S[(size_t)k * n + q] = sn * skp + c * skq;
        }
        for (int k = 0; k < n; ++k) {
          const double spk = S[(size_t)p * n + k], sqk = S[(size_t)q * n + k];
          S[(size_t)p * n + k] = c * spk - sn * sqk;
          S[(size_t)q * n + k] = sn * spk + c * sqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * vkp - sn * vkq;
          V[(size_t)k * n + q] = sn * vkp + c * vkq;
        }
      }
  }
  lam.resize(n);
  for (int i = 0; i < n; ++i) lam[i] = S[(size_t)i * n + i];
}

// Schwarz patch tables of one level (layout in dg_internal.h): for every axis
// and element position, the generalised eigenpairs of the 1-D operator
// restricted to the patch nodes [e n1 - oL, (e+1) n1 - 1 + oR].
std::vector<double> schwarz_tables(const LevelOp& L) {
  const int n1 = L.n1, MP = n1 + 2, STR = schwarz_axis_stride(n1);
  std::vector<double> out((size_t)(L.n[0] + L.n[1] + L.n[2]) * STR, 0.0);
  size_t off = 0;
  for (int d = 0; d < 3; ++d) {
    const int n = L.n[d], Ld = n * n1;
    const std::vector<double> A = axis_matrix(L.ax[d], L);
    for (int e = 0; e < n; ++e, off += STR) {
      const int oL = e > 0 ? 1 : 0, oR = e < n - 1 ? 1 : 0;
      const int lo = e * n1 - oL, m = n1 + oL + oR;
      std::vector<double> Mi(m), S((size_t)m * m);
      for (int i = 0; i < m; ++i) Mi[i] = 1.0 / std::sqrt(L.ax[d].m[(lo + i) % n1]);
      for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) S[(size_t)i * m + j] = A[(size_t)(lo + i) * Ld + (lo + j)] * Mi[i] * Mi[j];
      std::vector<double> lam, V;
      sym_eig(S, m, lam, V);
      double* tb = out.data() + off;
      tb[0] = m;
      tb[1] = oL;
      for (int i = 0; i < m; ++i)
        for (int k = 0; k < m; ++k) tb[2 + i * MP + k] = Mi[i] * V[(size_t)i * m + k];
      for (int k = 0; k < m; ++k) tb[2 + MP * MP + k] = lam[k];
    }
  }
  return out;
}

// lambda_max(D^-1 A) of the 3-D Kronecker-sum operator: A <= mu_d diag(A_d) in
// each direction implies x^T A x <= max_d mu_d x^T D x, with equality for the
// product of the 1-D maximisers, so the bound is exact for isotropic meshes.
double level_lambda_max(const LevelOp& L) {
  double mu = 0.0;
  for (int d = 0; d < 3; ++d) {
    const int Ld = L.ax[d].n * L.n1;
    std::vector<double> M = axis_matrix(L.ax[d], L);
    std::vector<double> s(Ld);
    for (int i = 0; i < Ld; ++i) s[i] = 1.0 / std::sqrt(M[(size_t)i * Ld + i]);
    for (int i = 0; i < Ld; ++i)
      for (int j = 0; j < Ld; ++j) M[(size_t)i * Ld + j] *= s[i] * s[j];
    mu = std::max(mu, sym_max_eig(M, Ld));
  }
  return mu;
}

void build_transfer(TransferOp& T, const LevelOp& fine, const LevelOp& coarse) {
  std::memset(&T, 0, sizeof(T));
  T.n1f = fine.n1;
  T.n1c = coarse.n1;
  double xf[MAXN1], wf[MAXN1], xc[MAXN1], wc[MAXN1], L[MAXN1], dL[MAXN1];
  gauss_legendre(fine.n1, xf, wf);
  gauss_legendre(coarse.n1, xc, wc);
  if (fine.n[0] == coarse.n[0]) {
    T.kind = 0;
    for (int a = 0; a < fine.n1; ++a) {
      lagrange(xc, coarse.n1, xf[a], L, dL);
      for (int i = 0; i < coarse.n1; ++i) T.I[0][a * coarse.n1 + i] = L[i];
    }
  } else {
    T.kind = 1;
    for (int cp = 0; cp < 2; ++cp)
      for (int a = 0; a < fine.n1; ++a) {
        lagrange(xc, coarse.n1, (xf[a] + 2.0 * cp - 1.0) / 2.0, L, dL);
        for (int i = 0; i < coarse.n1; ++i) T.I[cp][a * coarse.n1 + i] = L[i];
      }
  }
}

// Dense SPD inverse via Cholesky (A = L L^T, A^-1 = L^-T L^-1).
bool spd_inverse(std::vector<double>& A, int n) {
  std::vector<double> Lm((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double s = A[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) s -= Lm[(size_t)j * n + k] * Lm[(size_t)j * n + k];
    if (!(s > 0.0)) return false;
    const double ljj = std::sqrt(s);
    Lm[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double t = A[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) t -= Lm[(size_t)i * n + k] * Lm[(size_t)j * n + k];
      Lm[(size_t)i * n + j] = t / ljj;
    }
  }
  // Linv (lower triangular)
  std::vector<double> Li((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    Li[(size_t)j * n + j] = 1.0 / Lm[(size_t)j * n + j];
    for (int i = j + 1; i < n; ++i) {
      double t = 0.0;
      for (int k = j; k < i; ++k) t -= Lm[(size_t)i * n + k] * Li[(size_t)k * n + j];
      Li[(size_t)i * n + j] = t / Lm[(size_t)i * n + i];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j) {
      double t = 0.0;
      for (int k = i; k < n; ++k) t += Li[(size_t)k * n + i] * Li[(size_t)k * n + j];
      A[(size_t)i * n + j] = t;
      A[(size_t)j * n + i] = t;
    }
  return true;
}

// Dense matrix of a (small) level in the element-blocked order.
std::vector<double> level_dense(const LevelOp& L) {
  const int n1 = L.n1, npe = n1 * n1 * n1;
  const long long N = L.Nq;
  std::vector<double> Ax[3];
  for (int d = 0; d < 3; ++d) Ax[d] = axis_matrix(L.ax[d], L);
  const int Lx = L.n[0] * n1, Ly = L.n[1] * n1;
  std::vector<int> X(N), Y(N), Z(N);
  for (long long q = 0; q < N; ++q) {
    const int e = (int)(q / npe), loc = (int)(q % npe);
    X[q] = (e % L.n[0]) * n1 + loc % n1;
    Y[q] = ((e / L.n[0]) % L.n[1]) * n1 + (loc / n1) % n1;
    Z[q] = (e / (L.n[0] * L.n[1])) * n1 + loc / (n1 * n1);
  }
  auto mass = [&](int d, int g) { return L.ax[d].m[g % n1]; };
  const int Lz = L.n[2] * n1;
  std::vector<double> M((size_t)N * N, 0.0);
  for (long long r = 0; r < N; ++r)
    for (long long c = 0; c < N; ++c) {
      double v = 0.0;
      if (Y[r] == Y[c] && Z[r] == Z[c]) v += Ax[0][(size_t)X[r] * Lx + X[c]] * mass(1, Y[r]) * mass(2, Z[r]);
      if (X[r] == X[c] && Z[r] == Z[c]) v += mass(0, X[r]) * Ax[1][(size_t)Y[r] * Ly + Y[c]] * mass(2, Z[r]);
      if (X[r] == X[c] && Y[r] == Y[c]) v += mass(0, X[r]) * mass(1, Y[r]) * Ax[2][(size_t)Z[r] * Lz + Z[c]];
      M[(size_t)r * N + c] = v;
    }
  return M;
}

// ---------------------------------------------------------------------------
// Gaussian-sum 1/r (Sec. 5.2): trapezoidal rule in t for
//   1/r = (2/sqrt(pi)) int_R exp(-r^2 e^{2t} + t) dt,
// giving c_k = (2/sqrt(pi)) dt e^{t_k}, alpha_k = e^{2 t_k}. The range of t is
// cut where the neglected tails are below tol (e^{t_lo} <= tol sqrt(pi)/(2 rmax)
// at the far end, erfc(rmin e^{t_hi}) <= tol/2 at the near end); the step is the
// largest of a decreasing sequence whose measured max relative error on
// [rmin, rmax] is below tol.
// ---------------------------------------------------------------------------
// max over log-spaced r in [rmin, rmax] of |r sum_k c_k exp(-a_k r^2) - 1|
static double gauss_sum_error(const std::vector<double>& c, const std::vector<double>& a, double rmin, double rmax) {
  const int nsamp = 3000;
  double err = 0.0;
  for (int i = 0; i < nsamp; ++i) {
    const double r = std::exp(std::log(rmin) + (std::log(rmax) - std::log(rmin)) * i / (nsamp - 1));
    double s = 0.0;
    for (size_t k = 0; k < c.size(); ++k) s += c[k] * std::exp(-a[k] * r * r);
    err = std::max(err, std::fabs(s * r - 1.0));
  }
  return err;
}

// Tabulated short sums (gen_gauss_tables.py): an entry fitted on [1, R] with
// R >= rmax / rmin and tolerance <= tol, rescaled to [rmin, rmax]
// (alpha / rmin^2, c / rmin) and accepted after the same sampled check; the
// fewest-term entry that passes is taken.
static bool tabulated_gauss_sum(double rmin, double rmax, double tol, GaussSum& G) {
  const double R = rmax / rmin;
  int best = -1;
  for (int e = 0; e < gtab::kEntries; ++e) {
    const gtab::Entry& T = gtab::kEntry[e];
    if (T.tol > tol || T.R < R) continue;
    if (best >= 0 && gtab::kEntry[best].n <= T.n) continue;
    best = e;
  }
  if (best < 0) return false;
  const gtab::Entry& T = gtab::kEntry[best];
  std::vector<double> c(T.n), a(T.n);
  for (int k = 0; k < T.n; ++k) {
    c[k] = gtab::kCoef[T.off + k] / rmin;
    a[k] = gtab::kAlpha[T.off + k] / (rmin * rmin);
  }
  const double err = gauss_sum_error(c, a, rmin, rmax);
  if (!(err <= tol)) return false;
  G.c = c;
  G.a = a;
  G.relerr = err;
  return true;
}

GaussSum make_gauss_sum(double rmin, double rmax, double tol, bool tabulated) {
  GaussSum G;
  G.rmin = rmin;
  G.rmax = rmax;
  if (tabulated && tabulated_gauss_sum(rmin, rmax, tol, G)) return G;
  const double t_lo = std::log(tol * std::sqrt(M_PI) / (2.0 * rmax));
  double xs = 0.5;
  while (std::erfc(xs) > 0.5 * tol) xs += 0.01;
  const double t_hi = std::log(xs / rmin);
  const int nsamp = 3000;
  std::vector<double> rs(nsamp);
  for (int i = 0; i < nsamp; ++i) rs[i] = std::exp(std::log(rmin) + (std::log(rmax) - std::log(rmin)) * i / (nsamp - 1));
  const double dt0 = std::min(0.6, 1.5 * M_PI * M_PI / (2.0 * std::log(1.0 / tol)));
  for (double dt = dt0; dt > 0.05; dt -= 0.005) {
    const int nt = (int)std::ceil((t_hi - t_lo) / dt) + 1;
    std::vector<double> c(nt), a(nt);
    for (int k = 0; k < nt; ++k) {
      const double t = t_lo + k * dt;
      c[k] = 2.0 / std::sqrt(M_PI) * dt * std::exp(t);
      a[k] = std::exp(2.0 * t);
    }
    double err = 0.0;
    for (int i = 0; i < nsamp; ++i) {
      double s = 0.0;
      for (int k = 0; k < nt; ++k) s += c[k] * std::exp(-a[k] * rs[i] * rs[i]);
      err = std::max(err, std::fabs(s * rs[i] - 1.0));
    }
    if (err <= tol) {
      G.c = c;
      G.a = a;
      G.relerr = err;
      return G;
    }
  }
  return G;  // empty: failure
}

}  // namespace dg

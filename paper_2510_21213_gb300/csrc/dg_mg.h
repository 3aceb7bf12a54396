// Multigrid V-cycle of the preconditioner (Sec. 6.4: degree coarsening to 1,
// then geometric), shared by the solver and the learned initial guess.
#pragma once

#include <algorithm>

#include "dg_ctx.h"

namespace dg {

template <typename T>
struct MG {
  dg_ctx* h;
  PrecWork<T>* w;
  const int* act;
  int nact;
  cudaStream_t s;

  // Chebyshev-Jacobi smoothing of A x = b on level l (degree k), Chebyshev
  // semi-iteration on D^-1 A over [lam/range, lam]. On exit, if want_res,
  // lev[l].res holds b - A x.
  int cheb(int l, const T* b, T* x, bool zero_init, bool want_res) {
    Level& L = h->levels[l];
    LevelWork& W = w->lev[l];
    T* res = W.res.as<T>();
    T* d = W.d.as<T>();
    const bool sw = (l > 0 && L.op.p == 1 && h->opts.p1_smoother >= 0 ? h->opts.p1_smoother : h->opts.smoother) ==
                    DG_SMOOTH_SCHWARZ;
    // sw: the smoother preconditioner is M_S (z = M_S res), else D^-1 (fused)
    const T* invD = sw ? nullptr : W.invD.as<T>();
    const long long Nq = L.op.Nq;
    const int deg = (l > 0 && h->opts.coarse_smoother_degree > 0) ? h->opts.coarse_smoother_degree
                                                                  : h->opts.smoother_degree;
    const int k = std::max(1, deg);
    const double bmax = sw ? L.lam_sw : L.lam_max * (1.0 + 1e-6);
    const double amin = bmax / std::max(1.5, h->opts.cheb_range);
    const double theta = 0.5 * (bmax + amin), delta = 0.5 * (bmax - amin);
    const double sig1 = theta / delta;
    const T* r0 = b;
    if (!zero_init) {
      DG_CK(launch_apply<T>(L.op, L.dop, 1, x, res, b, act, nact, s));
      r0 = res;
    }
    if (sw)
      DG_CK(launch_schwarz<T>(L.op, L.dop, L.sw_tabs.as<double>(), r0, W.zp.as<T>(), d, x, zero_init ? 1 : 2,
                              1.0 / theta, 0.0, act, nact, s, L.tc()));
    else
      DG_CK(launch_cheb_first<T>(x, d, r0, invD, 1.0 / theta, zero_init ? 1 : 0, Nq, act, nact, s));
    double rho_prev = 1.0 / sig1;
    bool res_is_b = zero_init;  // the residual of the current x is b - A d when res_is_b
    for (int j = 2; j <= k; ++j) {
      if (res_is_b)
        DG_CK(launch_apply<T>(L.op, L.dop, 1, d, res, b, act, nact, s));
      else
        DG_CK(launch_apply<T>(L.op, L.dop, 2, d, res, nullptr, act, nact, s));
      res_is_b = false;
      const double rho = 1.0 / (2.0 * sig1 - rho_prev);
      if (sw)
        DG_CK(launch_schwarz<T>(L.op, L.dop, L.sw_tabs.as<double>(), res, W.zp.as<T>(), d, x, 3, rho * rho_prev,
                                2.0 * rho / delta, act, nact, s, L.tc()));
      else
        DG_CK(launch_cheb_step<T>(x, d, res, invD, rho * rho_prev, 2.0 * rho / delta, Nq, act, nact, s));
      rho_prev = rho;
    }
    if (want_res) {
      if (res_is_b)
        DG_CK(launch_apply<T>(L.op, L.dop, 1, d, res, b, act, nact, s));
      else
        DG_CK(launch_apply<T>(L.op, L.dop, 2, d, res, nullptr, act, nact, s));
    }
    return DG_OK;
  }

  // x = V(b) on level l (x overwritten)
  int vcycle(int l, const T* b, T* x) {
    if (l == h->nlev - 1) {
      DG_CK(launch_coarse_solve<T>(h->coarse_inv.as<double>(), h->Nc, b, x, act, nact, s));
      return DG_OK;
    }
    Level& L = h->levels[l];
    Level& C = h->levels[l + 1];
    LevelWork& Wc = w->lev[l + 1];
    DG_RET(cheb(l, b, x, true, true));
    DG_CK(launch_restrict<T>(L.tr, L.dtr, L.op, C.op, w->lev[l].res.template as<T>(), Wc.b.as<T>(), act, nact, s));
    DG_RET(vcycle(l + 1, Wc.b.as<T>(), Wc.x.as<T>()));
    DG_CK(launch_prolong_add<T>(L.tr, L.dtr, L.op, C.op, Wc.x.as<T>(), x, act, nact, s));
    DG_RET(cheb(l, b, x, false, false));
    return DG_OK;
  }
};

}  // namespace dg

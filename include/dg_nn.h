/*
 * dg_nn.h -- learned initial guess of the pair solves (precision
 * DG_PREC_MIXED_LEARNED). Not part of the paper's method: a per-element
 * network that only changes where conjugate gradients start. The solver still
 * iterates to the same FP64 true residual, so the converged potentials, K and
 * the energies are those of the plain solver within its tolerance.
 *
 * Network (per element, on the (p+1)^3 Gauss-Legendre nodes, x fastest):
 *   in  [2]  : c0 = s * hbar^2 * b / m    (right-hand side over the nodal
 *                                          mass: 4 pi f in the interior)
 *              c1 = s * x_c               (coarse guess, below)
 *   conv 3x3x3 (2 -> 32) + ReLU, conv 3x3x3 (32 -> 32) + ReLU, conv 3x3x3
 *   (32 -> 2), zero padding at the element border; hbar^3 = hx hy hz.
 *   out [2]  : o0 (fine correction), o1 (correction of the coarse guess)
 *   guess    : y = x_c (1 + o1) + o0 / s; x0 = the fine level's Chebyshev
 *              smoother (the V-cycle's pre-smoothing, Sec. 6.4) applied to
 *              A x = b starting from y, which removes the high-frequency
 *              error that BF16 leaves in y; then x0 is scaled by the
 *              energy-optimal alpha = b^T x0 / x0^T A x0 (never worse than
 *              x = 0 in the A-norm).
 * x_c is the prolongation to the fine level of two multigrid V-cycles on the
 * first degree-1 level of the hierarchy (Sec. 6.4), applied to the restricted
 * right-hand side, times its energy-optimal factor b^T x_c / x_c^T A x_c;
 * s = 1 / rms(x_c) per source. Without the network (dg_nn_guess use_net = 0)
 * y = x_c.
 * The guess is kept only if its FP64 true residual is below ||b||; otherwise
 * the source starts from zero and dg_solve_stats.used_fallback = 1.
 *
 * Parameters: DG_NN_NPARAM floats, in this order (t = 9 (dz+1) + 3 (dy+1) +
 * (dx+1) is the tap reading the input at node offset (dx, dy, dz)):
 *   W1 [27][2][32], b1 [32], W2 [27][32][32], b2 [32], W3 [27][32][2], b3 [2]
 * with W[t][ci][co]. Kept in FP32 (master copy, Adam); the 32 -> 32 layer runs
 * in BF16 on the tensor cores, activations are stored in BF16, every sum
 * accumulates in FP32.
 *
 * Weights file (dg_solver_opts.nn_weights_path): 16-byte header "DGNN",
 * int32 version = 1, int32 DG_NN_NPARAM, int32 p the weights were trained for,
 * then DG_NN_NPARAM little-endian float32.
 *
 * All entry points need a handle of a mesh with p <= 7 and synchronise the
 * stream before returning. "dev" pointers are device memory, "host" pointers
 * host memory; the caller owns both.
 */
#ifndef DG_NN_H
#define DG_NN_H

#include <stdint.h>

#include "dg_poisson.h"

#ifdef __cplusplus
extern "C" {
#endif

#define DG_NN_NPARAM 31170
#define DG_NN_HIDDEN 32

/* Sets the network parameters (host, DG_NN_NPARAM floats) and resets the Adam
 * state. DG_ERR_INVALID_ARG on a null pointer or non-finite value. */
int dg_nn_set_params(dg_handle h, const float* params_host);

/* Copies the current parameters to params_host (DG_NN_NPARAM floats).
 * DG_ERR_INVALID_ARG if none are set. */
int dg_nn_get_params(dg_handle h, float* params_host);

/* out_dev = net(in_dev) for n_elem elements of the handle's degree:
 * in_dev [n_elem][(p+1)^3][2], out_dev [n_elem][(p+1)^3][2] (FP32, device).
 * save_act = 1 keeps the activations for a following dg_nn_backward on the
 * same input. DG_ERR_INVALID_ARG without parameters or for p > 7. */
int dg_nn_forward(dg_handle h, const float* in_dev, float* out_dev, int64_t n_elem, int32_t save_act, void* stream);

/* grad_dev [DG_NN_NPARAM] = gradient of sum(gout_dev * out) over all elements,
 * out = net(in_dev); needs the activations of dg_nn_forward(in_dev, n_elem,
 * save_act = 1) (DG_ERR_INVALID_ARG otherwise). Summation order is fixed:
 * repeated calls give identical results. */
int dg_nn_backward(dg_handle h, const float* in_dev, const float* gout_dev, float* grad_dev, int64_t n_elem,
                   void* stream);

/* One Adam step on the handle's parameters with gradient grad_dev (device,
 * DG_NN_NPARAM floats), bias-corrected, step count kept by the handle. */
int dg_nn_adam(dg_handle h, const float* grad_dev, float lr, float beta1, float beta2, float eps, void* stream);

/* One training step on B sources f_dev [B][Nq] with target potentials v_dev
 * [B][Nq] (FP64, device; e.g. dg_pair_solve_batch's solutions): right-hand
 * sides as in dg_pair_solve_batch, the network's guess y above (FP32, before
 * smoothing), the loss
 *   L = (1/B) sum_k sum_q m_q (y_kq - v_kq)^2 / sum_q m_q v_kq^2
 * (relative squared L2 error in the discrete mass norm), its gradient through
 * the network (backward kernels) and an Adam step (beta1 0.9, beta2 0.999,
 * eps 1e-8) with learning rate lr. loss_host [B + 1]: [0] = L, [1 + k] the
 * term of source k. */
int dg_nn_train_step(dg_handle h, const double* f_dev, const double* v_dev, int64_t B, float lr, double* loss_host,
                     void* stream);

/* The initial guess the solver starts from, for B sources f_dev [B][Nq]:
 * use_net = 0 gives the coarse guess x_c alone, use_net = 1 the network's guess,
 * each after the alpha scaling and the fallback test. x0_dev [B][Nq] (FP64,
 * device) receives it, rel_host [B] its FP64 relative residual
 * ||b - A x0|| / ||b|| (1 where the zero guess is kept). */
int dg_nn_guess(dg_handle h, const double* f_dev, int64_t B, int32_t use_net, double* x0_dev, double* rel_host,
                void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DG_NN_H */

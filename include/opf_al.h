/*
 * opf_al.h — C ABI of a first-order augmented-Lagrangian loop on the GPU
 * that consumes the callbacks of include/opf.h: a solver-side user of the
 * objective, gradient, constraint and J^T v kernels, with every step of the
 * iteration in the library's kernels (no host round trip per iteration).
 *
 * The paper's solvers (Sec. IV) are second-order interior-point methods
 * whose KKT solves are out of scope here; this loop shows the callbacks in a
 * solver iteration and serves as the consumer of the learned warm start.
 *
 * Problem: min f(x) s.t. gl <= g(x) <= gu, xl <= x <= xu (the NLP of
 * include/opf.h). With multipliers lambda (one per row) and penalty rho > 0,
 * the augmented Lagrangian is
 *   L(x; lambda) = f(x) + sum_i [ rho/2 d_i(x)^2 - lambda_i^2 / (2 rho) ],
 *   d_i(x) = s_i - clip(s_i, gl_i, gu_i),  s_i = g_i(x) + lambda_i / rho,
 * and its gradient is grad f(x) + J(x)^T mu, mu_i = rho d_i(x).
 * Inner iteration (Adam, Kingma and Ba; beta1 0.9, beta2 0.999, eps 1e-8,
 * step count kept across calls until opf_al_reset):
 *   G = grad f(x) + J(x)^T mu(x);  m = b1 m + (1 - b1) G;
 *   v = b2 v + (1 - b2) G^2;  x = clip(x - lr (m / (1 - b1^k)) r, xl, xu),
 *   r = 1 / (sqrt(v / (1 - b2^k)) + eps), where r, a step-size scale, is
 *   formed in FP32 with correctly rounded operations (v / (1 - b2^k)
 *   rounded to FP32, square root, + eps, reciprocal) and the rest in FP64.
 * Outer update: lambda = mu(x).
 *
 * Ownership and errors as in include/opf.h: device buffers are caller-owned,
 * calls are asynchronous on the given stream, codes OPF_*.
 */
#ifndef OPF_AL_H
#define OPF_AL_H

#include <stdint.h>

#include "opf.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct opf_al opf_al;

typedef struct {
    double rho; /* penalty, > 0 */
    double lr;  /* Adam step size, > 0 */
} opf_al_opts;

/* Loop state for one model (the model must outlive it): work vectors, Adam
 * moments and device copies of the bounds. */
int opf_al_create(opf_model *model, const opf_al_opts *opts, opf_al **out);
int opf_al_destroy(opf_al *al);

/* `iters` inner iterations on d_x (n, device, updated in place, projected
 * onto [xl, xu] after every step) at fixed d_lambda (m, device). d_stats
 * (device, 3 doubles, may be NULL) receives, at the final point: f(x), the
 * largest row violation max_i max(gl_i - g_i, g_i - gu_i, 0), and
 * L(x; lambda). One iteration is captured once per (d_x, d_lambda) pair as
 * a CUDA graph and replayed (the step count's bias corrections live on the
 * device); opf_al_reset drops the captured graphs. */
int opf_al_iterate(opf_al *al, double *d_x, const double *d_lambda, int32_t iters, double *d_stats,
                   void *stream);

/* Multiplier update at d_x: d_lambda = mu(x). d_stats as above, at d_x. */
int opf_al_update(opf_al *al, const double *d_x, double *d_lambda, double *d_stats, void *stream);

/* One projected Newton-CG step of L(.; lambda) on d_x (a second-order inner
 * step that uses the Jacobian and Lagrangian-Hessian values of
 * include/opf.h): x is first projected onto [xl, xu] (in place); at x, with c = g(x), s = c + lambda / rho, mu = rho (s -
 * clip(s, gl, gu)) and D_i = 1 where s_i lies outside [gl_i, gu_i] (else 0),
 *   G = grad f(x) + J^T mu,  K = H(x; mu, sigma = 1) + rho J^T diag(D) J
 * (H from opf_eval_hess with the multipliers mu, J from opf_eval_jac; K is
 * L's generalised Hessian). Free entries: all but x_j at xl_j with G_j > 0
 * and x_j at xu_j with G_j < 0. With the Jacobi diagonal M_j = K_jj (1
 * where K_jj <= 1e-12) and a Levenberg-Marquardt weight delta: conjugate
 * gradients with the preconditioner M (1 + delta) on (K + delta diag(M)) p =
 * -G over the free entries, from p = 0, at most cg_iters iterations,
 * stopping at non-positive curvature (taking the first direction itself if
 * that happens at once) or when r^T z falls below 1e-24 of its first value.
 * p is scaled by 1 / max_j |p_j| where that is above 1 (no entry moves by
 * more than 1 in one step). Then x_t = clip(x + 2^-t p, xl, xu), t = 0..7,
 * and x becomes the x_t of
 * the smallest t with L(x_t) <= L(x) + 1e-4 2^-t G^T p; else the x_t of
 * least L if below L(x); else x is left unchanged. delta starts at 1e-2
 * (again after opf_al_reset) and is kept on the device between steps:
 * divided by 4 after a full step, multiplied by 10 after a step of 1/8 or
 * less (or none), within [1e-8, 1e4]. Every sum is a fixed-
 * order reduction and every scalar stays on the device (no host round
 * trip). d_stats (3 doubles, may be NULL) as in opf_al_iterate, at the new
 * x; d_step (n, may be NULL) receives p. cg_iters >= 1. The Adam state is
 * not touched. The first call builds the sparse structures; the CG
 * iterations are captured once per cg_iters as a CUDA graph and replayed
 * (opf_al_reset drops it, since it holds rho). The paper's interior-point solvers (Sec. IV-A) take Newton
 * steps on the KKT system with a sparse direct solver; this is the matrix-
 * free counterpart on the augmented Lagrangian. */
int opf_al_newton(opf_al *al, double *d_x, const double *d_lambda, int32_t cg_iters, double *d_stats,
                  double *d_step, void *stream);

/* Clear the Adam moments and step count; set the penalty and step size. */
int opf_al_reset(opf_al *al, double rho, double lr);

#ifdef __cplusplus
}
#endif
#endif

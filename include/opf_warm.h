/*
 * opf_warm.h — C ABI of the learned warm start: a three-layer BF16 MLP that
 * maps a grid's load profile to a starting point (voltage angles and
 * magnitudes, generator active and reactive outputs) for the AC-OPF NLP of
 * include/opf.h, trained on the GPU with the library's own kernels.
 *
 * The paper points to learned proxies of OPF solutions as a way to move work
 * offline (Sec. I, machine-learning proxies) and warm-starts its largest
 * model from an existing solution (Sec. IV-C); this component learns such a
 * starting point. Network: u -> GELU(W1 u + b1) -> GELU(W2 h1 + b2) ->
 * W3 h2 + b3 = y, GELU the tanh form 0.5 z (1 + tanh(sqrt(2/pi)(z + 0.044715
 * z^3))) (Hendrycks and Gimpel, 2016). Weights and activations in BF16,
 * products accumulated in FP32 in tensor memory (tcgen05.mma fed by TMA),
 * master weights, biases and optimiser state in FP32.
 *
 * Input u (2 nload, zero-padded to a multiple of 128): for every load l,
 * (Pd_l / Pd0_l - 1) / 0.2 then (Qd_l / Qd0_l - 1) / 0.2, Pd0/Qd0 the
 * network's base loads (0 where the base load is 0).
 * Output y: four blocks [ya | yv | yp | yq] of widths nbp, nbp, ngp, ngp
 * (nbus and ngen rounded up to multiples of 128; padding unused). The point
 * is va = va_scale ya (va_ref = 0, its output unused), vm = (vmin + vmax)/2
 * + yv, pg = (pmin + pmax)/2 + (pmax - pmin)/2 yp, qg likewise; p and q are
 * the branch flows at (va, vm), so every flow row is zero. y = 0 is the flat
 * start (every angle 0, magnitudes and generator outputs at mid-range).
 * Training loss of a batch of B load profiles (the mean over profiles of)
 *   f(x) + penalty * (sum_i rho_i^2 + sum_j r_j^2),
 *   rho = g(x) - clip(g(x), gl, gu),  r = x - clip(x, xl, xu),
 * f the generation cost, g the constraints and xl, xu the variable bounds of
 * include/opf.h, evaluated by its kernels; the gradient is (grad f + 2
 * penalty (J^T rho + r)) / B, chained through p, q = flows(va, vm) with a
 * second J^T product, then through the output map and the network.
 * Optimiser: Adam; the output layer's bias has its own learning rate
 * (lr_out), so that the mean point moves at the speed of a per-coordinate
 * method while the weights learn the load-dependent part slowly.
 *
 * Ownership and errors as in include/opf.h: device buffers are caller-owned,
 * calls are asynchronous on the given stream, codes OPF_*.
 */
#ifndef OPF_WARM_H
#define OPF_WARM_H

#include <stdint.h>

#include "opf.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct opf_warm opf_warm;

typedef struct {
    int32_t batch;     /* profiles per training step and per prediction call;
                          a multiple of 128 */
    int32_t hidden;    /* width of both hidden layers; a multiple of 128 */
    double penalty;    /* weight of the squared constraint residuals */
    double lr;         /* Adam learning rate of the weights and hidden biases
                          (beta1 0.9, beta2 0.999, eps 1e-8) */
    double lr_out;     /* Adam learning rate of the output bias */
    double va_scale;   /* radians per unit of the angle outputs */
    uint64_t seed;     /* initial W1, W2: N(0, 1/fan_in); W3 and every bias start at 0,
                          so the untrained network proposes the flat start */
} opf_warm_opts;

/* A warm-start model for one single-period network (net->nperiod == 1).
 * Allocates the weights, the optimiser state, activation buffers for
 * opts->batch profiles and an internal callback model of batch periods. */
int opf_warm_create(const opf_network *net, const opf_warm_opts *opts, opf_warm **out);
int opf_warm_destroy(opf_warm *w);

/* Network input and output widths (padded), and n of one profile's x. */
int opf_warm_dims(const opf_warm *w, int32_t *n_in, int32_t *n_out, int32_t *n_x,
                  int64_t *n_params);

/* One Adam step on a batch of load profiles d_load_pd, d_load_qd
 * ([batch][nload] device doubles). d_stats (device, 3 doubles) receives
 * the batch means of the loss, of the cost and of sum(rho^2) + sum(r^2). */
int opf_warm_train_step(opf_warm *w, const double *d_load_pd, const double *d_load_qd,
                        double *d_stats, void *stream);

/* Starting points for a batch of profiles: d_x receives the x of a
 * `batch`-period model of the network (include/opf.h layout, period t =
 * profile t), every flow row zero and va_ref zero. */
int opf_warm_predict(opf_warm *w, const double *d_load_pd, const double *d_load_qd, double *d_x,
                     void *stream);

/* The network alone, for checking: forward pass of a batch into the
 * outputs d_y ([batch][n_out] floats); backward pass of a given output
 * gradient d_dy ([batch][n_out] floats, padding entries zero) into d_grad
 * (n_params floats, layout W1, b1, W2, b2, W3, b3, row-major [out][in]). */
int opf_warm_forward(opf_warm *w, const double *d_load_pd, const double *d_load_qd, float *d_y,
                     void *stream);
int opf_warm_backward(opf_warm *w, const float *d_dy, float *d_grad, void *stream);

/* The network's intermediate tensors after the last forward (and backward)
 * pass, for checking each layer against the oracle on its own inputs: into
 * HOST buffers (any may be NULL) the BF16 input u ([batch][n_in], raw 16-bit
 * words), the FP32 pre-activations z1, z2 ([batch][hidden]), their BF16
 * GELU outputs h1, h2 (raw 16-bit), and the FP32 pre-activation gradients
 * dz2, dz1 of the last backward pass ([batch][hidden]; the next GEMM takes
 * them rounded to BF16). Synchronises the device. */
int opf_warm_get_activations(const opf_warm *w, uint16_t *h_u, float *h_z1, uint16_t *h_h1, float *h_z2,
                             uint16_t *h_h2, float *h_dz2, float *h_dz1);

/* The physics half of a training step, for checking: from given network
 * outputs d_y ([batch][n_out] floats), the batch loss statistics (as in
 * opf_warm_train_step) and its gradient with respect to y into d_dy. */
int opf_warm_loss_grad(opf_warm *w, const double *d_load_pd, const double *d_load_qd,
                       const float *d_y, float *d_dy, double *d_stats, void *stream);

/* Learning rates of the following training steps (a schedule is the caller's). */
int opf_warm_set_lr(opf_warm *w, double lr, double lr_out);

/* FP32 master parameters to / from HOST memory (n_params floats, layout as
 * above); setting also refreshes the BF16 copies and clears Adam's state.
 * Getting synchronises the device and also returns OPF_ECUDA if a
 * tensor-core GEMM gave up waiting on one of its barriers since the last
 * check (the results of that GEMM are then invalid). */
int opf_warm_get_params(const opf_warm *w, float *h_params);
int opf_warm_set_params(opf_warm *w, const float *h_params);

#ifdef __cplusplus
}
#endif
#endif

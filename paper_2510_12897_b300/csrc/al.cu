// Augmented-Lagrangian loop (include/opf_al.h): Adam inner iterations on
// L(x; lambda) with the library's callback kernels, multiplier updates, and
// the statistics of a point, all on the device.
#include <cmath>
#include <vector>

#include "../../include/opf_al.h"
#include "model.h"

namespace opf {
void bounds(const Model &M, double *xl, double *xu, double *gl, double *gu);
}  // namespace opf

using namespace opf;

struct opf_al {
    Model *M = nullptr;  // not owned
    int64_t n = 0, m = 0;
    double rho = 1.0, lr = 1e-3;
    int64_t step = 0;
    int nparts = 0;
    std::vector<void *> allocs;
    double *xl = nullptr, *xu = nullptr, *gl = nullptr, *gu = nullptr;
    double *grad = nullptr, *c = nullptr, *mu = nullptr, *u = nullptr, *m1 = nullptr, *m2 = nullptr;
    double *obj = nullptr, *part = nullptr;  // part: [3][nparts] block partials
    double *bpow = nullptr;  // device: beta1^k, beta2^k, 1 - beta1^k, 1 - beta2^k and their reciprocals
    // one inner iteration captured as a CUDA graph per (x, lambda) pair: the
    // loop replays it instead of launching its five kernels one by one
    cudaStream_t cap = nullptr;
    struct Graph {
        const double *x, *lam;
        cudaGraphExec_t exec;
    };
    std::vector<Graph> graphs;
};

namespace {

int al_check(cudaError_t e, const char *what)
{
    if (e != cudaSuccess) {
        set_error("opf_al: %s: %s", what, cudaGetErrorString(e));
        return OPF_ECUDA;
    }
    return OPF_OK;
}

template <class T>
int al_alloc(opf_al *a, T **p, size_t count)
{
    void *q = nullptr;
    if (cudaMalloc(&q, sizeof(T) * (count ? count : 1)) != cudaSuccess) {
        cudaGetLastError();
        set_error("opf_al: cudaMalloc of %zu bytes failed", sizeof(T) * count);
        return OPF_ENOMEM;
    }
    a->allocs.push_back(q);
    *p = static_cast<T *>(q);
    return OPF_OK;
}

void al_drop_graphs(opf_al *a)
{
    for (auto &g : a->graphs)
        cudaGraphExecDestroy(g.exec);
    a->graphs.clear();
}

void al_free(opf_al *a)
{
    if (!a)
        return;
    al_drop_graphs(a);
    if (a->cap) {
        cudaStreamSynchronize(a->cap);
        cudaStreamDestroy(a->cap);
    }
    for (void *p : a->allocs)
        cudaFree(p);
    delete a;
}

__device__ __forceinline__ double block_sum(double v, double *red)
{
    for (int off = 16; off; off >>= 1)
        v += __shfl_down_sync(0xffffffffu, v, off);
    __syncthreads();
    if ((threadIdx.x & 31) == 0)
        red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < (int)(blockDim.x >> 5); q++)
            s += red[q];
    return s;
}

__device__ __forceinline__ double block_max(double v, double *red)
{
    for (int off = 16; off; off >>= 1)
        v = fmax(v, __shfl_down_sync(0xffffffffu, v, off));
    __syncthreads();
    if ((threadIdx.x & 31) == 0)
        red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < (int)(blockDim.x >> 5); q++)
            s = fmax(s, red[q]);
    return s;
}

// mu = rho (s - clip(s, gl, gu)), s = c + lambda / rho (lambda times the
// host's 1 / rho, as the J^T mu kernels form it); per-block partials of the
// row violation (max), sum mu^2 and sum lambda^2
__global__ void al_mu_kernel(const double *c, const double *lam, const double *gl, const double *gu, int64_t m,
                             double rho, double inv_rho, double *mu, double *part, int nparts)
{
    __shared__ double red[32];
    double viol = 0.0, smu = 0.0, slam = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double ci = c[i], li = lam ? lam[i] : 0.0;
        const double s = fma(li, inv_rho, ci);
        const double d = s - fmin(fmax(s, gl[i]), gu[i]);
        const double mi = rho * d;
        mu[i] = mi;
        viol = fmax(viol, fmax(fmax(gl[i] - ci, ci - gu[i]), 0.0));
        smu = fma(mi, mi, smu);
        slam = fma(li, li, slam);
    }
    const double a = block_max(viol, red);
    const double b = block_sum(smu, red);
    const double e = block_sum(slam, red);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = a;
        part[nparts + blockIdx.x] = b;
        part[2 * nparts + blockIdx.x] = e;
    }
}

// stats = (f, max violation, L) from the partials, in a fixed order
__global__ void al_stats_kernel(const double *obj, const double *part, int nparts, double rho, double *stats)
{
    double viol = 0.0, smu = 0.0, slam = 0.0;
    for (int q = threadIdx.x; q < nparts; q += 32) {
        viol = fmax(viol, part[q]);
        smu += part[nparts + q];
        slam += part[2 * nparts + q];
    }
    for (int off = 16; off; off >>= 1) {
        viol = fmax(viol, __shfl_down_sync(0xffffffffu, viol, off));
        smu += __shfl_down_sync(0xffffffffu, smu, off);
        slam += __shfl_down_sync(0xffffffffu, slam, off);
    }
    if (threadIdx.x == 0) {
        stats[0] = obj[0];
        stats[1] = viol;
        stats[2] = obj[0] + (smu - slam) / (2.0 * rho);
    }
}

// Adam step on G = grad + u, then projection onto [xl, xu]; the bias
// corrections enter as two per-thread scalars, lr / (1 - b1^k) and
// 1 / (1 - b2^k), leaving one square root and one division per entry
__global__ void al_adam_kernel(double *x, const double *grad, const double *u, const double *xl, const double *xu,
                               double *m1, double *m2, int64_t n, double lr, const double *bp)
{
    const double b1 = 0.9, b2 = 0.999;
    const double k1 = lr * bp[4], k2 = bp[5];  // the reciprocals of 1 - b1^k, 1 - b2^k, formed once per step
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const double G = grad ? grad[j] + u[j] : u[j];  // u alone: the whole gradient
        const double a = fma(b1, m1[j], (1.0 - b1) * G);
        const double b = fma(b2, m2[j], (1.0 - b2) * G * G);
        m1[j] = a;
        m2[j] = b;
        // the scale 1 / (sqrt(v_hat) + eps) in FP32, correctly rounded at
        // every operation: FP64 square roots and divisions would cost about
        // 30 FP64 pipe operations per entry
        const float den = __fadd_rn(__fsqrt_rn(__double2float_rn(b * k2)), 1e-8f);
        const double xn = x[j] - k1 * a * (double)__frcp_rn(den);
        x[j] = fmin(fmax(xn, xl[j]), xu[j]);
    }
}

int grid_of(int64_t n)
{
    int64_t g = (n + 255) / 256;
    if (g > 148 * 8)
        g = 148 * 8;
    return (int)(g < 1 ? 1 : g);
}

// f, grad f, g at x; mu; optional statistics
int al_point(opf_al *a, const double *x, const double *lam, bool want_grad, double *d_stats, cudaStream_t s)
{
    EvalArgs e{x, nullptr, 1.0, a->obj, want_grad ? a->grad : nullptr, a->c, nullptr, nullptr};
    int rc = launch_eval(*a->M, e, W_OBJ | (want_grad ? W_GRAD : 0u) | W_CONS, s);
    if (rc)
        return rc;
    al_mu_kernel<<<a->nparts, 256, 0, s>>>(a->c, lam, a->gl, a->gu, a->m, a->rho, 1.0 / a->rho, a->mu, a->part,
                                           a->nparts);
    if (d_stats)
        al_stats_kernel<<<1, 32, 0, s>>>(a->obj, a->part, a->nparts, a->rho, d_stats);
    return al_check(cudaGetLastError(), "multiplier kernels");
}

}  // namespace

extern "C" {

int opf_al_create(opf_model *model, const opf_al_opts *opts, opf_al **out)
{
    if (!out) {
        set_error("out is NULL");
        return OPF_EINVAL;
    }
    *out = nullptr;
    if (!model || !model->M || !opts || !(opts->rho > 0.0) || !(opts->lr > 0.0) || !std::isfinite(opts->rho) ||
        !std::isfinite(opts->lr)) {
        set_error("opf_al_create: need a model and finite rho > 0, lr > 0");
        return OPF_EINVAL;
    }
    if (!model->M->on_device) {
        set_error("opf_al_create: structure-only model");
        return OPF_ESTATE;
    }
    opf_al *a = new opf_al();
    a->M = model->M;
    a->n = model->M->n;
    a->m = model->M->m;
    a->rho = opts->rho;
    a->lr = opts->lr;
    a->nparts = 148 * 4;
    std::vector<double> xl(a->n), xu(a->n), gl(a->m), gu(a->m);
    bounds(*a->M, xl.data(), xu.data(), gl.data(), gu.data());
    int rc = OPF_OK;
    if (!rc) rc = al_alloc(a, &a->xl, a->n);
    if (!rc) rc = al_alloc(a, &a->xu, a->n);
    if (!rc) rc = al_alloc(a, &a->gl, a->m);
    if (!rc) rc = al_alloc(a, &a->gu, a->m);
    if (!rc) rc = al_alloc(a, &a->grad, a->n);
    if (!rc) rc = al_alloc(a, &a->c, a->m);
    if (!rc) rc = al_alloc(a, &a->mu, a->m);
    if (!rc) rc = al_alloc(a, &a->u, a->n);
    if (!rc) rc = al_alloc(a, &a->m1, a->n);
    if (!rc) rc = al_alloc(a, &a->m2, a->n);
    if (!rc) rc = al_alloc(a, &a->obj, 1);
    if (!rc) rc = al_alloc(a, &a->part, 3 * (size_t)a->nparts);
    if (!rc) rc = al_alloc(a, &a->bpow, 6);
    if (!rc) {
        const double init[6] = {1.0, 1.0, 0.0, 0.0, 0.0, 0.0};
        rc = al_check(cudaMemcpy(a->bpow, init, sizeof(init), cudaMemcpyHostToDevice), "step state");
    }
    if (!rc)
        rc = al_check(cudaStreamCreateWithFlags(&a->cap, cudaStreamNonBlocking), "capture stream");
    if (!rc)
        rc = al_check(cudaMemcpy(a->xl, xl.data(), sizeof(double) * a->n, cudaMemcpyHostToDevice), "upload bounds");
    if (!rc)
        rc = al_check(cudaMemcpy(a->xu, xu.data(), sizeof(double) * a->n, cudaMemcpyHostToDevice), "upload bounds");
    if (!rc)
        rc = al_check(cudaMemcpy(a->gl, gl.data(), sizeof(double) * a->m, cudaMemcpyHostToDevice), "upload bounds");
    if (!rc)
        rc = al_check(cudaMemcpy(a->gu, gu.data(), sizeof(double) * a->m, cudaMemcpyHostToDevice), "upload bounds");
    if (!rc)
        rc = al_check(cudaMemset(a->m1, 0, sizeof(double) * a->n), "clear moments");
    if (!rc)
        rc = al_check(cudaMemset(a->m2, 0, sizeof(double) * a->n), "clear moments");
    if (rc) {
        al_free(a);
        return rc;
    }
    *out = a;
    return OPF_OK;
}

int opf_al_destroy(opf_al *al)
{
    al_free(al);
    return OPF_OK;
}

int opf_al_reset(opf_al *al, double rho, double lr)
{
    if (!al || !(rho > 0.0) || !(lr > 0.0) || !std::isfinite(rho) || !std::isfinite(lr)) {
        set_error("opf_al_reset: need a loop and finite rho > 0, lr > 0");
        return OPF_EINVAL;
    }
    cudaDeviceSynchronize();  // no replay of the old graphs may still run
    al_drop_graphs(al);       // they hold rho and lr
    al->rho = rho;
    al->lr = lr;
    al->step = 0;
    const double init[6] = {1.0, 1.0, 0.0, 0.0, 0.0, 0.0};
    int rc = al_check(cudaMemset(al->m1, 0, sizeof(double) * al->n), "clear moments");
    if (!rc)
        rc = al_check(cudaMemset(al->m2, 0, sizeof(double) * al->n), "clear moments");
    if (!rc)
        rc = al_check(cudaMemcpy(al->bpow, init, sizeof(init), cudaMemcpyHostToDevice), "step state");
    return rc;
}

namespace {

// one inner iteration on stream s: grad f and g at x; J^T mu with mu formed
// from g where the product reads it (and the step count advanced); Adam
int al_inner(opf_al *al, double *d_x, const double *d_lambda, cudaStream_t s)
{
    // the whole gradient in one kernel where the model allows it; else the
    // constraints and grad f, then J^T mu formed from them
    const bool one = al_grad_fused_ok(*al->M);
    int rc = OPF_OK;
    if (one) {
        rc = launch_al_grad(*al->M, d_x, d_lambda, al->gl, al->gu, al->rho, al->u, al->bpow, s);
    } else {
        EvalArgs e{d_x, nullptr, 1.0, nullptr, al->grad, al->c, nullptr, nullptr};
        rc = launch_eval(*al->M, e, W_GRAD | W_CONS, s);
        if (!rc)
            rc = launch_jtprod_al(*al->M, d_x, al->c, d_lambda, al->gl, al->gu, al->rho, al->u, al->bpow, s);
    }
    if (rc)
        return rc;
    al_adam_kernel<<<grid_of(al->n), 256, 0, s>>>(d_x, one ? nullptr : al->grad, al->u, al->xl, al->xu, al->m1,
                                                  al->m2, al->n, al->lr, al->bpow);
    return al_check(cudaGetLastError(), "Adam step");
}

// the captured iteration for (x, lambda), built on first use
int al_graph(opf_al *al, double *d_x, const double *d_lambda, cudaGraphExec_t *out)
{
    for (auto &g : al->graphs)
        if (g.x == d_x && g.lam == d_lambda) {
            *out = g.exec;
            return OPF_OK;
        }
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int rc = al_check(cudaStreamBeginCapture(al->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    if (rc)
        return rc;
    const int rc_inner = al_inner(al, d_x, d_lambda, al->cap);
    cudaError_t e = cudaStreamEndCapture(al->cap, &graph);
    if (rc_inner)
        rc = rc_inner;
    else if (e == cudaSuccess)
        rc = al_check(cudaGraphInstantiate(&exec, graph, 0), "graph instantiate");
    else
        rc = al_check(e, "end capture");
    if (graph)
        cudaGraphDestroy(graph);
    if (rc)
        return rc;
    al->graphs.push_back({d_x, d_lambda, exec});
    *out = exec;
    return OPF_OK;
}

}  // namespace

int opf_al_iterate(opf_al *al, double *d_x, const double *d_lambda, int32_t iters, double *d_stats, void *stream)
{
    if (!al || !d_x || !d_lambda || iters < 0) {
        set_error("opf_al_iterate: need a loop, d_x, d_lambda and iters >= 0");
        return OPF_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaGraphExec_t exec = nullptr;
    int rc = iters > 0 ? al_graph(al, d_x, d_lambda, &exec) : OPF_OK;
    for (int it = 0; it < iters && !rc; it++)
        rc = al_check(cudaGraphLaunch(exec, s), "graph launch");
    al->step += iters;
    if (!rc && d_stats)  // statistics at the final point
        rc = al_point(al, d_x, d_lambda, false, d_stats, s);
    return rc;
}

int opf_al_update(opf_al *al, const double *d_x, double *d_lambda, double *d_stats, void *stream)
{
    if (!al || !d_x || !d_lambda) {
        set_error("opf_al_update: need a loop, d_x and d_lambda");
        return OPF_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = al_point(al, d_x, d_lambda, false, d_stats, s);
    if (!rc)
        rc = al_check(cudaMemcpyAsync(d_lambda, al->mu, sizeof(double) * al->m, cudaMemcpyDeviceToDevice, s),
                      "multiplier update");
    return rc;
}

}  // extern "C"

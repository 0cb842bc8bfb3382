// Augmented-Lagrangian loop (include/opf_al.h): Adam inner iterations on
// L(x; lambda) with the library's callback kernels, multiplier updates, and
// the statistics of a point, all on the device.
#include <climits>
#include <cmath>
#include <vector>

#include "../../include/opf_al.h"
#include "model.h"

namespace opf {
void bounds(const Model &M, double *xl, double *xu, double *gl, double *gu);
void jac_pattern(const Model &M, int64_t *rows, int64_t *cols);
void hess_pattern(const Model &M, int64_t *rows, int64_t *cols);
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
    // projected Newton-CG step (opf_al_newton), set up on first use: the
    // Jacobian as CSR (its pattern order) and CSC (a permutation of its
    // values), the Hessian's lower triangle as CSR and its strict upper part
    // (the transpose) as CSR with a permutation, the diagonal's position
    bool nt_ready = false;
    int32_t *jptr = nullptr, *jcol = nullptr, *tptr = nullptr, *trow = nullptr, *tperm = nullptr;
    int32_t *hptr = nullptr, *hcol = nullptr, *uptr = nullptr, *ucol = nullptr, *uperm = nullptr, *hdiag = nullptr;
    double *jv = nullptr, *hv = nullptr, *G = nullptr, *r = nullptr, *z = nullptr, *dv = nullptr, *q = nullptr;
    double *p = nullptr, *minv = nullptr, *t = nullptr, *Dm = nullptr, *xt = nullptr, *tstats = nullptr;
    double *cgs = nullptr;  // device scalars of the step (see nt_scalar_kernel), delta kept across steps
    double *mdiag = nullptr;  // Jacobi diagonal of K
    unsigned char *F = nullptr;  // free entries
    // the CG loop of a step as one CUDA graph (its kernels read only the
    // loop's own buffers), captured for one iteration count at a time
    cudaGraphExec_t cg_exec = nullptr;
    int cg_iters = 0;
    unsigned *ticket = nullptr;  // last-block counter of the CG reductions (0 between launches)
    // the step's Jacobian values in CSC order (jv[tperm]) and the Hessian's
    // strict upper part in its CSR order (hv[uperm]), gathered once per step
    // so that the CG products read them without the permutation
    double *jvt = nullptr, *hvu = nullptr;
    int64_t nu = 0;  // strict upper entries of the Hessian
};

// the Newton step's device scalars (opf_al_newton)
enum { CG_RZ = 0, CG_RZ0, CG_ALPHA, CG_BETA, CG_DONE, CG_GP, CG_COPY, CG_MOVE, CG_ASTAR, CG_DELTA, CG_SCALE, CG_N };
constexpr double kDelta0 = 1e-2;  // first Levenberg-Marquardt weight

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
    if (a->cg_exec)
        cudaGraphExecDestroy(a->cg_exec);
    a->cg_exec = nullptr;
    a->cg_iters = 0;
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
    if (!rc && al->nt_ready)  // the Newton step's first weight again
        rc = al_check(cudaMemcpy(al->cgs + CG_DELTA, &kDelta0, sizeof(double), cudaMemcpyHostToDevice), "delta");
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

// ---- projected Newton-CG step (opf_al_newton) -------------------------
//
// K = H(x; mu, 1) + rho J^T diag(D) J (H the Lagrangian Hessian, D_i = 1
// where s_i = c_i + lambda_i / rho lies outside [gl_i, gu_i]); Jacobi-
// preconditioned CG on K p = -G over the free entries; a backtracking search
// over eight step lengths. Every reduction is a fixed-order two-level sum
// (block partials, then one warp), and every scalar of the iteration lives
// on the device, so the whole step runs without a host round trip.

constexpr int kNls = 8;  // trial step lengths 1, 1/2, ..., 1/128


// per-column setup: G = grad f + J^T mu; the free set; the Jacobi diagonal
// M_j = H_jj + rho sum_i D_i J_ij^2 (1 where <= 1e-12) and the inverse of
// the preconditioner M_j (1 + delta); r = -G on the free set, z, d = z,
// p = 0; block partials of r^T z
// out[k] = v[perm[k]] for k < count, two arrays in one pass
__global__ void nt_gather_kernel(int64_t n1, const int32_t *perm1, const double *v1, double *out1, int64_t n2,
                                 const int32_t *perm2, const double *v2, double *out2)
{
    const int64_t total = n1 > n2 ? n1 : n2;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        if (k < n1)
            out1[k] = v1[perm1[k]];
        if (k < n2)
            out2[k] = v2[perm2[k]];
    }
}

__global__ void nt_setup_kernel(int64_t n, const double *grad, const double *jv, const int32_t *tptr,
                                const int32_t *trow, const int32_t *tperm, const double *mu, const double *Dm,
                                const double *hv, const int32_t *hdiag, double rho, const double *x, const double *xl,
                                const double *xu, double *G, unsigned char *F, double *mdiag, double *minv, double *r,
                                double *z, double *dv, double *p, double *part, int nparts, const double *cgs)
{
    const double delta = cgs[CG_DELTA];
    __shared__ double red[32];
    double acc = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        double g = 0.0, dsum = 0.0;
        for (int32_t k = tptr[j]; k < tptr[j + 1]; k++) {
            const double a = jv[tperm[k]];
            const int32_t i = trow[k];
            g = fma(a, mu[i], g);
            dsum = fma(Dm[i] * a, a, dsum);
        }
        g += grad[j];
        const bool free_j = !((x[j] <= xl[j] && g > 0.0) || (x[j] >= xu[j] && g < 0.0));
        double mj = fma(rho, dsum, hdiag[j] >= 0 ? hv[hdiag[j]] : 0.0);
        if (mj <= 1e-12)
            mj = 1.0;
        const double mi = 1.0 / (mj * (1.0 + delta));
        const double rj = free_j ? -g : 0.0;
        const double zj = rj * mi;
        G[j] = g;
        F[j] = free_j;
        mdiag[j] = mj;
        minv[j] = mi;
        r[j] = rj;
        z[j] = zj;
        dv[j] = zj;
        p[j] = 0.0;
        acc = fma(rj, zj, acc);
    }
    const double b = block_sum(acc, red);
    if (threadIdx.x == 0)
        part[blockIdx.x] = b;
}

// D_i from s_i = c_i + lambda_i / rho (as the multiplier kernel forms it)
__global__ void nt_active_kernel(int64_t m, const double *c, const double *lam, const double *gl, const double *gu,
                                 double inv_rho, double *Dm)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const double s = fma(lam ? lam[i] : 0.0, inv_rho, c[i]);
        Dm[i] = (s < gl[i] || s > gu[i]) ? 1.0 : 0.0;
    }
}

// acc + sum over e in [e0, e1) of val[e] x[idx[e]], added in order of e:
// the first eight entries' indices and values are loaded together and then
// their gathers (a row's loads in flight at once rather than one dependent
// pair per entry), the rest one by one
__device__ __forceinline__ double row_dot(const int32_t *idx, const double *val, const double *x, int32_t e0,
                                          int32_t e1, double acc)
{
    int32_t c[8];
    double v[8], g[8];
#pragma unroll
    for (int u = 0; u < 8; u++)
        if (e0 + u < e1) {
            c[u] = __ldg(idx + e0 + u);
            v[u] = __ldg(val + e0 + u);
        }
#pragma unroll
    for (int u = 0; u < 8; u++)
        if (e0 + u < e1)
            g[u] = x[c[u]];
#pragma unroll
    for (int u = 0; u < 8; u++)
        if (e0 + u < e1)
            acc = fma(v[u], g[u], acc);
    for (int32_t e = e0 + 8; e < e1; e++)
        acc = fma(val[e], x[idx[e]], acc);
    return acc;
}

// t_i = D_i (J d)_i
__global__ void nt_jd_kernel(int64_t m, const int32_t *jptr, const int32_t *jcol, const double *jv, const double *Dm,
                             const double *dv, double *t, const double *cgs)
{
    if (cgs[CG_DONE] != 0.0)
        return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        if (Dm[i] != 0.0)
            acc = row_dot(jcol, jv, dv, jptr[i], jptr[i + 1], acc);
        t[i] = acc;
    }
}

enum { NT_INIT, NT_DQ, NT_RZ, NT_GP, NT_PMAX };

// the sum of the partials (one warp, fixed order) and the step's scalar logic
// the scalar step of a mode from the sum v of the partials (one thread)
__device__ void nt_scalar_apply(double v, double *cgs, int mode, int k)
{
    if (mode == NT_INIT) {
        cgs[CG_RZ] = cgs[CG_RZ0] = v;
        cgs[CG_DONE] = v == 0.0 ? 1.0 : 0.0;
        cgs[CG_COPY] = 0.0;
    } else if (mode == NT_DQ) {
        if (cgs[CG_DONE] != 0.0)
            return;
        if (v <= 0.0) {  // non-positive curvature: stop (the first direction itself if k == 0)
            cgs[CG_DONE] = 1.0;
            cgs[CG_COPY] = k == 0 ? 1.0 : 0.0;
        } else {
            cgs[CG_ALPHA] = cgs[CG_RZ] / v;
        }
    } else if (mode == NT_RZ) {
        if (cgs[CG_DONE] != 0.0)
            return;
        if (v <= 1e-24 * cgs[CG_RZ0]) {
            cgs[CG_DONE] = 1.0;
        } else {
            cgs[CG_BETA] = v / cgs[CG_RZ];
            cgs[CG_RZ] = v;
        }
    } else {
        cgs[CG_GP] = v;
    }
}

// one warp: the partials summed in a fixed order (lane-strided, then a
// shuffle tree), then the mode's scalar step by lane 0
__device__ void nt_scalar_warp(const double *part, int nparts, double *cgs, int mode, int k)
{
    double v = 0.0;
    for (int q = threadIdx.x; q < nparts; q += 32)
        v += __ldcg(part + q);  // through L2: other blocks' partials
    for (int off = 16; off; off >>= 1)
        v += __shfl_down_sync(0xffffffffu, v, off);
    if (threadIdx.x == 0)
        nt_scalar_apply(v, cgs, mode, k);
}

__global__ void nt_scalar_kernel(const double *part, int nparts, double *cgs, int mode, int k)
{
    nt_scalar_warp(part, nparts, cgs, mode, k);
}

// the end of a kernel whose nparts (= gridDim.x) blocks each wrote one
// partial: every block takes a ticket after its partial is visible, and the
// block with the last ticket runs the scalar step (nt_scalar_warp, the same
// fixed-order sum) and returns the ticket to 0 for the next launch. Only
// that block writes the scalars, after every block has read them.
__device__ void nt_scalar_last(const double *part, int nparts, double *cgs, int mode, int k, unsigned *ticket)
{
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();  // this block's partial before its ticket
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x >= 32)
        return;
    __threadfence();
    nt_scalar_warp(part, nparts, cgs, mode, k);
    if (threadIdx.x == 0)
        *ticket = 0u;
}

// q = ((K + delta diag(M)) d) on the free set: the lower triangle, its
// transpose, rho J^T t, delta M_j d_j; block partials of d^T q
__global__ void nt_kd_kernel(int64_t n, const int32_t *hptr, const int32_t *hcol, const double *hv,
                             const int32_t *uptr, const int32_t *ucol, const double *hvu, const int32_t *tptr,
                             const int32_t *trow, const double *jvt, const double *t, double rho,
                             const unsigned char *F, const double *mdiag, const double *dv, double *q, double *part,
                             int nparts, double *cgs, int k_iter, unsigned *ticket)
{
    __shared__ double red[32];
    if (cgs[CG_DONE] != 0.0)
        return;
    const double delta = cgs[CG_DELTA];
    double acc = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        double h = row_dot(hcol, hv, dv, hptr[j], hptr[j + 1], 0.0);
        h = row_dot(ucol, hvu, dv, uptr[j], uptr[j + 1], h);
        const double a = row_dot(trow, jvt, t, tptr[j], tptr[j + 1], 0.0);
        const double qj = F[j] ? fma(delta * mdiag[j], dv[j], fma(rho, a, h)) : 0.0;
        q[j] = qj;
        acc = fma(dv[j], qj, acc);
    }
    const double b = block_sum(acc, red);
    if (threadIdx.x == 0)
        part[blockIdx.x] = b;
    nt_scalar_last(part, nparts, cgs, NT_DQ, k_iter, ticket);  // d^T q: alpha or the stop
}

// p += alpha d, r -= alpha q, z = r / M; block partials of r^T z (or, where
// the first curvature test failed, p = d)
__global__ void nt_update_kernel(int64_t n, const double *dv, const double *q, const double *minv, double *p, double *r,
                                 double *z, double *part, int nparts, double *cgs, int k_iter, unsigned *ticket)
{
    __shared__ double red[32];
    if (cgs[CG_DONE] != 0.0) {
        if (cgs[CG_COPY] != 0.0)
            for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
                 j += (int64_t)gridDim.x * blockDim.x)
                p[j] = dv[j];
        return;
    }
    const double a = cgs[CG_ALPHA];
    double acc = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        p[j] = fma(a, dv[j], p[j]);
        const double rj = fma(-a, q[j], r[j]);
        const double zj = rj * minv[j];
        r[j] = rj;
        z[j] = zj;
        acc = fma(rj, zj, acc);
    }
    const double b = block_sum(acc, red);
    if (threadIdx.x == 0)
        part[blockIdx.x] = b;
    nt_scalar_last(part, nparts, cgs, NT_RZ, k_iter, ticket);  // r^T z: beta or the stop
}

// d = z + beta d
__global__ void nt_dir_kernel(int64_t n, const double *z, double *dv, const double *cgs)
{
    if (cgs[CG_DONE] != 0.0)
        return;
    const double b = cgs[CG_BETA];
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        dv[j] = fma(b, dv[j], z[j]);
}

// block partials of a^T b
__global__ void nt_dot_kernel(int64_t n, const double *a, const double *b, double *part, int nparts)
{
    __shared__ double red[32];
    double acc = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        acc = fma(a[j], b[j], acc);
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0)
        part[blockIdx.x] = s;
}

// max |p_j| (block partials, then one warp): the step's cap, scale =
// 1 / max|p_j| where that is above 1
__global__ void nt_pmax_kernel(int64_t n, const double *p, double *part)
{
    __shared__ double red[32];
    double v = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        v = fmax(v, fabs(p[j]));
    const double b = block_max(v, red);
    if (threadIdx.x == 0)
        part[blockIdx.x] = b;
}

__global__ void nt_pscale_kernel(const double *part, int nparts, double *cgs)
{
    double v = 0.0;
    for (int q = threadIdx.x; q < nparts; q += 32)
        v = fmax(v, part[q]);
    for (int off = 16; off; off >>= 1)
        v = fmax(v, __shfl_down_sync(0xffffffffu, v, off));
    if (threadIdx.x == 0)
        cgs[CG_SCALE] = v > 1.0 ? 1.0 / v : 1.0;
}

__global__ void nt_scale_kernel(int64_t n, double *p, const double *cgs)
{
    const double c = cgs[CG_SCALE];
    if (c == 1.0)
        return;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        p[j] = p[j] * c;
}

// x = clip(x, xl, xu)
__global__ void nt_clip_kernel(int64_t n, double *x, const double *xl, const double *xu)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        x[j] = fmin(fmax(x[j], xl[j]), xu[j]);
}

// trial point x_t = clip(x + a p, xl, xu)
__global__ void nt_trial_kernel(int64_t n, const double *x, const double *p, double a, const double *xl,
                                const double *xu, double *xt)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        xt[j] = fmin(fmax(fma(a, p[j], x[j]), xl[j]), xu[j]);
}

// the step length: the largest 2^-t with L_t <= L_0 + 1e-4 2^-t G^T p, else
// the one of least L_t if below L_0, else none (tstats: [3] per trial, then
// the base point's); the next Levenberg-Marquardt weight: delta / 4 after a
// full step, delta 10 after a step of 1/8 or less (or none), within
// [1e-8, 1e4]
__global__ void nt_select_kernel(const double *tstats, double *cgs)
{
    const double L0 = tstats[3 * kNls + 2], gp = cgs[CG_GP];
    int pick = -1;
    for (int t = 0; t < kNls && pick < 0; t++)
        if (tstats[3 * t + 2] <= fma(1e-4 * ldexp(1.0, -t), gp, L0))
            pick = t;
    if (pick < 0) {
        int best = 0;
        for (int t = 1; t < kNls; t++)
            if (tstats[3 * t + 2] < tstats[3 * best + 2])
                best = t;
        if (tstats[3 * best + 2] < L0)
            pick = best;
    }
    cgs[CG_MOVE] = pick >= 0 ? 1.0 : 0.0;
    cgs[CG_ASTAR] = pick >= 0 ? ldexp(1.0, -pick) : 0.0;
    double dl = cgs[CG_DELTA];
    if (pick == 0)
        dl = dl / 4.0;
    else if (pick < 0 || pick > 2)
        dl = dl * 10.0;
    cgs[CG_DELTA] = fmin(fmax(dl, 1e-8), 1e4);
}

__global__ void nt_apply_kernel(int64_t n, double *x, const double *p, const double *xl, const double *xu,
                                const double *cgs)
{
    if (cgs[CG_MOVE] == 0.0)
        return;
    const double a = cgs[CG_ASTAR];
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        x[j] = fmin(fmax(fma(a, p[j], x[j]), xl[j]), xu[j]);
}

// host: the sparse structures of the step, from the model's patterns
int nt_setup(opf_al *a)
{
    if (a->nt_ready)
        return OPF_OK;
    const Model &M = *a->M;
    const int64_t n = a->n, m = a->m, nj = M.nnzj, nh = M.nnzh;
    if (nj >= INT32_MAX || nh >= INT32_MAX || n >= INT32_MAX || m >= INT32_MAX) {
        set_error("opf_al_newton: model too large for 32-bit sparse indices");
        return OPF_EINVAL;
    }
    std::vector<int64_t> jr(nj), jc(nj), hr(nh), hc(nh);
    jac_pattern(M, jr.data(), jc.data());
    hess_pattern(M, hr.data(), hc.data());
    std::vector<int32_t> jptr(m + 1, 0), jcol(nj), tptr(n + 1, 0), trow(nj), tperm(nj);
    for (int64_t k = 0; k < nj; k++) {
        jptr[jr[k] + 1]++;
        tptr[jc[k] + 1]++;
        jcol[k] = (int32_t)jc[k];
    }
    for (int64_t i = 0; i < m; i++)
        jptr[i + 1] += jptr[i];
    for (int64_t j = 0; j < n; j++)
        tptr[j + 1] += tptr[j];
    {  // CSC: entries of each column in ascending row (the pattern is row-major)
        std::vector<int32_t> fill(tptr.begin(), tptr.end() - 1);
        for (int64_t k = 0; k < nj; k++) {
            const int32_t at = fill[jc[k]]++;
            trow[at] = (int32_t)jr[k];
            tperm[at] = (int32_t)k;
        }
    }
    std::vector<int32_t> hptr(n + 1, 0), hcol(nh), uptr(n + 1, 0), hdiag(n, -1);
    for (int64_t k = 0; k < nh; k++) {
        hptr[hr[k] + 1]++;
        hcol[k] = (int32_t)hc[k];
        if (hr[k] == hc[k])
            hdiag[hr[k]] = (int32_t)k;
        else
            uptr[hc[k] + 1]++;
    }
    for (int64_t j = 0; j < n; j++) {
        hptr[j + 1] += hptr[j];
        uptr[j + 1] += uptr[j];
    }
    std::vector<int32_t> ucol(uptr[n]), uperm(uptr[n]);
    {
        std::vector<int32_t> fill(uptr.begin(), uptr.end() - 1);
        for (int64_t k = 0; k < nh; k++)
            if (hr[k] != hc[k]) {
                const int32_t at = fill[hc[k]]++;
                ucol[at] = (int32_t)hr[k];
                uperm[at] = (int32_t)k;
            }
    }
    auto up = [&](int32_t **dst, const std::vector<int32_t> &v) {
        int rc = al_alloc(a, dst, v.size());
        if (!rc && !v.empty())
            rc = al_check(cudaMemcpy(*dst, v.data(), sizeof(int32_t) * v.size(), cudaMemcpyHostToDevice),
                          "upload Newton structures");
        return rc;
    };
    int rc = OPF_OK;
    if (!rc) rc = up(&a->jptr, jptr);
    if (!rc) rc = up(&a->jcol, jcol);
    if (!rc) rc = up(&a->tptr, tptr);
    if (!rc) rc = up(&a->trow, trow);
    if (!rc) rc = up(&a->tperm, tperm);
    if (!rc) rc = up(&a->hptr, hptr);
    if (!rc) rc = up(&a->hcol, hcol);
    if (!rc) rc = up(&a->uptr, uptr);
    if (!rc) rc = up(&a->ucol, ucol);
    if (!rc) rc = up(&a->uperm, uperm);
    if (!rc) rc = up(&a->hdiag, hdiag);
    if (!rc) rc = al_alloc(a, &a->jv, nj);
    if (!rc) rc = al_alloc(a, &a->hv, nh);
    if (!rc) rc = al_alloc(a, &a->jvt, nj);
    if (!rc) rc = al_alloc(a, &a->hvu, ucol.size());
    a->nu = (int64_t)ucol.size();
    for (double **v : {&a->G, &a->r, &a->z, &a->dv, &a->q, &a->p, &a->minv, &a->xt})
        if (!rc)
            rc = al_alloc(a, v, n);
    if (!rc) rc = al_alloc(a, &a->t, m);
    if (!rc) rc = al_alloc(a, &a->Dm, m);
    if (!rc) rc = al_alloc(a, &a->tstats, 3 * (kNls + 1));
    if (!rc) rc = al_alloc(a, &a->cgs, CG_N);
    if (!rc) rc = al_alloc(a, &a->ticket, 1);
    if (!rc) rc = al_alloc(a, &a->F, n);
    if (!rc) rc = al_alloc(a, &a->mdiag, n);
    if (!rc)
        rc = al_check(cudaMemcpy(a->cgs + CG_DELTA, &kDelta0, sizeof(double), cudaMemcpyHostToDevice), "delta");
    if (!rc)
        a->nt_ready = true;
    return rc;
}

// one projected Newton-CG step on stream s (see opf_al_newton)
// the CG iterations of a step, four kernels each (the d^T q and r^T z
// scalar steps run in the last block of the kernels that form the partials),
// launched on stream s
void nt_cg_kernels(opf_al *a, int cg_iters, cudaStream_t s)
{
    const int64_t n = a->n, m = a->m;
    const int gn = grid_of(n), gm = grid_of(m), np = a->nparts;
    for (int k = 0; k < cg_iters; k++) {
        nt_jd_kernel<<<gm, 256, 0, s>>>(m, a->jptr, a->jcol, a->jv, a->Dm, a->dv, a->t, a->cgs);
        nt_kd_kernel<<<np, 256, 0, s>>>(n, a->hptr, a->hcol, a->hv, a->uptr, a->ucol, a->hvu, a->tptr, a->trow,
                                        a->jvt, a->t, a->rho, a->F, a->mdiag, a->dv, a->q, a->part, np, a->cgs, k,
                                        a->ticket);
        nt_update_kernel<<<np, 256, 0, s>>>(n, a->dv, a->q, a->minv, a->p, a->r, a->z, a->part, np, a->cgs, k,
                                            a->ticket);
        nt_dir_kernel<<<gn, 256, 0, s>>>(n, a->z, a->dv, a->cgs);
    }
}

// the CG iterations as one CUDA graph (captured on the loop's private
// stream, replayed on the caller's): the kernels read only the loop's own
// buffers and rho, so the graph serves every step with the same iteration
// count until a reset changes rho
int nt_cg_graph(opf_al *a, int cg_iters, cudaGraphExec_t *out)
{
    if (a->cg_exec && a->cg_iters == cg_iters) {
        *out = a->cg_exec;
        return OPF_OK;
    }
    if (a->cg_exec)
        cudaGraphExecDestroy(a->cg_exec);
    a->cg_exec = nullptr;
    a->cg_iters = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int rc = al_check(cudaStreamBeginCapture(a->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    if (rc)
        return rc;
    nt_cg_kernels(a, cg_iters, a->cap);
    const cudaError_t le = cudaGetLastError();
    const cudaError_t e = cudaStreamEndCapture(a->cap, &graph);
    if (le != cudaSuccess)
        rc = al_check(le, "CG kernels");
    else if (e != cudaSuccess)
        rc = al_check(e, "end capture");
    else
        rc = al_check(cudaGraphInstantiate(&exec, graph, 0), "graph instantiate");
    if (graph)
        cudaGraphDestroy(graph);
    if (rc)
        return rc;
    a->cg_exec = exec;
    a->cg_iters = cg_iters;
    *out = exec;
    return OPF_OK;
}

int nt_step(opf_al *a, double *d_x, const double *d_lambda, int cg_iters, double *d_stats, cudaStream_t s)
{
    const int64_t n = a->n, m = a->m;
    const int gn = grid_of(n), gm = grid_of(m), np = a->nparts;
    nt_clip_kernel<<<gn, 256, 0, s>>>(n, d_x, a->xl, a->xu);  // the step starts inside the bounds
    // base point: f, grad f, g, J; the multipliers mu and the statistics (L_0)
    EvalArgs e{d_x, nullptr, 1.0, a->obj, a->grad, a->c, a->jv, nullptr};
    int rc = launch_eval(*a->M, e, W_OBJ | W_GRAD | W_CONS | W_JAC, s);
    if (rc)
        return rc;
    al_mu_kernel<<<np, 256, 0, s>>>(a->c, d_lambda, a->gl, a->gu, m, a->rho, 1.0 / a->rho, a->mu, a->part, np);
    al_stats_kernel<<<1, 32, 0, s>>>(a->obj, a->part, np, a->rho, a->tstats + 3 * kNls);
    nt_active_kernel<<<gm, 256, 0, s>>>(m, a->c, d_lambda, a->gl, a->gu, 1.0 / a->rho, a->Dm);
    // the Lagrangian Hessian with the AL multipliers mu, sigma = 1
    EvalArgs eh{d_x, a->mu, 1.0, nullptr, nullptr, nullptr, nullptr, a->hv};
    rc = launch_eval(*a->M, eh, W_HESS, s);
    if (rc)
        return rc;
    {
        const int64_t nj = a->M->nnzj, big = nj > a->nu ? nj : a->nu;
        nt_gather_kernel<<<grid_of(big), 256, 0, s>>>(nj, a->tperm, a->jv, a->jvt, a->nu, a->uperm, a->hv, a->hvu);
    }
    nt_setup_kernel<<<np, 256, 0, s>>>(n, a->grad, a->jv, a->tptr, a->trow, a->tperm, a->mu, a->Dm, a->hv, a->hdiag,
                                       a->rho, d_x, a->xl, a->xu, a->G, a->F, a->mdiag, a->minv, a->r, a->z, a->dv,
                                       a->p, a->part, np, a->cgs);
    nt_scalar_kernel<<<1, 32, 0, s>>>(a->part, np, a->cgs, NT_INIT, 0);
    cudaGraphExec_t cg = nullptr;
    rc = nt_cg_graph(a, cg_iters, &cg);
    if (!rc)  // the counter is 0 after every complete launch; set it so for this step in any case
        rc = al_check(cudaMemsetAsync(a->ticket, 0, sizeof(unsigned), s), "CG ticket");
    if (!rc)
        rc = al_check(cudaGraphLaunch(cg, s), "CG graph launch");
    if (rc)
        return rc;
    // no entry moves by more than 1 (per-unit) in one step
    nt_pmax_kernel<<<np, 256, 0, s>>>(n, a->p, a->part);
    nt_pscale_kernel<<<1, 32, 0, s>>>(a->part, np, a->cgs);
    nt_scale_kernel<<<gn, 256, 0, s>>>(n, a->p, a->cgs);
    nt_dot_kernel<<<np, 256, 0, s>>>(n, a->G, a->p, a->part, np);
    nt_scalar_kernel<<<1, 32, 0, s>>>(a->part, np, a->cgs, NT_GP, 0);
    for (int t = 0; t < kNls && !rc; t++) {
        nt_trial_kernel<<<gn, 256, 0, s>>>(n, d_x, a->p, ldexp(1.0, -t), a->xl, a->xu, a->xt);
        rc = al_point(a, a->xt, d_lambda, false, a->tstats + 3 * t, s);
    }
    if (rc)
        return rc;
    nt_select_kernel<<<1, 1, 0, s>>>(a->tstats, a->cgs);
    nt_apply_kernel<<<gn, 256, 0, s>>>(n, d_x, a->p, a->xl, a->xu, a->cgs);
    rc = al_check(cudaGetLastError(), "line search kernels");
    if (!rc && d_stats)
        rc = al_point(a, d_x, d_lambda, false, d_stats, s);
    return rc;
}

}  // namespace

int opf_al_newton(opf_al *al, double *d_x, const double *d_lambda, int32_t cg_iters, double *d_stats,
                  double *d_step, void *stream)
{
    if (!al || !d_x || !d_lambda || cg_iters < 1) {
        set_error("opf_al_newton: need a loop, d_x, d_lambda and cg_iters >= 1");
        return OPF_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = nt_setup(al);
    if (!rc)
        rc = nt_step(al, d_x, d_lambda, cg_iters, d_stats, s);
    if (!rc && d_step)
        rc = al_check(cudaMemcpyAsync(d_step, al->p, sizeof(double) * al->n, cudaMemcpyDeviceToDevice, s),
                      "copy the CG direction");
    return rc;
}

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

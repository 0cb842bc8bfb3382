// extern "C" entry points of libopf (declared in include/opf.h).
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "model.h"

namespace opf {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

int build_model(const opf_network *nets, int32_t ninst, const opf_batch_opts *opts, bool device, Model **out);
void free_model(Model *M);
void jac_pattern(const Model &M, int64_t *rows, int64_t *cols);
void hess_pattern(const Model &M, int64_t *rows, int64_t *cols);
void bounds(const Model &M, double *xl, double *xu, double *gl, double *gu);

}  // namespace opf

using namespace opf;

namespace {

int check(const opf_model *m)
{
    if (!m || !m->M) {
        set_error("NULL model");
        return OPF_EINVAL;
    }
    return OPF_OK;
}

// eval-type calls need the device arrays
int check_dev(const opf_model *m)
{
    int rc = check(m);
    if (rc)
        return rc;
    if (!m->M->on_device) {
        set_error("structure-only model: create it with opf_model_create / opf_batch_create to evaluate");
        return OPF_ESTATE;
    }
    return OPF_OK;
}

int eval(opf_model *m, unsigned what, const EvalArgs &a, void *stream, int phases = 3)
{
    int rc = check_dev(m);
    if (rc)
        return rc;
    if (!a.x) {
        set_error("d_x is NULL");
        return OPF_EINVAL;
    }
    if ((what & W_HESS) && !a.lam) {
        set_error("d_lambda is NULL but the Hessian was requested");
        return OPF_EINVAL;
    }
    if (!what)
        return OPF_OK;
    return launch_eval(*m->M, a, what, static_cast<cudaStream_t>(stream), phases);
}

unsigned mask_of(const EvalArgs &a)
{
    return (a.obj ? W_OBJ : 0u) | (a.grad ? W_GRAD : 0u) | (a.c ? W_CONS : 0u) |
           (a.jac ? W_JAC : 0u) | (a.hess ? W_HESS : 0u);
}

}  // namespace

extern "C" {

const char *opf_last_error(void) { return g_err; }

int opf_model_create(const opf_network *net, opf_model **out)
{
    if (!out) {
        set_error("out is NULL");
        return OPF_EINVAL;
    }
    *out = nullptr;
    if (!net) {
        set_error("net is NULL");
        return OPF_EINVAL;
    }
    Model *M = nullptr;
    int rc = build_model(net, 1, nullptr, true, &M);
    if (rc)
        return rc;
    *out = new opf_model{M};
    return OPF_OK;
}

int opf_batch_create(const opf_network *nets, int32_t ninst, const opf_batch_opts *opts,
                     opf_model **out)
{
    if (!out) {
        set_error("out is NULL");
        return OPF_EINVAL;
    }
    *out = nullptr;
    Model *M = nullptr;
    int rc = build_model(nets, ninst, opts, true, &M);
    if (rc)
        return rc;
    *out = new opf_model{M};
    return OPF_OK;
}

int opf_structure_create(const opf_network *nets, int32_t ninst, const opf_batch_opts *opts,
                         opf_model **out)
{
    if (!out) {
        set_error("out is NULL");
        return OPF_EINVAL;
    }
    *out = nullptr;
    Model *M = nullptr;
    int rc = build_model(nets, ninst, opts, false, &M);
    if (rc)
        return rc;
    *out = new opf_model{M};
    return OPF_OK;
}

int opf_model_destroy(opf_model *m)
{
    if (!m)
        return OPF_OK;
    free_model(m->M);
    delete m;
    return OPF_OK;
}

int opf_dims(const opf_model *m, int64_t *n, int64_t *mm, int64_t *nnzj, int64_t *nnzh)
{
    int rc = check(m);
    if (rc)
        return rc;
    if (n)
        *n = m->M->n;
    if (mm)
        *mm = m->M->m;
    if (nnzj)
        *nnzj = m->M->nnzj;
    if (nnzh)
        *nnzh = m->M->nnzh;
    return OPF_OK;
}

int opf_sparsity(const opf_model *m, int32_t kind, int64_t *rows, int64_t *cols)
{
    int rc = check(m);
    if (rc)
        return rc;
    if (!rows || !cols) {
        set_error("rows/cols NULL");
        return OPF_EINVAL;
    }
    if (kind == OPF_JAC)
        jac_pattern(*m->M, rows, cols);
    else if (kind == OPF_HESS)
        hess_pattern(*m->M, rows, cols);
    else {
        set_error("unknown pattern kind %d", kind);
        return OPF_EINVAL;
    }
    return OPF_OK;
}

int opf_bounds(const opf_model *m, double *xl, double *xu, double *gl, double *gu)
{
    int rc = check(m);
    if (rc)
        return rc;
    if ((xl == nullptr) != (xu == nullptr) || (gl == nullptr) != (gu == nullptr)) {
        set_error("bounds come in pairs (xl with xu, gl with gu)");
        return OPF_EINVAL;
    }
    bounds(*m->M, xl, xu, gl, gu);
    return OPF_OK;
}

int opf_eval_obj_grad(opf_model *m, const double *d_x, double *d_obj, double *d_grad, void *stream)
{
    EvalArgs a{d_x, nullptr, 1.0, d_obj, d_grad, nullptr, nullptr, nullptr};
    return eval(m, mask_of(a), a, stream);
}

int opf_eval_cons(opf_model *m, const double *d_x, double *d_c, void *stream)
{
    if (!d_c) {
        set_error("d_c is NULL");
        return OPF_EINVAL;
    }
    EvalArgs a{d_x, nullptr, 1.0, nullptr, nullptr, d_c, nullptr, nullptr};
    return eval(m, W_CONS, a, stream);
}

int opf_eval_jac(opf_model *m, const double *d_x, double *d_jvals, void *stream)
{
    if (!d_jvals) {
        set_error("d_jvals is NULL");
        return OPF_EINVAL;
    }
    EvalArgs a{d_x, nullptr, 1.0, nullptr, nullptr, nullptr, d_jvals, nullptr};
    return eval(m, W_JAC, a, stream);
}

int opf_eval_hess(opf_model *m, const double *d_x, const double *d_lambda, double obj_weight,
                  double *d_hvals, void *stream)
{
    if (!d_hvals) {
        set_error("d_hvals is NULL");
        return OPF_EINVAL;
    }
    EvalArgs a{d_x, d_lambda, obj_weight, nullptr, nullptr, nullptr, nullptr, d_hvals};
    return eval(m, W_HESS, a, stream);
}

int opf_eval_jac_hess(opf_model *m, const double *d_x, const double *d_lambda, double obj_weight,
                      double *d_jvals, double *d_hvals, void *stream)
{
    if (!d_jvals || !d_hvals) {
        set_error("d_jvals or d_hvals is NULL");
        return OPF_EINVAL;
    }
    EvalArgs a{d_x, d_lambda, obj_weight, nullptr, nullptr, nullptr, d_jvals, d_hvals};
    return eval(m, W_JAC | W_HESS, a, stream);
}

int opf_eval_all(opf_model *m, const double *d_x, const double *d_lambda, double obj_weight,
                 double *d_obj, double *d_grad, double *d_c, double *d_jvals, double *d_hvals,
                 void *stream)
{
    EvalArgs a{d_x, d_lambda, obj_weight, d_obj, d_grad, d_c, d_jvals, d_hvals};
    return eval(m, mask_of(a), a, stream);
}

int opf_eval_phases(opf_model *m, int32_t phases, const double *d_x, const double *d_lambda,
                    double obj_weight, double *d_obj, double *d_grad, double *d_c, double *d_jvals,
                    double *d_hvals, void *stream)
{
    if (phases < 1 || phases > 3) {
        set_error("phases must be OPF_PHASE_BRANCH, OPF_PHASE_BUS or both");
        return OPF_EINVAL;
    }
    EvalArgs a{d_x, d_lambda, obj_weight, d_obj, d_grad, d_c, d_jvals, d_hvals};
    return eval(m, mask_of(a), a, stream, phases);
}

namespace {
// the device staging of the host-buffer calls: x, lambda, obj, grad, c, J,
// H, each starting on a 512-byte boundary (like separately allocated
// buffers; packed 8 bytes apart they slowed the kernels' stores)
struct StageLayout {
    size_t x, l, obj, g, c, j, h, words;
};

StageLayout stage_layout(const Model &M)
{
    auto up = [](int64_t k) { return (size_t)((k + 63) / 64 * 64); };  // doubles, 512-byte multiples
    StageLayout L;
    L.x = 0;
    L.l = L.x + up(M.n);
    L.obj = L.l + up(M.m);
    L.g = L.obj + up(1);
    L.c = L.g + up(M.n);
    L.j = L.c + up(M.m);
    L.h = L.j + up(M.nnzj);
    L.words = L.h + up(M.nnzh);
    return L;
}
}  // namespace

int opf_eval_all_host(opf_model *m, const double *h_x, const double *h_lambda, double obj_weight,
                      double *h_obj, double *h_grad, double *h_c, double *h_jvals, double *h_hvals,
                      void *stream)
{
    int rc = check_dev(m);
    if (rc)
        return rc;
    Model &M = *m->M;
    if (!h_x || (h_hvals && !h_lambda)) {
        set_error("h_x is NULL, or h_lambda is NULL with h_hvals requested");
        return OPF_EINVAL;
    }
    // staging: x, lambda, obj, grad, c, J, H
    const StageLayout SL = stage_layout(M);
    const size_t need = sizeof(double) * SL.words;
    if (M.stage_bytes < need) {
        if (M.stage)
            cudaFree(M.stage);
        M.stage = nullptr;
        M.stage_bytes = 0;
        if (cudaMalloc(&M.stage, need) != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaMalloc of %zu staging bytes failed", need);
            return OPF_ENOMEM;
        }
        M.stage_bytes = need;
    }
    double *dx = M.stage + SL.x, *dl = M.stage + SL.l, *dobj = M.stage + SL.obj, *dg = M.stage + SL.g;
    double *dc = M.stage + SL.c, *dj = M.stage + SL.j, *dh = M.stage + SL.h;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(dx, h_x, sizeof(double) * M.n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && h_hvals)
        e = cudaMemcpyAsync(dl, h_lambda, sizeof(double) * M.m, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        set_error("host to device copy failed: %s", cudaGetErrorString(e));
        return OPF_ECUDA;
    }
    EvalArgs a{dx, h_hvals ? dl : nullptr, obj_weight, h_obj ? dobj : nullptr, h_grad ? dg : nullptr,
               h_c ? dc : nullptr, h_jvals ? dj : nullptr, h_hvals ? dh : nullptr};
    rc = eval(m, mask_of(a), a, stream);
    if (rc)
        return rc;
    struct {
        double *h;
        const double *d;
        int64_t n;
    } outs[5] = {{h_obj, dobj, 1}, {h_grad, dg, M.n}, {h_c, dc, M.m}, {h_jvals, dj, M.nnzj},
                 {h_hvals, dh, M.nnzh}};
    for (auto &o : outs)
        if (o.h && e == cudaSuccess)
            e = cudaMemcpyAsync(o.h, o.d, sizeof(double) * o.n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_error("device to host copy failed: %s", cudaGetErrorString(e));
        return OPF_ECUDA;
    }
    return OPF_OK;
}

int opf_eval_all_host_async(opf_model *m, const double *h_x, const double *h_lambda, double obj_weight,
                            double *h_obj, double *h_grad, double *h_c, double *h_jvals, double *h_hvals,
                            void *stream)
{
    int rc = check_dev(m);
    if (rc)
        return rc;
    Model &M = *m->M;
    if (!h_x || (h_hvals && !h_lambda)) {
        set_error("h_x is NULL, or h_lambda is NULL with h_hvals requested");
        return OPF_EINVAL;
    }
    const StageLayout SL = stage_layout(M);
    const size_t words = SL.words;
    if (!M.s_cmp) {  // first use: two staging slots, three streams, events
        bool ok = true;
        for (int k = 0; k < 2 && ok; k++)
            ok = cudaMalloc(&M.astage[k], sizeof(double) * words) == cudaSuccess;
        ok = ok && cudaStreamCreateWithFlags(&M.s_in, cudaStreamNonBlocking) == cudaSuccess &&
             cudaStreamCreateWithFlags(&M.s_cmp, cudaStreamNonBlocking) == cudaSuccess &&
             cudaStreamCreateWithFlags(&M.s_out, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&M.ev_entry, cudaEventDisableTiming) == cudaSuccess;
        for (int k = 0; k < 2 && ok; k++)
            ok = cudaEventCreateWithFlags(&M.ev_in[k], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&M.ev_cmp[k], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&M.ev_out[k], cudaEventDisableTiming) == cudaSuccess;
        if (!ok || !M.s_cmp) {
            cudaGetLastError();
            set_error("opf_eval_all_host_async: staging or stream creation failed");
            return OPF_ENOMEM;
        }
    }
    const int k = M.aslot;
    M.aslot ^= 1;
    double *const base = M.astage[k];
    double *dx = base + SL.x, *dl = base + SL.l, *dobj = base + SL.obj, *dg = base + SL.g;
    double *dc = base + SL.c, *dj = base + SL.j, *dh = base + SL.h;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // copy-in after the compute that last read this slot (not after the
    // caller's stream: it waits for the previous call's outputs, and
    // ordering on it would serialise the pipeline)
    cudaError_t e = cudaStreamWaitEvent(M.s_in, M.ev_cmp[k], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dx, h_x, sizeof(double) * M.n, cudaMemcpyHostToDevice, M.s_in);
    if (e == cudaSuccess && h_hvals)
        e = cudaMemcpyAsync(dl, h_lambda, sizeof(double) * M.m, cudaMemcpyHostToDevice, M.s_in);
    if (e == cudaSuccess) e = cudaEventRecord(M.ev_in[k], M.s_in);
    // compute after the copy-in and after the copy-out that last read this slot's outputs
    if (e == cudaSuccess) e = cudaStreamWaitEvent(M.s_cmp, M.ev_in[k], 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(M.s_cmp, M.ev_out[k], 0);
    if (e != cudaSuccess) {
        set_error("opf_eval_all_host_async: %s", cudaGetErrorString(e));
        return OPF_ECUDA;
    }
    EvalArgs a{dx, h_hvals ? dl : nullptr, obj_weight, h_obj ? dobj : nullptr, h_grad ? dg : nullptr,
               h_c ? dc : nullptr, h_jvals ? dj : nullptr, h_hvals ? dh : nullptr};
    rc = eval(m, mask_of(a), a, M.s_cmp);
    if (rc)
        return rc;
    e = cudaEventRecord(M.ev_cmp[k], M.s_cmp);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(M.s_out, M.ev_cmp[k], 0);
    struct {
        double *h;
        const double *d;
        int64_t n;
    } outs[5] = {{h_obj, dobj, 1}, {h_grad, dg, M.n}, {h_c, dc, M.m}, {h_jvals, dj, M.nnzj},
                 {h_hvals, dh, M.nnzh}};
    for (auto &o : outs)
        if (o.h && e == cudaSuccess)
            e = cudaMemcpyAsync(o.h, o.d, sizeof(double) * o.n, cudaMemcpyDeviceToHost, M.s_out);
    if (e == cudaSuccess) e = cudaEventRecord(M.ev_out[k], M.s_out);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, M.ev_out[k], 0);  // the caller's stream sees completion
    if (e != cudaSuccess) {
        set_error("opf_eval_all_host_async: %s", cudaGetErrorString(e));
        return OPF_ECUDA;
    }
    return OPF_OK;
}

int opf_host_register(void *ptr, size_t bytes)
{
    if (!ptr || bytes == 0) {
        set_error("opf_host_register: NULL pointer or zero size");
        return OPF_EINVAL;
    }
    cudaError_t e = cudaHostRegister(ptr, bytes, cudaHostRegisterDefault);
    if (e != cudaSuccess) {
        set_error("cudaHostRegister failed: %s", cudaGetErrorString(e));
        return OPF_ECUDA;
    }
    return OPF_OK;
}

int opf_host_unregister(void *ptr)
{
    if (!ptr) {
        set_error("opf_host_unregister: NULL pointer");
        return OPF_EINVAL;
    }
    cudaError_t e = cudaHostUnregister(ptr);
    if (e != cudaSuccess) {
        set_error("cudaHostUnregister failed: %s", cudaGetErrorString(e));
        return OPF_ECUDA;
    }
    return OPF_OK;
}

int opf_flat_start(opf_model *m, double *d_x, void *stream)
{
    int rc = check_dev(m);
    if (rc)
        return rc;
    if (!d_x) {
        set_error("d_x is NULL");
        return OPF_EINVAL;
    }
    return launch_flat_start(*m->M, d_x, static_cast<cudaStream_t>(stream));
}

int opf_sincos(opf_model *m, const double *d_angle, int64_t n, double *d_sin, double *d_cos,
               void *stream)
{
    int rc = check_dev(m);
    if (rc)
        return rc;
    if (n < 0 || (n > 0 && (!d_angle || !d_sin || !d_cos))) {
        set_error("opf_sincos: bad arguments");
        return OPF_EINVAL;
    }
    if (n == 0)
        return OPF_OK;
    return launch_sincos(*m->M, d_angle, n, d_sin, d_cos, static_cast<cudaStream_t>(stream));
}

int opf_eval_jtprod(opf_model *m, const double *d_x, const double *d_v, double *d_out, void *stream)
{
    int rc = check_dev(m);
    if (rc)
        return rc;
    if (!d_x || !d_v || !d_out) {
        set_error("opf_eval_jtprod: d_x, d_v and d_out are required");
        return OPF_EINVAL;
    }
    return launch_jtprod(*m->M, d_x, d_v, d_out, static_cast<cudaStream_t>(stream));
}

int opf_eval_flows(opf_model *m, double *d_x, void *stream)
{
    int rc = check_dev(m);
    if (rc)
        return rc;
    if (!d_x) {
        set_error("opf_eval_flows: d_x is NULL");
        return OPF_EINVAL;
    }
    return launch_flows(*m->M, d_x, static_cast<cudaStream_t>(stream));
}

int opf_set_loads(opf_model *m, const double *d_load_pd, const double *d_load_qd, void *stream)
{
    int rc = check_dev(m);
    if (rc)
        return rc;
    if (m->M->nload_total > 0 && (!d_load_pd || !d_load_qd)) {
        set_error("opf_set_loads: d_load_pd and d_load_qd are required");
        return OPF_EINVAL;
    }
    return launch_set_loads(*m->M, d_load_pd, d_load_qd, static_cast<cudaStream_t>(stream));
}

int opf_get_launch(const opf_model *m, opf_launch *cfg)
{
    int rc = check(m);
    if (rc)
        return rc;
    if (!cfg) {
        set_error("cfg is NULL");
        return OPF_EINVAL;
    }
    *cfg = m->M->launch;
    return OPF_OK;
}

int opf_set_launch(opf_model *m, const opf_launch *cfg)
{
    int rc = check(m);
    if (rc)
        return rc;
    if (!cfg) {
        set_error("cfg is NULL");
        return OPF_EINVAL;
    }
    for (int b : {cfg->branch_block, cfg->bus_block})
        if (b < 32 || b > 1024 || b % 32) {
            set_error("block size %d not a multiple of 32 in [32, 1024]", b);
            return OPF_EINVAL;
        }
    if (cfg->bus_order < 0 || cfg->bus_order > 3 || cfg->branch_occupancy < 0 || cfg->branch_occupancy > 2) {
        set_error("bus_order must be 0, 1, 2 or 3 and branch_occupancy 0, 1 or 2");
        return OPF_EINVAL;
    }
    if (cfg->branch_block > (cfg->branch_occupancy == 1 ? 256 : 512)) {
        set_error("branch_block %d above the branch kernel's limit (%d)", cfg->branch_block,
                  cfg->branch_occupancy == 1 ? 256 : 512);
        return OPF_EINVAL;
    }
    if (cfg->branch_ctas_per_sm < 0 || cfg->bus_ctas_per_sm < 0 || cfg->branch_ctas_per_sm > 64 ||
        cfg->bus_ctas_per_sm > 64) {
        set_error("ctas_per_sm must be in [0, 64]");
        return OPF_EINVAL;
    }
    m->M->launch = *cfg;
    return OPF_OK;
}

namespace {
// Time `reps` back-to-back fused evaluations in the model's current launch
// shape as one CUDA graph (the way evaluations are replayed in a solver
// loop), captured on `cs` and launched `launches` times; returns the best
// launch's time in ms, or a negative value on error.
float time_graph(Model &M, const EvalArgs &a, int reps, int launches, cudaStream_t cs, cudaEvent_t e0,
                 cudaEvent_t e1)
{
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return -1.f;
    int rc = OPF_OK;
    for (int r = 0; r < reps && !rc; r++)
        rc = launch_eval(M, a, W_OBJ | W_GRAD | W_CONS | W_JAC | W_HESS, cs);
    const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    if (rc || ce != cudaSuccess || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
        if (graph)
            cudaGraphDestroy(graph);
        cudaGetLastError();
        return -1.f;
    }
    float best = 1e30f;
    bool ok = cudaGraphLaunch(exec, cs) == cudaSuccess;  // warm-up
    for (int l = 0; l < launches && ok; l++) {
        ok = cudaEventRecord(e0, cs) == cudaSuccess && cudaGraphLaunch(exec, cs) == cudaSuccess &&
             cudaEventRecord(e1, cs) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
        float ms = 0.f;
        if (ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best)
            best = ms;
    }
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    return ok ? best : -1.f;
}
}  // namespace

namespace {
// the autotuner; with `ranked`, also its finalists with their final-stage
// times per evaluation (us), fastest first
int autotune_impl(opf_model *m, const double *d_x, const double *d_lambda, int32_t reps, void *stream,
                  opf_launch *best, double *best_us, std::vector<std::pair<double, opf_launch>> *ranked)
{
    int rc = check_dev(m);
    if (rc)
        return rc;
    if (!d_x || !d_lambda || reps < 1) {
        set_error("autotune needs d_x, d_lambda and reps >= 1");
        return OPF_EINVAL;
    }
    Model &M = *m->M;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the outputs in one allocation, each starting on a 512-byte boundary
    // like separately allocated buffers (their alignment changes the
    // kernels' store transactions, and so the timings being compared)
    auto up = [](int64_t k) { return (size_t)((k + 63) / 64 * 64); };  // doubles, 512-byte multiples
    const size_t o_grad = up(1), o_c = o_grad + up(M.n), o_j = o_c + up(M.m), o_h = o_j + up(M.nnzj);
    double *buf = nullptr;
    const size_t need = sizeof(double) * (o_h + up(M.nnzh));
    if (cudaMalloc(&buf, need) != cudaSuccess) {
        cudaGetLastError();
        set_error("autotune: cudaMalloc of %zu bytes failed", need);
        return OPF_ENOMEM;
    }
    EvalArgs a{d_x, d_lambda, 1.0, buf, buf + o_grad, buf + o_c, buf + o_j, buf + o_h};
    // candidates are timed on a private stream that first waits for the
    // caller's stream (whatever produced d_x and d_lambda)
    cudaStream_t cs = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr, ready = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(ready, s) != cudaSuccess || cudaStreamWaitEvent(cs, ready, 0) != cudaSuccess) {
        set_error("autotune: stream or event setup failed: %s", cudaGetErrorString(cudaGetLastError()));
        rc = OPF_ECUDA;
    }
    const opf_launch saved = M.launch;
    // stage 1: every candidate, one graph of `reps` evaluations, best of 2
    // launches; stage 2 (below): the 8 fastest, interleaved
    std::vector<std::pair<float, opf_launch>> timed;
    const int bblocks[] = {32, 64, 128, 256, 512};
    const int ublocks[] = {32, 64, 128, 256};  // the bus kernel stages at most 8 warps
    const int ctas[] = {0, 2, 4, 8, 16};
    // bus_order 3 (the fused evaluation, where the model allows it) has no
    // branch kernel: its candidates vary the bus block and persistence only
    for (int occ = 0; occ < 3 && !rc; occ++)
    for (int order = 0; order < (M.fuse_ok ? 4 : 3) && !rc; order++)
    for (int bb : bblocks)
        for (int bu : ublocks)
            for (int cb : ctas)
                for (int cu : ctas) {
                    if (rc || (cu != 0 && cu != cb))  // keep the search small: equal persistence
                        continue;
                    if (occ == 1 && bb > 256)
                        continue;
                    if (order == 3 && (occ == 1 || bb != 128))  // occupancy 2: two roles per packed warp
                        continue;
                    M.launch = opf_launch{bb, bu, cb, cu, order, occ};
                    const float ms = time_graph(M, a, reps, 2, cs, e0, e1);
                    if (ms < 0.f) {
                        set_error("autotune: timing a candidate failed: %s", cudaGetErrorString(cudaGetLastError()));
                        rc = OPF_ECUDA;
                    } else {
                        timed.push_back({ms, M.launch});
                    }
                }
    opf_launch bestc = saved;
    float best_ms = 1e30f;
    if (!rc) {
        std::sort(timed.begin(), timed.end(),
                  [](const std::pair<float, opf_launch> &x, const std::pair<float, opf_launch> &y) {
                      return x.first < y.first;
                  });
        // stage 2: the finalists, each captured once, then timed in 6
        // interleaved rounds (the round's first candidate rotating), best
        // launch each: drift of clocks or power between candidates falls on
        // all of them alike, and the top shapes (often within a few percent
        // of each other) are compared under the same conditions. The
        // finalists are the fastest candidate of each structural class (bus
        // order and branch occupancy: different kernels, which a caller
        // with other conditions may rank differently), then the fastest of
        // the rest, 12 in all at most
        {
            auto same = [](const opf_launch &x, const opf_launch &y) {
                return x.branch_block == y.branch_block && x.bus_block == y.bus_block &&
                       x.branch_ctas_per_sm == y.branch_ctas_per_sm && x.bus_ctas_per_sm == y.bus_ctas_per_sm &&
                       x.bus_order == y.bus_order && x.branch_occupancy == y.branch_occupancy;
            };
            std::vector<std::pair<float, opf_launch>> finals;
            bool seen[16] = {};
            for (const auto &c : timed) {
                const int cls = (c.second.bus_order & 3) * 4 + (c.second.branch_occupancy & 3);
                if (!seen[cls]) {
                    seen[cls] = true;
                    finals.push_back(c);
                }
            }
            for (const auto &c : timed) {
                if (finals.size() >= 12)
                    break;
                bool in = false;
                for (const auto &f : finals)
                    in = in || same(f.second, c.second);
                if (!in)
                    finals.push_back(c);
            }
            if (finals.size() > 12)
                finals.resize(12);
            timed.swap(finals);
        }
        const size_t nf = timed.size();
        std::vector<cudaGraph_t> graphs(nf, nullptr);
        std::vector<cudaGraphExec_t> execs(nf, nullptr);
        std::vector<float> fbest(nf, 1e30f);
        for (size_t k = 0; k < nf && !rc; k++) {
            M.launch = timed[k].second;
            if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                rc = OPF_ECUDA;
                break;
            }
            int lrc = OPF_OK;
            for (int r = 0; r < reps && !lrc; r++)
                lrc = launch_eval(M, a, W_OBJ | W_GRAD | W_CONS | W_JAC | W_HESS, cs);
            const cudaError_t ce = cudaStreamEndCapture(cs, &graphs[k]);
            if (lrc || ce != cudaSuccess || cudaGraphInstantiate(&execs[k], graphs[k], 0) != cudaSuccess ||
                cudaGraphLaunch(execs[k], cs) != cudaSuccess)  // warm-up
                rc = OPF_ECUDA;
        }
        for (int round = 0; round < 6 && !rc; round++)
            for (size_t q = 0; q < nf && !rc; q++) {
                const size_t k = (q + (size_t)round) % nf;
                float ms = 0.f;
                if (cudaEventRecord(e0, cs) != cudaSuccess || cudaGraphLaunch(execs[k], cs) != cudaSuccess ||
                    cudaEventRecord(e1, cs) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                    cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                    rc = OPF_ECUDA;
                else if (ms < fbest[k])
                    fbest[k] = ms;
            }
        if (rc)
            set_error("autotune: timing a candidate failed: %s", cudaGetErrorString(cudaGetLastError()));
        for (size_t k = 0; k < nf; k++) {
            if (!rc && fbest[k] < best_ms) {
                best_ms = fbest[k];
                bestc = timed[k].second;
            }
            if (!rc && ranked)
                ranked->push_back({1000.0 * fbest[k] / reps, timed[k].second});
            if (execs[k])
                cudaGraphExecDestroy(execs[k]);
            if (graphs[k])
                cudaGraphDestroy(graphs[k]);
        }
    }
    if (cs) {
        cudaStreamSynchronize(cs);
        cudaStreamDestroy(cs);
    }
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    if (ready)
        cudaEventDestroy(ready);
    cudaFree(buf);
    M.launch = rc ? saved : bestc;
    if (rc)
        return rc;
    if (best)
        *best = bestc;
    if (best_us)
        *best_us = 1000.0 * best_ms / reps;
    if (ranked)
        std::stable_sort(ranked->begin(), ranked->end(),
                         [](const std::pair<double, opf_launch> &x, const std::pair<double, opf_launch> &y) {
                             return x.first < y.first;
                         });
    return OPF_OK;
}
}  // namespace

int opf_autotune(opf_model *m, const double *d_x, const double *d_lambda, int32_t reps, void *stream,
                 opf_launch *best, double *best_us)
{
    return autotune_impl(m, d_x, d_lambda, reps, stream, best, best_us, nullptr);
}

int opf_autotune_list(opf_model *m, const double *d_x, const double *d_lambda, int32_t reps, void *stream,
                      opf_launch *shapes, double *us, int32_t max_shapes, int32_t *n_shapes)
{
    if (!shapes || !us || !n_shapes || max_shapes < 1) {
        set_error("opf_autotune_list needs shapes, us, n_shapes and max_shapes >= 1");
        return OPF_EINVAL;
    }
    std::vector<std::pair<double, opf_launch>> ranked;
    const int rc = autotune_impl(m, d_x, d_lambda, reps, stream, nullptr, nullptr, &ranked);
    if (rc)
        return rc;
    const int32_t k = ranked.size() < (size_t)max_shapes ? (int32_t)ranked.size() : max_shapes;
    for (int32_t q = 0; q < k; q++) {
        shapes[q] = ranked[q].second;
        us[q] = ranked[q].first;
    }
    *n_shapes = k;
    return OPF_OK;
}

}  // extern "C"

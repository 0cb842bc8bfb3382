/*
 * opf.h — C ABI of libopf: GPU evaluation of the AC optimal power flow NLP
 * callbacks (polar or rectangular voltages, branch-flow variables) at a
 * fixed sparsity pattern, for one instance, many periods, or a batch of
 * instances.
 *
 * The problem is the static polar model of the paper's Listing 3 (Sec. III-B),
 * written in the NLP form of Sec. II-A, with the multi-period extension of
 * Sec. III-C-2 (per-period demand, generator ramp limits between consecutive
 * periods, corrective_action_ratio) and batches of independent instances
 * (the batch-solve direction of Sec. V), optionally tied to instance 0 by
 * linking rows on generator output. The callbacks are those of Listing 1
 * (Sec. II-B): obj, grad!, cons!, jac!, hess!(x, lambda; obj_weight).
 *
 * Layout (per instance; instances are concatenated, linking rows last):
 *   x = [va, vm, pg, qg, p, q]; within a group the index is
 *       elem + count * period (the 2-D index rule of Listing 10).
 *       Arc a < nbranch is the from-end of branch a, arc nbranch + k the
 *       to-end of branch k.
 *   g = [ref (1 per period), flow P from-arc, flow Q from-arc, flow P to-arc,
 *        flow Q to-arc, angle difference, P balance, Q balance,
 *        thermal from-arc, thermal to-arc, ramp (ngen x (nperiod-1))],
 *       each group elem + count * period (ramp: g + ngen * (t - 1)).
 *   Flow rows are p_arc - P(v) and q_arc - Q(v) (bounds [0, 0]); thermal rows
 *   p^2 + q^2 - rate_a^2 (bounds [-inf, 0]); balance rows
 *   Pd + gs vm^2 + sum(arc p) - sum(pg) and Qd - bs vm^2 + sum(arc q) - sum(qg).
 *   Rectangular form (opf_batch_opts.form = OPF_FORM_RECT; the paper's
 *   form = :rect of Sec. III-C-1, whose equations it leaves to the
 *   rectangular AC model of PowerModels): x = [vr, vi, pg, qg, p, q] with
 *   -vmax <= vr, vi <= vmax; the same flow functions with V = vr + j vi;
 *   the reference row is vi_ref (bounds [0, 0]); the angle-difference group
 *   holds Im(w) - tan(angmax) Re(w) (bounds [-inf, 0]), w = V_f conj(V_t),
 *   and two groups follow the thermal rows: Im(w) - tan(angmin) Re(w)
 *   (bounds [0, inf]) per branch and vr^2 + vi^2 (bounds [vmin^2, vmax^2])
 *   per bus; balance rows use gs |V|^2 and -bs |V|^2; angle limits must lie
 *   in (-pi/2, pi/2).
 *   Jacobian: values in row-major order of the deduplicated pattern, columns
 *   ascending within a row. Hessian of the Lagrangian
 *   obj_weight * grad^2 f + sum_i lambda_i grad^2 g_i: lower triangle
 *   (row >= col), deduplicated, row-major, columns ascending.
 *   opf_sparsity returns both patterns.
 *
 * Ownership: every opf_network array is a HOST pointer read during the
 * create call only and owned by the caller. The model owns its device copies
 * of the network, layout tables and scratch. Every d_* argument of an eval
 * call is a caller-owned DEVICE buffer of the stated length (doubles); the
 * call is asynchronous on the given stream (NULL = legacy default stream),
 * performs no host<->device transfer and no allocation, and may be captured
 * in a CUDA graph. Evaluations on one model share its scratch: calls on the
 * same model must be ordered on one stream (or otherwise serialised).
 *
 * Errors: every call returns OPF_OK (0) or a positive code and never aborts,
 * exits or traps; opf_last_error() gives a thread-local message. Invalid
 * networks are rejected on the host at create time, before any launch.
 */
#ifndef OPF_H
#define OPF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    OPF_OK = 0,
    OPF_EINVAL = 1,   /* bad size, index out of range, self-loop, r = x = 0, tap < 0,
                         nperiod < 1, NULL where a value is required, bad kind */
    OPF_ENOMEM = 2,   /* device or host allocation failed */
    OPF_ECUDA = 3,    /* a CUDA runtime call or launch failed */
    OPF_ESTATE = 4    /* the model cannot serve this request (e.g. linking rows
                         with unequal generator counts) */
};

enum { OPF_JAC = 0, OPF_HESS = 1 };

/* One network (Listing 3 data; per-unit values, radians, 0-based indices). */
typedef struct {
    int32_t nbus, nbranch, ngen, nload, nperiod; /* nperiod >= 1 */
    int32_t ref_bus;                             /* 0-based reference bus */
    const double *bus_vmin, *bus_vmax;           /* [nbus] */
    const double *bus_gs, *bus_bs;               /* [nbus]; NULL means 0 */
    const int32_t *br_f, *br_t;                  /* [nbranch] endpoints, f != t */
    const double *br_r, *br_x, *br_b;            /* series r, x; total charging b */
    const double *br_tap;                        /* [nbranch]; NULL or 0 means 1 */
    const double *br_shift;                      /* [nbranch]; NULL means 0 */
    const double *br_rate_a, *br_angmin, *br_angmax;
    const int32_t *gen_bus;                      /* [ngen] */
    const double *gen_pmin, *gen_pmax, *gen_qmin, *gen_qmax;
    const double *gen_c2, *gen_c1, *gen_c0;      /* cost c2 pg^2 + c1 pg + c0; c0 NULL = 0 */
    const int32_t *load_bus;                     /* [nload] */
    const double *load_pd, *load_qd;             /* [nperiod][nload], period-major */
    double ramp_ratio;                           /* ramp rows |pg_t - pg_{t-1}| <= ratio pmax
                                                    when > 0 and nperiod > 1 (Listing 6) */
} opf_network;

enum { OPF_FORM_POLAR = 0, OPF_FORM_RECT = 1 };

/* Storage units of one network: the multi-period model with storage of
 * Sec. III-C-2 (the storage model of Geth, Coffrin and Fobes the paper
 * builds on), polar form only. Per unit k and period t the variables
 * ps, qs (power drawn from bus[k], added to its P and Q balance rows),
 * sc in [0, charge_rating], sd in [0, discharge_rating] and
 * se in [0, energy_rating] follow q in x (each group k + nstor * t, in
 * that order; ps in [-thermal_rating, thermal_rating], qs in [qmin, qmax]);
 * the instance's rows gain, after its ramp rows (each group k + nstor * t):
 *   state of charge  se_t - se_{t-1} - dt (eta_c sc_t - sd_t / eta_d) = 0,
 *                    and = e_init in the first period (no se_{t-1} term)
 *   converter losses ps + sd - sc - r (ps^2 + qs^2) / vm_bus^2 = p_loss
 *   thermal          ps^2 + qs^2 <= thermal_rating^2
 *   complementarity  sc sd <= 0, when opf_batch_opts.storage_complementarity
 * Jacobian rows list their columns ascending; the Hessian gains (ps, vm),
 * (ps, ps), (qs, vm), (qs, qs) per unit and period, (sd, sc) with the
 * complementarity rows, and the loss term's part of (vm, vm). */
typedef struct {
    int32_t nstor;
    const int32_t *bus;                                 /* [nstor] */
    const double *energy_rating, *charge_rating, *discharge_rating, *thermal_rating;
    const double *eta_c, *eta_d;                        /* > 0 */
    const double *r, *p_loss, *qmin, *qmax, *e_init;    /* [nstor] */
    double dt;                                          /* hours per period, > 0 */
} opf_storage;

typedef struct {
    double link_ratio; /* > 0: rows pg_s - pg_0 in [-ratio pmax, ratio pmax] for every
                          instance s >= 1 (all instances need equal ngen, nperiod 1) */
    const double *link_ratios; /* NULL, or [ninst] per-instance corrective ratios (entry s
                                  replaces link_ratio for instance s >= 1; entry 0 unused;
                                  every entry finite and >= 0) */
    double reserve;    /* > 0: one reserve row per instance and period,
                          sum_g pg_g <= sum_g pmax_g - reserve * (total Pd of the period),
                          i.e. the spare capacity covers that share of the demand */
    int32_t form;      /* OPF_FORM_POLAR (va, vm) or OPF_FORM_RECT (vr, vi), for every
                          instance; models from opf_model_create are polar */
    const opf_storage *storage;      /* NULL, or [ninst] storage units per instance
                                        (nstor 0 for none); polar form only */
    int32_t storage_complementarity; /* nonzero: the rows sc sd <= 0 */
} opf_batch_opts;

typedef struct opf_model opf_model;

/* Launch shape of the two evaluation kernels (branch phase, bus phase). */
typedef struct {
    int32_t branch_block; /* threads per block, branch kernel (32..512, multiple of 32;
                             at most 256 with branch_occupancy 1) */
    int32_t bus_block;    /* threads per block, bus/generator kernel (32..1024, multiple of
                             32; more than 256 runs as 256) */
    int32_t branch_ctas_per_sm; /* persistent grid = ctas_per_sm * SMs; 0 = one thread per item */
    int32_t bus_ctas_per_sm;
    int32_t bus_order;    /* 0: buses in id order; 1: buses sorted by arc count into warps
                             of 32, warps dealt heaviest and lightest alternately (fewer
                             idle lanes in the slot loops: better for large batches);
                             2: buses with more than 6 arc slots (and at most 32) a warp
                             each, one lane per slot, the others a thread each in id order
                             (shorter longest thread: better for single instances;
                             storage models run 2 as 0); 3: the fused evaluation, one
                             kernel per evaluation and no arc scratch: whole buses
                             packed into warps, one lane per arc slot, each lane
                             evaluating its arc end's rows and second-order parts,
                             summed per bus by segmented warp scans (models
                             without storage whose buses have at most 32 arc
                             slots, either form; other models run 3 as 2; the branch fields are unused, except
                             branch_occupancy 2: two warps per packed warp, one for
                             the rows and Jacobian, one for the Hessian) */
    int32_t branch_occupancy; /* 0: branch kernel compiled for up to 128 registers per
                                 thread (shortest chains); 1: for 80 (three blocks of 256
                                 per SM: more warps to hide latency in large batches);
                                 2: two threads per branch, one per end (shorter chains:
                                 better for single instances; both forms) */
} opf_launch;

/* Create a model for one network (Listing 3; multi-period if nperiod > 1).
 * Validates every index and parameter on the host, precomputes the branch
 * admittances of the pi-model (Yff, Yft, Ytf, Ytt), builds both sparsity
 * patterns and the per-bus layout tables, and copies them to the current
 * CUDA device. *out receives the model, or NULL on error. */
int opf_model_create(const opf_network *net, opf_model **out);

/* Create one model over ninst independent instances of uneven size
 * (scenarios, N-1 contingencies), evaluated by the same kernels in one
 * launch per phase. opts may be NULL (no linking rows). */
int opf_batch_create(const opf_network *nets, int32_t ninst, const opf_batch_opts *opts,
                     opf_model **out);

/* Host-only model over ninst networks (ninst = 1: a single network): the
 * same validation and layout as opf_batch_create, no device memory and no
 * CUDA call. Serves opf_dims, opf_sparsity and opf_bounds (for example a
 * solver's symbolic analysis before a GPU is attached); every eval call on
 * it returns OPF_ESTATE. */
int opf_structure_create(const opf_network *nets, int32_t ninst, const opf_batch_opts *opts,
                         opf_model **out);

int opf_model_destroy(opf_model *model);

/* n variables, m constraints, Jacobian and Hessian (lower) nonzeros of the
 * model of Listing 3 (Sec. III-B): the sizes of the arrays the callbacks of
 * Listing 1 (Sec. II-B) fill. */
int opf_dims(const opf_model *model, int64_t *n, int64_t *m, int64_t *nnz_jac,
             int64_t *nnz_hess);

/* Pattern of kind OPF_JAC or OPF_HESS into HOST arrays of nnz entries each
 * (the structure behind jac! and hess! of Listing 1; the automatic
 * sparsity detection of Sec. II-B, done once here from the model's layout): (row,
 * col) pairs, 0-based, sorted row-major, the Hessian as its lower triangle.
 * The indices are int64 so that batches beyond 2^31 entries need no second
 * call; every value array of the eval calls is in this order. */
int opf_sparsity(const opf_model *model, int32_t kind, int64_t *rows, int64_t *cols);

/* Variable and constraint bounds into HOST arrays (n and m entries);
 * infinite bounds are +-INFINITY. */
int opf_bounds(const opf_model *model, double *xl, double *xu, double *gl, double *gu);

/* Objective (one double, d_obj) and gradient (n) at d_x (n): obj and grad!
 * of Listing 1, the generator cost of Listing 3 summed over generators,
 * periods and instances. Either output may be NULL. The objective is a
 * fixed-order (deterministic) reduction. */
int opf_eval_obj_grad(opf_model *model, const double *d_x, double *d_obj, double *d_grad,
                      void *stream);

/* Constraint values g(x) into d_c (m): cons! of Listing 1, the rows of
 * Listing 3 (reference angle, flow rows, angle difference, P and Q balance
 * with their constraint! augmentations, thermal) and the ramp rows of
 * Listings 6-7 (Sec. III-C-2), in the order and index rule of Listing 10. */
int opf_eval_cons(opf_model *model, const double *d_x, double *d_c, void *stream);

/* Jacobian values (nnz_jac) in pattern order: jac! of Listing 1. */
int opf_eval_jac(opf_model *model, const double *d_x, double *d_jvals, void *stream);

/* Values (nnz_hess, lower triangle, pattern order) of obj_weight * Hessian
 * of f plus sum_i lambda_i * Hessian of g_i at d_x (n), d_lambda (m):
 * hess!(x, l, H; obj_weight) of Listing 1. */
int opf_eval_hess(opf_model *model, const double *d_x, const double *d_lambda,
                  double obj_weight, double *d_hvals, void *stream);

/* Fused Jacobian and Hessian (opf_eval_jac and opf_eval_hess in one pass
 * over the network): the pair a Newton-type solver requests each iteration
 * (Sec. IV, the callbacks inside the paper's solvers). */
int opf_eval_jac_hess(opf_model *model, const double *d_x, const double *d_lambda,
                      double obj_weight, double *d_jvals, double *d_hvals, void *stream);

/* Every callback of Listing 1 (obj, grad!, cons!, jac!, hess!)
 * in one pass; any output may be NULL (skipped). d_lambda may be NULL only
 * if d_hvals is NULL. */
int opf_eval_all(opf_model *model, const double *d_x, const double *d_lambda, double obj_weight,
                 double *d_obj, double *d_grad, double *d_c, double *d_jvals, double *d_hvals,
                 void *stream);

/* The two kernels of one opf_eval_all, selectable: phases = OPF_PHASE_BRANCH
 * (per-branch rows, Jacobian and Hessian parts, and the per-arc scratch),
 * OPF_PHASE_BUS (balance rows, bus Hessian rows assembled from that scratch,
 * generator terms, objective), or both (= opf_eval_all). A bus phase alone
 * reads the scratch of the last branch phase run on this model, which must
 * have had the same outputs selected and the same d_x / d_lambda. For timing
 * and for overlapping the phases of independent models. With the fused
 * evaluation (bus_order 3, where the model allows it) there is one kernel:
 * OPF_PHASE_BUS runs the whole evaluation and OPF_PHASE_BRANCH alone runs
 * nothing. */
enum { OPF_PHASE_BRANCH = 1, OPF_PHASE_BUS = 2 };
int opf_eval_phases(opf_model *model, int32_t phases, const double *d_x, const double *d_lambda,
                    double obj_weight, double *d_obj, double *d_grad, double *d_c,
                    double *d_jvals, double *d_hvals, void *stream);

/* opf_eval_all on HOST buffers: copies h_x (and h_lambda) to device staging
 * buffers owned by the model, evaluates, copies the requested outputs back
 * and synchronises the stream before returning. The staging buffers are
 * allocated on the first call (so this call allocates once per model).
 * Pinned host memory gives asynchronous copies. */
int opf_eval_all_host(opf_model *model, const double *h_x, const double *h_lambda,
                      double obj_weight, double *h_obj, double *h_grad, double *h_c,
                      double *h_jvals, double *h_hvals, void *stream);

/* opf_eval_all for callers that cannot allocate device memory while they
 * run (the paper has no counterpart: this is a deployment variant). Typical
 * callers: a solver embedded in a process whose device memory is owned by
 * another runtime (a fixed arena or a pool that must not grow), or a loop
 * that must keep cudaMalloc / cudaFree, which can synchronise the device,
 * out of its iterations. It evaluates exactly what opf_eval_all evaluates,
 * with the same kernels and outputs, but its scratch (per-arc slots,
 * per-block objective partials, a block counter) lives in one static device
 * array of OPF_NOALLOC_SCRATCH_BYTES bytes that every device loading this
 * library holds until the process exits; the call itself calls no
 * allocator. Limits: models needing more than 174,074 arc slots (2 x
 * branches x periods, summed over instances) are rejected with OPF_EINVAL
 * and a message naming the sizes, unless the model's launch shape is the
 * one-kernel fused evaluation (bus_order 3 where the model allows it),
 * which writes no arc slots and so has no such limit. The current device
 * must be the model's (else OPF_EINVAL). The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress, with that device current)
 * and caches it: make that first call before any stream capture. Every
 * call, on every model, shares the one array and leaves its last contents
 * there; the block counter is cleared at the start of each call. Calls whose
 * executions overlap on the GPU (other streams, or concurrent host threads)
 * race on the array: serialise them. */
#define OPF_NOALLOC_SCRATCH_BYTES (8u << 20)
int opf_eval_all_noalloc(opf_model *model, const double *d_x, const double *d_lambda,
                         double obj_weight, double *d_obj, double *d_grad, double *d_c,
                         double *d_jvals, double *d_hvals, void *stream);

/* Jacobian-transpose product d_out (n) = J(x)^T d_v (d_v has m entries),
 * evaluated term by term like the Hessian (no Jacobian values needed):
 * NLPModels' jtprod!, the companion of Listing 1's jac!. Deterministic. */
int opf_eval_jtprod(opf_model *model, const double *d_x, const double *d_v, double *d_out,
                    void *stream);

/* Sets the p and q entries of d_x (n) to the branch flows at d_x's voltages
 * (the pi-model of Listing 3, in the model's form), so every flow row is
 * zero; the other entries are left as they are. */
int opf_eval_flows(opf_model *model, double *d_x, void *stream);

/* Replaces the model's loads on the device: d_load_pd, d_load_qd hold each
 * instance's [nperiod][nload] values (instances concatenated, in creation
 * order). The demand of each bus and period becomes the sum of its loads in
 * ascending load order, exactly as at creation. Asynchronous on stream;
 * later evaluations on that stream see the new loads. */
int opf_set_loads(opf_model *model, const double *d_load_pd, const double *d_load_qd, void *stream);

/* Flat start (reading of the usual OPF initial point): va = 0, vm = 1
 * clipped into [vmin, vmax] (rectangular form: vr = that magnitude, vi = 0),
 * pg and qg at the midpoint of their bounds, p and q equal to the branch
 * flows at those voltages. Into d_x (n). */
int opf_flat_start(opf_model *model, double *d_x, void *stream);

/* The sine and cosine the evaluation kernels use (table-driven: a table of
 * sin and cos at multiples of 1/256, short Taylor series of the remainder
 * whose small terms are formed in FP32, and the angle-addition formulas;
 * CUDA's sincos for |d| >= 3.140625), applied to n
 * angles d_angle into d_sin, d_cos (device buffers). For checking its
 * accuracy against other implementations. */
int opf_sincos(opf_model *model, const double *d_angle, int64_t n, double *d_sin, double *d_cos,
               void *stream);

/* Launch shape used by the eval calls; the default suits large instances. */
int opf_get_launch(const opf_model *model, opf_launch *cfg);
int opf_set_launch(opf_model *model, const opf_launch *cfg);

/* Autotuner: times each candidate launch shape (block sizes, persistence,
 * bus order, branch occupancy) of the fused opf_eval_all on this model as a
 * CUDA graph of `reps` back-to-back evaluations (the way a solver loop
 * replays them), on a private stream that first waits for `stream`; the
 * finalists (the fastest shape of each class of bus order and branch
 * occupancy, then the fastest others, twelve at most) are then timed again
 * in six interleaved rounds (each captured once, best launch each, so that
 * drift between candidates falls on all of them alike). Keeps the fastest
 * and returns
 * it in *best with its time per eval in *best_us (CUDA events). Allocates
 * temporary output buffers and a stream for the duration of the call, which
 * synchronises with its own work before returning. */
int opf_autotune(opf_model *model, const double *d_x, const double *d_lambda, int32_t reps,
                 void *stream, opf_launch *best, double *best_us);

/* opf_autotune that also returns its finalists: into the HOST arrays
 * shapes[] and us[] (caller-owned, max_shapes >= 1 entries each) the shapes
 * of its final stage, fastest first, with their times per evaluation in us,
 * and their number in *n_shapes (at most max_shapes, at most twelve). For a
 * caller whose conditions differ from the tuner's (the tuner times one
 * buffer set, resident in L2 for small models) and who re-times the few
 * finalists under its own. Sets the model's shape to the fastest, as
 * opf_autotune does. OPF_EINVAL for a null array or max_shapes < 1. */
int opf_autotune_list(opf_model *model, const double *d_x, const double *d_lambda, int32_t reps,
                      void *stream, opf_launch *shapes, double *us, int32_t max_shapes, int32_t *n_shapes);

/* opf_eval_all_host without the final synchronisation, pipelined across
 * calls: inputs are copied in on an internal stream into one of two staging
 * slots, the evaluation runs on a second internal stream and the outputs
 * are copied out on a third, so the copies of one call overlap the
 * evaluation and copies of the next. The call starts at once (the host
 * inputs must be ready; it does not wait for earlier work on `stream`);
 * `stream` (the caller's) is made to wait for the call's outputs: the host
 * outputs are complete, and the inputs may be reused, once `stream` has
 * been synchronised. Host buffers should be page-locked
 * (opf_host_register). Calls on one model must come from one thread and
 * must not overlap evaluations of the same model on other streams;
 * allocates its staging and streams on first use (freed with the model). */
int opf_eval_all_host_async(opf_model *model, const double *h_x, const double *h_lambda,
                            double obj_weight, double *h_obj, double *h_grad, double *h_c,
                            double *h_jvals, double *h_hvals, void *stream);

/* Page-lock caller host memory for this library's host<->device copies
 * (opf_eval_all_host) so they run at full DMA bandwidth; unregister before
 * freeing. Memory page-locked by another CUDA runtime loaded in the same
 * process (for example a framework's pinned allocator) can be copied by
 * this library only at pageable speed, so register it here. Errors:
 * OPF_EINVAL for NULL or zero size, OPF_ECUDA if the runtime refuses. */
int opf_host_register(void *ptr, size_t bytes);
int opf_host_unregister(void *ptr);

/* Thread-local description of the last error on this thread. */
const char *opf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif

/*
 * FP64 CPU oracle for the polar AC-OPF callbacks with branch-flow variables.
 *
 * TEST INFRASTRUCTURE ONLY. This header belongs to the oracle, which exists to
 * judge the CUDA path: only the tests, the smoke check and the benchmark's CPU
 * baseline may load it. It shares no code, header, constant or helper with the
 * library under paper_2510_12897_b300/, and the library never calls it.
 *
 * The problem is the one of the paper's Listing 3 (Sec. III-B), in the NLP
 * form of Sec. II-A, with the multi-period extension of Sec. III-C-2 (demand
 * per period, ramp limits between consecutive periods) and a batch of
 * independent instances (the batch-solve direction of Sec. V), optionally tied
 * to instance 0 by linking rows on generator output.
 *
 * Variable order per instance:  va, vm, pg, qg, p, q, each group indexed
 * elem + count * period (the 2-D index rule of Listing 10).
 * Constraint groups per instance, in Listing 3 order:
 *   ref, flow P (from arc), flow Q (from arc), flow P (to arc), flow Q (to arc),
 *   angle difference, P balance, Q balance, thermal (from), thermal (to),
 *   then ramp rows g + ngen * (t - 1), t = 1..T-1.
 * Instances are concatenated; linking rows come last.
 *
 * Rectangular form (form 1): vr, vi take the places of va, vm; the reference
 * row is vi_ref; the angle group holds Im(w) - tan(angmax) Re(w) <= 0 and two
 * groups follow the thermal rows: Im(w) - tan(angmin) Re(w) >= 0 per branch
 * and vmin^2 <= vr^2 + vi^2 <= vmax^2 per bus (w = V_f conj(V_t)).
 *
 * Storage (polar form): variables ps, qs, sc, sd, se of every unit follow q,
 * each group unit + nstor * period; rows, each group unit + nstor * period,
 * follow the ramp rows:
 *   state of charge  se_t - se_{t-1} - dt (eta_c sc_t - sd_t / eta_d) = 0
 *                    (t = 0: se_0 - dt (...) = e_init)
 *   converter losses ps + sd - sc - r (ps^2 + qs^2) / vm_bus^2 = p_loss
 *   thermal          ps^2 + qs^2 <= thermal_rating^2
 *   complementarity  sc sd <= 0 (only when requested)
 * and ps, qs are drawn from the bus (added to its P and Q balance rows).
 */
#ifndef OPF_ORACLE_H
#define OPF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t nbus, nbranch, ngen, nload, nperiod, ref_bus;
    const double *vmin, *vmax, *gs, *bs;                 /* [nbus] */
    const int32_t *f, *t;                                /* [nbranch] */
    const double *r, *x, *b, *tap, *shift, *rate_a, *angmin, *angmax;
    const int32_t *gen_bus;                              /* [ngen] */
    const double *pmin, *pmax, *qmin, *qmax, *c2, *c1, *c0;
    const int32_t *load_bus;                             /* [nload] */
    const double *pd, *qd;                               /* [nperiod][nload] */
    double ramp_ratio;                                   /* ramp rows if > 0 and nperiod > 1 */
} ora_net;

/* Storage units of one instance (multi-period model with storage): unit k
 * at bus[k]; per period the variables ps, qs (power drawn from the bus),
 * sc, sd (charging, discharging) and se (stored energy); dt hours per period. */
typedef struct {
    int32_t nstor;
    const int32_t *bus;
    const double *energy_rating, *charge_rating, *discharge_rating, *thermal_rating;
    const double *eta_c, *eta_d, *r, *p_loss, *qmin, *qmax, *e_init;
    double dt;
} ora_storage;

typedef struct ora_ctx ora_ctx;

/* Builds layout and sparsity patterns. Copies every array. NULL on bad input. */
ora_ctx *ora_create(const ora_net *nets, int32_t ninst, double link_ratio);
/* As ora_create, with per-instance corrective ratios (NULL: link_ratio for
 * every instance; entry 0 unused) and reserve rows when reserve > 0: per
 * instance and period, sum_g pg_g <= sum_g pmax_g - reserve * (total Pd). */
ora_ctx *ora_create2(const ora_net *nets, int32_t ninst, double link_ratio, const double *link_ratios,
                     double reserve);
/* As ora_create2 in the polar (form 0) or rectangular (form 1) voltages. */
ora_ctx *ora_create3(const ora_net *nets, int32_t ninst, double link_ratio, const double *link_ratios,
                     double reserve, int32_t form);
/* As ora_create3 (polar form only) with storage: stor[s] describes instance
 * s's units (stor NULL: none). Per instance, after its ramp rows: state of
 * charge, converter losses and thermal rows, and the complementarity rows
 * sc sd <= 0 when compl != 0. */
ora_ctx *ora_create4(const ora_net *nets, int32_t ninst, double link_ratio, const double *link_ratios,
                     double reserve, int32_t form, const ora_storage *stor, int32_t compl);
void ora_destroy(ora_ctx *);
const char *ora_error(void);

void ora_dims(const ora_ctx *, int64_t *n, int64_t *m, int64_t *nnzj, int64_t *nnzh);
void ora_jac_pattern(const ora_ctx *, int64_t *rows, int64_t *cols);
void ora_hess_pattern(const ora_ctx *, int64_t *rows, int64_t *cols);
void ora_bounds(const ora_ctx *, double *xl, double *xu, double *gl, double *gu);

/* Each evaluator optionally fills a magnitude scale per output entry: the sum,
 * over all contributions to the entry, of a bound on each contribution's
 * absolute value. Tolerances are stated relative to it. Pass NULL to skip. */
double ora_obj(const ora_ctx *, const double *x);
double ora_obj_scale(const ora_ctx *, const double *x);  /* sum of |terms| of f */
void ora_grad(const ora_ctx *, const double *x, double *g);
void ora_cons(const ora_ctx *, const double *x, double *c, double *scale);
int ora_jac(const ora_ctx *, const double *x, double *vals, double *scale);
int ora_hess(const ora_ctx *, const double *x, const double *lambda, double sigma,
             double *vals, double *scale);

/* Maximum constraint violation of Sec. IV-A (componentwise positive parts)
 * and the maximum variable-bound violation, at x. */
void ora_cvio(const ora_ctx *, const double *x, double *cons_viol, double *var_viol);

#ifdef __cplusplus
}
#endif
#endif

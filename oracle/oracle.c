/*
 * FP64 CPU oracle for the polar AC-OPF callbacks with branch-flow variables.
 *
 * TEST INFRASTRUCTURE ONLY: it judges the CUDA path. Only the tests, the smoke
 * check and the benchmark's CPU baseline may load it; the library never does,
 * and the two share no code.
 *
 * What it computes, and where the paper states it:
 *   - NLP form  min f(x)  s.t.  xl <= x <= xu,  gl <= g(x) <= gu      (Sec. II-A)
 *   - callbacks obj, grad, cons, jac, hess(x, lambda; obj_weight)       (Listing 1)
 *   - the static polar model with branch-flow variables                 (Listing 3)
 *       variables va, vm, pg, qg, p, q and their bounds
 *       objective sum of generator costs (quadratic c2 pg^2 + c1 pg + c0)
 *       ref angle, four branch-flow rows, angle difference, P/Q balance with
 *       the arc and generator augmentations of constraint!, two thermal rows
 *     The flow functions follow the pi-model of the formulation the paper
 *     points to (Sec. III-C-1, "as described in" PowerModels / MATPOWER):
 *       ys = 1/(r + j x), tap tau (0 means 1), shift theta, charging b split
 *       Yff = (ys + j b/2)/tau^2, Yft = -ys/conj(tau e^{j theta}),
 *       Ytf = -ys/(tau e^{j theta}), Ytt = ys + j b/2,
 *       S_fr = V_f conj(Yff V_f + Yft V_t),  S_to = V_t conj(Ytf V_f + Ytt V_t).
 *   - multi-period: per-period demand, ramp rows |pg_t - pg_{t-1}| <= ratio pmax
 *     (Sec. III-C-2, Listing 6, corrective_action_ratio), 2-D layout of Listing 10
 *   - constraint violation Cvio (Sec. IV-A)
 *   - the rectangular form (form = :rect of Sec. III-C-1, whose equations the
 *     paper leaves to the rectangular AC model of PowerModels): variables
 *     vr, vi in the places of va, vm with bounds -vmax <= vr, vi <= vmax; the
 *     same pi-model flows with V = vr + j vi; the reference row vi_ref = 0;
 *     the angle-difference limits as two rows Im(w) - tan(angmax) Re(w) <= 0
 *     (in the angle group's place) and Im(w) - tan(angmin) Re(w) >= 0 (after
 *     the thermal rows), w = V_f conj(V_t), valid for limits inside
 *     (-pi/2, pi/2); a voltage-magnitude row vmin^2 <= vr^2 + vi^2 <= vmax^2
 *     per bus (after those); demand terms gs |V|^2 and -bs |V|^2.
 *   - multi-period with storage (Sec. III-C-2, the storage model of Geth,
 *     Coffrin and Fobes the paper builds on, in polar voltages): per unit and
 *     period ps, qs (power drawn from the bus, added to its balance rows),
 *     sc, sd in [0, rating], se in [0, energy rating]; rows: state of charge
 *     se_t - se_{t-1} - dt (eta_c sc_t - sd_t / eta_d) = 0 (the initial
 *     energy in place of se_{-1}), converter losses
 *     ps + sd - sc - r (ps^2 + qs^2) / vm^2 = p_loss (the loss through a
 *     series resistance r carrying the current |S| / vm), thermal
 *     ps^2 + qs^2 <= rating^2, and, when requested, the complementarity
 *     sc sd <= 0 (with sc, sd >= 0 the inequality form of sc sd = 0).
 *
 * Where the paper is silent this oracle takes these readings: a flow row is
 * the arc variable minus the flow function; the thermal row is
 * p^2 + q^2 - rate_a^2 <= 0; the demand terms are Pd + gs vm^2 and
 * Qd - bs vm^2; arc k is the from-end of branch k and arc nl + k its to-end;
 * the Hessian is the deduplicated lower triangle in (row, col) order.
 *
 * Every value is computed in complex arithmetic on the pi-model; derivatives
 * are derived by hand in complex form (polar: d/dva V = j V, d/dvm V = V/vm;
 * rectangular: d/dvr V = 1, d/dvi V = j). The
 * sparsity pattern is built from the term structure alone, then every term's
 * contribution is added into its entry found by binary search. No blocking,
 * no fusion, one thread.
 */
#include "oracle.h"

#include <complex.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

static __thread char g_err[512];

static void set_err(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

const char *ora_error(void) { return g_err; }

/* row groups; G_ANL and G_VM exist in the rectangular form only */
enum { G_REF, G_FPF, G_FQF, G_FPT, G_FQT, G_ANG, G_PB, G_QB, G_THF, G_THT, G_ANL, G_VM, G_RAMP };

typedef struct {
    ora_net net;     /* pointers into the owned copies below */
    void *own[64];
    int nown;
    int64_t xoff, coff;  /* first variable / first row of this instance */
    int64_t n, m;
    int ramp;
    int rect;            /* rectangular voltages: vr, vi in the places of va, vm */
    int ns, compl;       /* storage units; complementarity rows present */
    ora_storage st;      /* pointers into the owned copies */
    int64_t st_row;      /* first storage row, relative to coff */
    double *Pd, *Qd;     /* per bus and period: [nperiod][nbus] */
} inst_t;

struct ora_ctx {
    int ninst;
    int rect;
    inst_t *in;
    double link_ratio;
    double *link_ratios; /* per instance (entry 0 unused) */
    double reserve;      /* > 0: reserve rows, one per instance and period */
    int link;
    int64_t n, m, link_row, res_row;
    int64_t nnzj, nnzh;
    int64_t *jrow, *jcol, *jkey;
    int64_t *hrow, *hcol, *hkey;
};

/* ---------------------------------------------------------------- layout -- */

static int64_t v_va(const inst_t *s, int64_t i, int64_t t)
{
    return s->xoff + i + (int64_t)s->net.nbus * t;
}
static int64_t v_vm(const inst_t *s, int64_t i, int64_t t)
{
    int64_t nbT = (int64_t)s->net.nbus * s->net.nperiod;
    return s->xoff + nbT + i + (int64_t)s->net.nbus * t;
}
static int64_t v_pg(const inst_t *s, int64_t g, int64_t t)
{
    int64_t nbT = (int64_t)s->net.nbus * s->net.nperiod;
    return s->xoff + 2 * nbT + g + (int64_t)s->net.ngen * t;
}
static int64_t v_qg(const inst_t *s, int64_t g, int64_t t)
{
    int64_t T = s->net.nperiod, nbT = (int64_t)s->net.nbus * T, ngT = (int64_t)s->net.ngen * T;
    return s->xoff + 2 * nbT + ngT + g + (int64_t)s->net.ngen * t;
}
static int64_t v_p(const inst_t *s, int64_t a, int64_t t)
{
    int64_t T = s->net.nperiod, nbT = (int64_t)s->net.nbus * T, ngT = (int64_t)s->net.ngen * T;
    return s->xoff + 2 * nbT + 2 * ngT + a + 2 * (int64_t)s->net.nbranch * t;
}
static int64_t v_q(const inst_t *s, int64_t a, int64_t t)
{
    int64_t T = s->net.nperiod, nbT = (int64_t)s->net.nbus * T, ngT = (int64_t)s->net.ngen * T;
    int64_t naT = 2 * (int64_t)s->net.nbranch * T;
    return s->xoff + 2 * nbT + 2 * ngT + naT + a + 2 * (int64_t)s->net.nbranch * t;
}

/* storage variables of unit k in period t: ps, qs, sc, sd, se after q */
static int64_t v_st(const inst_t *s, int which, int64_t k, int64_t t)
{
    int64_t T = s->net.nperiod;
    int64_t base = T * (2 * (int64_t)s->net.nbus + 2 * (int64_t)s->net.ngen + 4 * (int64_t)s->net.nbranch);
    return s->xoff + base + (int64_t)which * s->ns * T + k + (int64_t)s->ns * t;
}
enum { V_PS, V_QS, V_SC, V_SD, V_SE };
/* storage rows of unit k in period t: state of charge, losses, thermal, complementarity */
enum { R_SOC, R_LOSS, R_STH, R_CMP };
static int64_t row_st(const inst_t *s, int which, int64_t k, int64_t t)
{
    return s->coff + s->st_row + (int64_t)which * s->ns * s->net.nperiod + k + (int64_t)s->ns * t;
}

/* row of element e of group grp in period t (ramp: t = 1..T-1) */
static int64_t row_of(const inst_t *s, int grp, int64_t e, int64_t t)
{
    int64_t T = s->net.nperiod, nl = s->net.nbranch, nb = s->net.nbus;
    int64_t size[12] = {1, nl, nl, nl, nl, nl, nb, nb, nl, nl, s->rect ? nl : 0, s->rect ? nb : 0};
    int64_t base = 0;
    for (int k = 0; k < grp && k < 12; k++)
        base += size[k] * T;
    if (grp == G_RAMP)
        return s->coff + base + e + (int64_t)s->net.ngen * (t - 1);
    return s->coff + base + e + size[grp] * t;
}

/* arc a: a < nbranch is the from-end of branch a, else the to-end of a - nbranch */
static int arc_bus(const inst_t *s, int64_t a)
{
    int64_t nl = s->net.nbranch;
    return a < nl ? s->net.f[a] : s->net.t[a - nl];
}

/* ------------------------------------------------------------ pi-model -- */

/* One end of a branch: S_i = V_i conj(Y_ii V_i + Y_ij V_j), V = vm e^{j va}.
 * Local variable order u = (vm_i, vm_j, va_i, va_j).  First and second
 * derivatives follow from dV/dvm = e^{j va} and dV/dva = j V. The b* fields
 * bound the modulus of each quantity by a sum of moduli of its terms. */
typedef struct {
    cplx S, dS[4], d2S[4][4];
    double bS, bdS[4], bd2S[4][4];
} bend_t;

static void branch_end(double vmi, double vmj, double vai, double vaj, cplx Yii, cplx Yij,
                       bend_t *e)
{
    cplx Ei = cexp(I * vai), Ej = cexp(I * vaj);
    cplx Vi = vmi * Ei, Vj = vmj * Ej;
    cplx Ii = Yii * Vi + Yij * Vj;
    cplx W = Vi * conj(Yij * Vj); /* the cross (transfer) part of S_i */
    double ai = cabs(Yii), aj = cabs(Yij);

    e->S = Vi * conj(Ii);
    e->bS = ai * vmi * vmi + aj * vmi * vmj;

    e->dS[0] = Ei * conj(Ii) + vmi * conj(Yii); /* d/dvm_i */
    e->dS[1] = Vi * conj(Yij * Ej);             /* d/dvm_j */
    e->dS[2] = I * W;                           /* d/dva_i */
    e->dS[3] = -I * W;                          /* d/dva_j */
    e->bdS[0] = ai * vmi + aj * vmj + ai * vmi;
    e->bdS[1] = aj * vmi;
    e->bdS[2] = aj * vmi * vmj;
    e->bdS[3] = aj * vmi * vmj;

    cplx d2[4][4];
    double b2[4][4];
    d2[0][0] = 2.0 * conj(Yii);             b2[0][0] = 2.0 * ai;
    d2[0][1] = Ei * conj(Yij * Ej);         b2[0][1] = aj;
    d2[1][1] = 0.0;                         b2[1][1] = 0.0;
    d2[0][2] = I * Ei * conj(Yij * Vj);     b2[0][2] = aj * vmj;
    d2[0][3] = -I * Ei * conj(Yij * Vj);    b2[0][3] = aj * vmj;
    d2[1][2] = I * Vi * conj(Yij * Ej);     b2[1][2] = aj * vmi;
    d2[1][3] = -I * Vi * conj(Yij * Ej);    b2[1][3] = aj * vmi;
    d2[2][2] = -W;                          b2[2][2] = aj * vmi * vmj;
    d2[2][3] = W;                           b2[2][3] = aj * vmi * vmj;
    d2[3][3] = -W;                          b2[3][3] = aj * vmi * vmj;
    for (int a = 0; a < 4; a++)
        for (int b = a; b < 4; b++) {
            e->d2S[a][b] = e->d2S[b][a] = d2[a][b];
            e->bd2S[a][b] = e->bd2S[b][a] = b2[a][b];
        }
}

/* One end of a branch in rectangular voltages, V = vr + j vi:
 * S_i = V_i conj(Y_ii V_i + Y_ij V_j), local order u = (vr_i, vr_j, vi_i, vi_j),
 * dV/dvr = 1 and dV/dvi = j, so that, with I_i = Y_ii V_i + Y_ij V_j,
 *   dS/dvr_i = conj(I_i) + V_i conj(Y_ii),  dS/dvi_i = j conj(I_i) - j V_i conj(Y_ii),
 *   dS/dvr_j = V_i conj(Y_ij),              dS/dvi_j = -j V_i conj(Y_ij),
 * and the second derivatives are constants: 2 conj(Y_ii) on (vr_i, vr_i) and
 * (vi_i, vi_i), conj(Y_ij) on (vr_i, vr_j) and (vi_i, vi_j), -j conj(Y_ij) on
 * (vr_i, vi_j), j conj(Y_ij) on (vi_i, vr_j), zero elsewhere. */
static void branch_end_rect(double vri, double vrj, double vii, double vij, cplx Yii, cplx Yij,
                            bend_t *e)
{
    cplx Vi = vri + I * vii, Vj = vrj + I * vij;
    cplx Ii = Yii * Vi + Yij * Vj;
    double ai = cabs(Yii), aj = cabs(Yij), mi = cabs(Vi), mj = cabs(Vj);

    e->S = Vi * conj(Ii);
    e->bS = ai * mi * mi + aj * mi * mj;

    e->dS[0] = conj(Ii) + Vi * conj(Yii);
    e->dS[1] = Vi * conj(Yij);
    e->dS[2] = I * conj(Ii) - I * Vi * conj(Yii);
    e->dS[3] = -I * Vi * conj(Yij);
    e->bdS[0] = e->bdS[2] = 2.0 * ai * mi + aj * mj;
    e->bdS[1] = e->bdS[3] = aj * mi;

    for (int a = 0; a < 4; a++)
        for (int b = 0; b < 4; b++) {
            e->d2S[a][b] = 0.0;
            e->bd2S[a][b] = 0.0;
        }
    e->d2S[0][0] = e->d2S[2][2] = 2.0 * conj(Yii);
    e->bd2S[0][0] = e->bd2S[2][2] = 2.0 * ai;
    e->d2S[0][1] = e->d2S[1][0] = conj(Yij);
    e->d2S[2][3] = e->d2S[3][2] = conj(Yij);
    e->d2S[0][3] = e->d2S[3][0] = -I * conj(Yij);
    e->d2S[1][2] = e->d2S[2][1] = I * conj(Yij);
    e->bd2S[0][1] = e->bd2S[1][0] = e->bd2S[2][3] = e->bd2S[3][2] = aj;
    e->bd2S[0][3] = e->bd2S[3][0] = e->bd2S[1][2] = e->bd2S[2][1] = aj;
}

/* the (a, b), a <= b, of a rectangular branch end's local order whose second
 * derivative is structurally nonzero (the others are identically zero) */
static const int RECT_D2[6][2] = {{0, 0}, {2, 2}, {0, 1}, {0, 3}, {1, 2}, {2, 3}};

/* Angle-difference row of the rectangular form, Im((1 - j tau) w) with
 * w = V_f conj(V_t) (= Im w - tau Re w), in the from-end's local order
 * (vr_f, vr_t, vi_f, vi_t): dw = (conj(V_t), V_f, j conj(V_t), -j V_f), and
 * d2w is 1 on (vr_f, vr_t) and (vi_f, vi_t), -j on (vr_f, vi_t), j on
 * (vi_f, vr_t). bnd bounds |value|; dbnd the derivatives' moduli. */
static void angle_rect(double vrf, double vrt, double vif, double vit, double tau, double *val,
                       double d[4], double d2[4][4], double *bnd, double dbnd[4])
{
    cplx Vf = vrf + I * vif, Vt = vrt + I * vit;
    cplx w = Vf * conj(Vt), k = 1.0 - I * tau;
    cplx dw[4] = {conj(Vt), Vf, I * conj(Vt), -I * Vf};
    double ak = cabs(k);
    *val = cimag(k * w);
    *bnd = ak * cabs(w);
    for (int a = 0; a < 4; a++) {
        d[a] = cimag(k * dw[a]);
        dbnd[a] = ak * cabs(dw[a]);
        for (int b = 0; b < 4; b++)
            d2[a][b] = 0.0;
    }
    d2[0][1] = d2[1][0] = cimag(k);
    d2[2][3] = d2[3][2] = cimag(k);
    d2[0][3] = d2[3][0] = cimag(-I * k);
    d2[1][2] = d2[2][1] = cimag(I * k);
}

/* the four admittances of branch k */
static void branch_Y(const ora_net *n, int k, cplx *Yff, cplx *Yft, cplx *Ytf, cplx *Ytt)
{
    cplx ys = 1.0 / (n->r[k] + I * n->x[k]);
    double tau = n->tap[k] == 0.0 ? 1.0 : n->tap[k];
    cplx T = tau * cexp(I * n->shift[k]);
    cplx ych = I * (n->b[k] / 2.0);
    *Yff = (ys + ych) / (tau * tau);
    *Yft = -ys / conj(T);
    *Ytf = -ys / T;
    *Ytt = ys + ych;
}

typedef struct {
    int64_t u[4];      /* global (vm_i, vm_j, va_i, va_j) */
    bend_t e;
    int64_t pvar, qvar; /* the arc's own flow variables */
} end_t;

static void ends_of(const inst_t *s, const double *x, int k, int t, end_t *fr, end_t *to)
{
    const ora_net *n = &s->net;
    int f = n->f[k], b = n->t[k];
    cplx Yff, Yft, Ytf, Ytt;
    branch_Y(n, k, &Yff, &Yft, &Ytf, &Ytt);
    if (s->rect) { /* first block vr, second vi; u = (vr_i, vr_j, vi_i, vi_j) */
        double vrf = x[v_va(s, f, t)], vrt = x[v_va(s, b, t)];
        double vif = x[v_vm(s, f, t)], vit = x[v_vm(s, b, t)];
        branch_end_rect(vrf, vrt, vif, vit, Yff, Yft, &fr->e);
        branch_end_rect(vrt, vrf, vit, vif, Ytt, Ytf, &to->e);
        fr->u[0] = v_va(s, f, t); fr->u[1] = v_va(s, b, t);
        fr->u[2] = v_vm(s, f, t); fr->u[3] = v_vm(s, b, t);
        to->u[0] = v_va(s, b, t); to->u[1] = v_va(s, f, t);
        to->u[2] = v_vm(s, b, t); to->u[3] = v_vm(s, f, t);
    } else {
        double vmf = x[v_vm(s, f, t)], vmt = x[v_vm(s, b, t)];
        double vaf = x[v_va(s, f, t)], vat = x[v_va(s, b, t)];
        branch_end(vmf, vmt, vaf, vat, Yff, Yft, &fr->e);
        branch_end(vmt, vmf, vat, vaf, Ytt, Ytf, &to->e);
        fr->u[0] = v_vm(s, f, t); fr->u[1] = v_vm(s, b, t);
        fr->u[2] = v_va(s, f, t); fr->u[3] = v_va(s, b, t);
        to->u[0] = v_vm(s, b, t); to->u[1] = v_vm(s, f, t);
        to->u[2] = v_va(s, b, t); to->u[3] = v_va(s, f, t);
    }
    fr->pvar = v_p(s, k, t); fr->qvar = v_q(s, k, t);
    to->pvar = v_p(s, n->nbranch + k, t); to->qvar = v_q(s, n->nbranch + k, t);
}

/* ---------------------------------------------------------------- create -- */

static void *own_copy(inst_t *s, const void *src, size_t bytes)
{
    void *p = malloc(bytes ? bytes : 1);
    if (bytes)
        memcpy(p, src, bytes);
    s->own[s->nown++] = p;
    return p;
}

static double *own_fill(inst_t *s, const double *src, int64_t count, double dflt)
{
    double *p = malloc(sizeof(double) * (count ? count : 1));
    for (int64_t i = 0; i < count; i++)
        p[i] = src ? src[i] : dflt;
    s->own[s->nown++] = p;
    return p;
}

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

static int64_t sort_unique(int64_t *k, int64_t cnt)
{
    qsort(k, (size_t)cnt, sizeof(int64_t), cmp_i64);
    int64_t w = 0;
    for (int64_t i = 0; i < cnt; i++)
        if (w == 0 || k[i] != k[w - 1])
            k[w++] = k[i];
    return w;
}

static int64_t find(const int64_t *keys, int64_t nnz, int64_t key)
{
    int64_t lo = 0, hi = nnz - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (keys[mid] == key)
            return mid;
        if (keys[mid] < key)
            lo = mid + 1;
        else
            hi = mid - 1;
    }
    return -1;
}

void ora_destroy(ora_ctx *C)
{
    if (!C)
        return;
    for (int s = 0; s < C->ninst; s++)
        for (int k = 0; k < C->in[s].nown; k++)
            free(C->in[s].own[k]);
    free(C->in);
    free(C->link_ratios);
    free(C->jrow); free(C->jcol); free(C->jkey);
    free(C->hrow); free(C->hcol); free(C->hkey);
    free(C);
}

static int validate(const ora_net *n)
{
    if (n->nbus < 1 || n->nbranch < 0 || n->ngen < 0 || n->nload < 0 || n->nperiod < 1) {
        set_err("bad sizes");
        return -1;
    }
    if (n->ref_bus < 0 || n->ref_bus >= n->nbus) {
        set_err("ref_bus out of range");
        return -1;
    }
    for (int k = 0; k < n->nbranch; k++) {
        if (n->f[k] < 0 || n->f[k] >= n->nbus || n->t[k] < 0 || n->t[k] >= n->nbus ||
            n->f[k] == n->t[k]) {
            set_err("branch %d endpoints invalid", k);
            return -1;
        }
        if (n->r[k] == 0.0 && n->x[k] == 0.0) {
            set_err("branch %d has zero impedance", k);
            return -1;
        }
        if (n->tap && n->tap[k] < 0.0) {
            set_err("branch %d has negative tap", k);
            return -1;
        }
    }
    for (int g = 0; g < n->ngen; g++)
        if (n->gen_bus[g] < 0 || n->gen_bus[g] >= n->nbus) {
            set_err("gen %d bus out of range", g);
            return -1;
        }
    for (int l = 0; l < n->nload; l++)
        if (n->load_bus[l] < 0 || n->load_bus[l] >= n->nbus) {
            set_err("load %d bus out of range", l);
            return -1;
        }
    return 0;
}

static void push(int64_t *keys, int64_t *cnt, int64_t n, int64_t r, int64_t c)
{
    keys[(*cnt)++] = r * n + c;
}

ora_ctx *ora_create(const ora_net *nets, int32_t ninst, double link_ratio)
{
    return ora_create2(nets, ninst, link_ratio, NULL, 0.0);
}

ora_ctx *ora_create2(const ora_net *nets, int32_t ninst, double link_ratio, const double *link_ratios,
                     double reserve)
{
    return ora_create3(nets, ninst, link_ratio, link_ratios, reserve, 0);
}

ora_ctx *ora_create3(const ora_net *nets, int32_t ninst, double link_ratio, const double *link_ratios,
                     double reserve, int32_t form)
{
    return ora_create4(nets, ninst, link_ratio, link_ratios, reserve, form, NULL, 0);
}

static int validate_storage(const ora_storage *st, int nbus)
{
    for (int k = 0; k < st->nstor; k++) {
        if (st->bus[k] < 0 || st->bus[k] >= nbus) {
            set_err("storage %d bus out of range", k);
            return -1;
        }
        if (!(st->eta_c[k] > 0.0) || !(st->eta_d[k] > 0.0) || !(st->energy_rating[k] >= 0.0) ||
            !(st->charge_rating[k] >= 0.0) || !(st->discharge_rating[k] >= 0.0) ||
            !(st->thermal_rating[k] >= 0.0) || !(st->r[k] >= 0.0)) {
            set_err("storage %d: efficiencies must be > 0 and ratings, r >= 0", k);
            return -1;
        }
    }
    if (!(st->dt > 0.0)) {
        set_err("storage dt must be > 0");
        return -1;
    }
    return 0;
}

ora_ctx *ora_create4(const ora_net *nets, int32_t ninst, double link_ratio, const double *link_ratios,
                     double reserve, int32_t form, const ora_storage *stor, int32_t compl)
{
    if (stor && form != 0) {
        set_err("storage needs the polar form");
        return NULL;
    }
    if (stor)
        for (int s = 0; s < ninst; s++)
            if (validate_storage(&stor[s], nets[s].nbus))
                return NULL;
    if (form != 0 && form != 1) {
        set_err("form must be 0 (polar) or 1 (rectangular)");
        return NULL;
    }
    if (ninst < 1) {
        set_err("ninst < 1");
        return NULL;
    }
    if (!(link_ratio >= 0.0) || !(reserve >= 0.0)) {
        set_err("link_ratio and reserve must be >= 0");
        return NULL;
    }
    for (int s = 0; s < ninst; s++)
        if (validate(&nets[s]))
            return NULL;
    if (form == 1) /* the tangent form of the angle rows needs |limit| < pi/2 */
        for (int s = 0; s < ninst; s++)
            for (int k = 0; k < nets[s].nbranch; k++)
                if (!(fabs(nets[s].angmin[k]) < M_PI / 2) || !(fabs(nets[s].angmax[k]) < M_PI / 2)) {
                    set_err("rectangular form: branch %d angle limits outside (-pi/2, pi/2)", k);
                    return NULL;
                }
    ora_ctx *C = calloc(1, sizeof *C);
    C->ninst = ninst;
    C->rect = form == 1;
    C->in = calloc((size_t)ninst, sizeof(inst_t));
    C->link_ratio = link_ratio;
    C->link_ratios = malloc(sizeof(double) * (size_t)ninst);
    for (int s = 0; s < ninst; s++)
        C->link_ratios[s] = link_ratios ? link_ratios[s] : link_ratio;
    C->reserve = reserve;
    C->link = (link_ratio > 0.0 || link_ratios) && ninst > 1;
    if (C->link)
        for (int s = 0; s < ninst; s++)
            if (nets[s].ngen != nets[0].ngen || nets[s].nperiod != 1) {
                set_err("linking rows need equal ngen and one period");
                ora_destroy(C);
                return NULL;
            }
    int64_t xo = 0, co = 0;
    for (int s = 0; s < ninst; s++) {
        inst_t *S = &C->in[s];
        const ora_net *n = &nets[s];
        ora_net *d = &S->net;
        *d = *n;
        int64_t nb = n->nbus, nl = n->nbranch, ng = n->ngen, nlo = n->nload, T = n->nperiod;
        d->vmin = own_copy(S, n->vmin, sizeof(double) * nb);
        d->vmax = own_copy(S, n->vmax, sizeof(double) * nb);
        d->gs = own_fill(S, n->gs, nb, 0.0);
        d->bs = own_fill(S, n->bs, nb, 0.0);
        d->f = own_copy(S, n->f, sizeof(int32_t) * nl);
        d->t = own_copy(S, n->t, sizeof(int32_t) * nl);
        d->r = own_copy(S, n->r, sizeof(double) * nl);
        d->x = own_copy(S, n->x, sizeof(double) * nl);
        d->b = own_copy(S, n->b, sizeof(double) * nl);
        d->tap = own_fill(S, n->tap, nl, 1.0);
        d->shift = own_fill(S, n->shift, nl, 0.0);
        d->rate_a = own_copy(S, n->rate_a, sizeof(double) * nl);
        d->angmin = own_copy(S, n->angmin, sizeof(double) * nl);
        d->angmax = own_copy(S, n->angmax, sizeof(double) * nl);
        d->gen_bus = own_copy(S, n->gen_bus, sizeof(int32_t) * ng);
        d->pmin = own_copy(S, n->pmin, sizeof(double) * ng);
        d->pmax = own_copy(S, n->pmax, sizeof(double) * ng);
        d->qmin = own_copy(S, n->qmin, sizeof(double) * ng);
        d->qmax = own_copy(S, n->qmax, sizeof(double) * ng);
        d->c2 = own_copy(S, n->c2, sizeof(double) * ng);
        d->c1 = own_copy(S, n->c1, sizeof(double) * ng);
        d->c0 = own_fill(S, n->c0, ng, 0.0);
        d->load_bus = own_copy(S, n->load_bus, sizeof(int32_t) * nlo);
        d->pd = own_copy(S, n->pd, sizeof(double) * nlo * T);
        d->qd = own_copy(S, n->qd, sizeof(double) * nlo * T);
        /* demand per bus and period: sum of the loads at the bus */
        S->Pd = own_fill(S, NULL, nb * T, 0.0);
        S->Qd = own_fill(S, NULL, nb * T, 0.0);
        for (int64_t t = 0; t < T; t++)
            for (int64_t l = 0; l < nlo; l++) {
                S->Pd[t * nb + d->load_bus[l]] += d->pd[t * nlo + l];
                S->Qd[t * nb + d->load_bus[l]] += d->qd[t * nlo + l];
            }
        S->ramp = T > 1 && n->ramp_ratio > 0.0;
        S->rect = C->rect;
        S->n = T * (2 * nb + 2 * ng + 4 * nl);
        S->m = T * (1 + 7 * nl + 2 * nb) + (S->ramp ? ng * (T - 1) : 0);
        if (S->rect) /* the lower angle rows and the voltage-magnitude rows */
            S->m += T * (nl + nb);
        S->ns = stor ? stor[s].nstor : 0;
        S->compl = compl != 0 && S->ns > 0;
        if (S->ns) {
            const ora_storage *a = &stor[s];
            ora_storage *b = &S->st;
            int64_t k = S->ns;
            *b = *a;
            b->bus = own_copy(S, a->bus, sizeof(int32_t) * k);
            b->energy_rating = own_copy(S, a->energy_rating, sizeof(double) * k);
            b->charge_rating = own_copy(S, a->charge_rating, sizeof(double) * k);
            b->discharge_rating = own_copy(S, a->discharge_rating, sizeof(double) * k);
            b->thermal_rating = own_copy(S, a->thermal_rating, sizeof(double) * k);
            b->eta_c = own_copy(S, a->eta_c, sizeof(double) * k);
            b->eta_d = own_copy(S, a->eta_d, sizeof(double) * k);
            b->r = own_copy(S, a->r, sizeof(double) * k);
            b->p_loss = own_copy(S, a->p_loss, sizeof(double) * k);
            b->qmin = own_copy(S, a->qmin, sizeof(double) * k);
            b->qmax = own_copy(S, a->qmax, sizeof(double) * k);
            b->e_init = own_copy(S, a->e_init, sizeof(double) * k);
            S->st_row = S->m;
            S->n += 5 * k * T;
            S->m += (3 + S->compl) * k * T;
        }
        S->xoff = xo;
        S->coff = co;
        xo += S->n;
        co += S->m;
    }
    C->n = xo;
    C->link_row = co;
    C->res_row = co + (C->link ? (int64_t)nets[0].ngen * (ninst - 1) : 0);
    C->m = C->res_row;
    if (C->reserve > 0.0)
        for (int s = 0; s < ninst; s++)
            C->m += nets[s].nperiod;

    /* ---- Jacobian pattern: one (row, col) per variable a term depends on */
    int64_t cap = 0;
    for (int s = 0; s < ninst; s++) {
        const ora_net *n = &C->in[s].net;
        int64_t T = n->nperiod;
        cap += T * (1 + 40 * (int64_t)n->nbranch + 6 * (int64_t)n->nbus + 2 * (int64_t)n->ngen) +
               2 * (int64_t)n->ngen * T + 16 * (int64_t)C->in[s].ns * T;
    }
    cap += C->link ? 2 * (int64_t)nets[0].ngen * ninst : 0;
    if (C->reserve > 0.0)
        for (int s = 0; s < ninst; s++)
            cap += (int64_t)nets[s].nperiod * nets[s].ngen;
    int64_t *keys = malloc(sizeof(int64_t) * (cap + 1));
    int64_t cnt = 0, N = C->n;
    for (int s = 0; s < ninst; s++) {
        const inst_t *S = &C->in[s];
        const ora_net *n = &S->net;
        int64_t nl = n->nbranch;
        for (int t = 0; t < n->nperiod; t++) {
            /* polar: va_ref; rectangular: vi_ref */
            push(keys, &cnt, N, row_of(S, G_REF, 0, t),
                 S->rect ? v_vm(S, n->ref_bus, t) : v_va(S, n->ref_bus, t));
            for (int k = 0; k < nl; k++) {
                int f = n->f[k], b = n->t[k];
                int64_t dep[4] = {v_vm(S, f, t), v_vm(S, b, t), v_va(S, f, t), v_va(S, b, t)};
                int64_t own[4] = {v_p(S, k, t), v_q(S, k, t), v_p(S, nl + k, t), v_q(S, nl + k, t)};
                int grp[4] = {G_FPF, G_FQF, G_FPT, G_FQT};
                for (int r = 0; r < 4; r++) {
                    int64_t row = row_of(S, grp[r], k, t);
                    push(keys, &cnt, N, row, own[r]);
                    for (int d = 0; d < 4; d++)
                        push(keys, &cnt, N, row, dep[d]);
                }
                if (S->rect) /* both angle rows depend on all four voltages */
                    for (int d = 0; d < 4; d++) {
                        push(keys, &cnt, N, row_of(S, G_ANG, k, t), dep[d]);
                        push(keys, &cnt, N, row_of(S, G_ANL, k, t), dep[d]);
                    }
                else {
                    push(keys, &cnt, N, row_of(S, G_ANG, k, t), v_va(S, f, t));
                    push(keys, &cnt, N, row_of(S, G_ANG, k, t), v_va(S, b, t));
                }
                push(keys, &cnt, N, row_of(S, G_THF, k, t), v_p(S, k, t));
                push(keys, &cnt, N, row_of(S, G_THF, k, t), v_q(S, k, t));
                push(keys, &cnt, N, row_of(S, G_THT, k, t), v_p(S, nl + k, t));
                push(keys, &cnt, N, row_of(S, G_THT, k, t), v_q(S, nl + k, t));
            }
            for (int i = 0; i < n->nbus; i++) {
                push(keys, &cnt, N, row_of(S, G_PB, i, t), v_vm(S, i, t));
                push(keys, &cnt, N, row_of(S, G_QB, i, t), v_vm(S, i, t));
                if (S->rect) { /* |V|^2 depends on vr too; the magnitude row */
                    push(keys, &cnt, N, row_of(S, G_PB, i, t), v_va(S, i, t));
                    push(keys, &cnt, N, row_of(S, G_QB, i, t), v_va(S, i, t));
                    push(keys, &cnt, N, row_of(S, G_VM, i, t), v_va(S, i, t));
                    push(keys, &cnt, N, row_of(S, G_VM, i, t), v_vm(S, i, t));
                }
            }
            for (int64_t a = 0; a < 2 * nl; a++) {
                int i = arc_bus(S, a);
                push(keys, &cnt, N, row_of(S, G_PB, i, t), v_p(S, a, t));
                push(keys, &cnt, N, row_of(S, G_QB, i, t), v_q(S, a, t));
            }
            for (int g = 0; g < n->ngen; g++) {
                int i = n->gen_bus[g];
                push(keys, &cnt, N, row_of(S, G_PB, i, t), v_pg(S, g, t));
                push(keys, &cnt, N, row_of(S, G_QB, i, t), v_qg(S, g, t));
            }
            if (S->ramp && t >= 1)
                for (int g = 0; g < n->ngen; g++) {
                    push(keys, &cnt, N, row_of(S, G_RAMP, g, t), v_pg(S, g, t));
                    push(keys, &cnt, N, row_of(S, G_RAMP, g, t), v_pg(S, g, t - 1));
                }
            for (int k = 0; k < S->ns; k++) { /* storage: balance terms and rows */
                int b = S->st.bus[k];
                push(keys, &cnt, N, row_of(S, G_PB, b, t), v_st(S, V_PS, k, t));
                push(keys, &cnt, N, row_of(S, G_QB, b, t), v_st(S, V_QS, k, t));
                int64_t r = row_st(S, R_SOC, k, t);
                push(keys, &cnt, N, r, v_st(S, V_SC, k, t));
                push(keys, &cnt, N, r, v_st(S, V_SD, k, t));
                push(keys, &cnt, N, r, v_st(S, V_SE, k, t));
                if (t >= 1)
                    push(keys, &cnt, N, r, v_st(S, V_SE, k, t - 1));
                r = row_st(S, R_LOSS, k, t);
                push(keys, &cnt, N, r, v_vm(S, b, t));
                for (int w = V_PS; w <= V_SD; w++)
                    push(keys, &cnt, N, r, v_st(S, w, k, t));
                push(keys, &cnt, N, row_st(S, R_STH, k, t), v_st(S, V_PS, k, t));
                push(keys, &cnt, N, row_st(S, R_STH, k, t), v_st(S, V_QS, k, t));
                if (S->compl) {
                    push(keys, &cnt, N, row_st(S, R_CMP, k, t), v_st(S, V_SC, k, t));
                    push(keys, &cnt, N, row_st(S, R_CMP, k, t), v_st(S, V_SD, k, t));
                }
            }
        }
    }
    if (C->link)
        for (int s = 1; s < ninst; s++)
            for (int g = 0; g < nets[0].ngen; g++) {
                int64_t row = C->link_row + g + (int64_t)nets[0].ngen * (s - 1);
                push(keys, &cnt, N, row, v_pg(&C->in[s], g, 0));
                push(keys, &cnt, N, row, v_pg(&C->in[0], g, 0));
            }
    if (C->reserve > 0.0) {
        int64_t row = C->res_row;
        for (int s = 0; s < ninst; s++)
            for (int t = 0; t < nets[s].nperiod; t++, row++)
                for (int g = 0; g < nets[s].ngen; g++)
                    push(keys, &cnt, N, row, v_pg(&C->in[s], g, t));
    }
    C->nnzj = sort_unique(keys, cnt);
    C->jkey = keys;
    C->jrow = malloc(sizeof(int64_t) * (C->nnzj + 1));
    C->jcol = malloc(sizeof(int64_t) * (C->nnzj + 1));
    for (int64_t e = 0; e < C->nnzj; e++) {
        C->jrow[e] = keys[e] / N;
        C->jcol[e] = keys[e] % N;
    }

    /* ---- Hessian pattern: lower triangle of every term's second-order
     * structure (row >= col), deduplicated */
    cap = 0;
    for (int s = 0; s < ninst; s++) {
        const ora_net *n = &C->in[s].net;
        /* per branch: 10 (polar) or 12 (rectangular, 6 per end) voltage pairs
         * and 4 thermal diagonals; 2 per bus; 1 per generator */
        cap += (int64_t)n->nperiod * (12 * (int64_t)n->nbranch + 2 * (int64_t)n->nbus + n->ngen +
                                      4 * (int64_t)n->nbranch + 6 * (int64_t)C->in[s].ns);
    }
    keys = malloc(sizeof(int64_t) * (cap + 1));
    cnt = 0;
    for (int s = 0; s < ninst; s++) {
        const inst_t *S = &C->in[s];
        const ora_net *n = &S->net;
        int64_t nl = n->nbranch;
        for (int t = 0; t < n->nperiod; t++) {
            for (int k = 0; k < nl; k++) {
                if (S->rect) { /* each end's structurally nonzero second derivatives;
                                  the angle rows' are a subset of the from-end's */
                    int f = n->f[k], b = n->t[k];
                    int64_t ue[2][4] = {{v_va(S, f, t), v_va(S, b, t), v_vm(S, f, t), v_vm(S, b, t)},
                                        {v_va(S, b, t), v_va(S, f, t), v_vm(S, b, t), v_vm(S, f, t)}};
                    for (int side = 0; side < 2; side++)
                        for (int q = 0; q < 6; q++) {
                            int64_t ua = ue[side][RECT_D2[q][0]], ub = ue[side][RECT_D2[q][1]];
                            push(keys, &cnt, N, ua > ub ? ua : ub, ua > ub ? ub : ua);
                        }
                    continue;
                }
                int64_t u[4] = {v_vm(S, n->f[k], t), v_vm(S, n->t[k], t), v_va(S, n->f[k], t),
                                v_va(S, n->t[k], t)};
                for (int a = 0; a < 4; a++)
                    for (int b = a; b < 4; b++) {
                        int64_t r = u[a] > u[b] ? u[a] : u[b], c = u[a] > u[b] ? u[b] : u[a];
                        push(keys, &cnt, N, r, c);
                    }
            }
            for (int i = 0; i < n->nbus; i++) { /* demand terms: quadratic in vm_i (|V_i|) */
                push(keys, &cnt, N, v_vm(S, i, t), v_vm(S, i, t));
                if (S->rect)
                    push(keys, &cnt, N, v_va(S, i, t), v_va(S, i, t));
            }
            for (int g = 0; g < n->ngen; g++) /* cost term */
                push(keys, &cnt, N, v_pg(S, g, t), v_pg(S, g, t));
            for (int64_t a = 0; a < 2 * nl; a++) { /* thermal terms */
                push(keys, &cnt, N, v_p(S, a, t), v_p(S, a, t));
                push(keys, &cnt, N, v_q(S, a, t), v_q(S, a, t));
            }
            for (int k = 0; k < S->ns; k++) { /* storage losses (ps, qs, vm), thermal, complementarity */
                int64_t vm = v_vm(S, S->st.bus[k], t);
                int64_t ps = v_st(S, V_PS, k, t), qs = v_st(S, V_QS, k, t);
                push(keys, &cnt, N, ps, vm);
                push(keys, &cnt, N, ps, ps);
                push(keys, &cnt, N, qs, vm);
                push(keys, &cnt, N, qs, qs);
                push(keys, &cnt, N, vm, vm);
                if (S->compl)
                    push(keys, &cnt, N, v_st(S, V_SD, k, t), v_st(S, V_SC, k, t));
            }
        }
    }
    C->nnzh = sort_unique(keys, cnt);
    C->hkey = keys;
    C->hrow = malloc(sizeof(int64_t) * (C->nnzh + 1));
    C->hcol = malloc(sizeof(int64_t) * (C->nnzh + 1));
    for (int64_t e = 0; e < C->nnzh; e++) {
        C->hrow[e] = keys[e] / N;
        C->hcol[e] = keys[e] % N;
    }
    return C;
}

void ora_dims(const ora_ctx *C, int64_t *n, int64_t *m, int64_t *nnzj, int64_t *nnzh)
{
    *n = C->n;
    *m = C->m;
    *nnzj = C->nnzj;
    *nnzh = C->nnzh;
}

void ora_jac_pattern(const ora_ctx *C, int64_t *rows, int64_t *cols)
{
    memcpy(rows, C->jrow, sizeof(int64_t) * C->nnzj);
    memcpy(cols, C->jcol, sizeof(int64_t) * C->nnzj);
}

void ora_hess_pattern(const ora_ctx *C, int64_t *rows, int64_t *cols)
{
    memcpy(rows, C->hrow, sizeof(int64_t) * C->nnzh);
    memcpy(cols, C->hcol, sizeof(int64_t) * C->nnzh);
}

void ora_bounds(const ora_ctx *C, double *xl, double *xu, double *gl, double *gu)
{
    for (int s = 0; s < C->ninst; s++) {
        const inst_t *S = &C->in[s];
        const ora_net *n = &S->net;
        int64_t nl = n->nbranch;
        for (int t = 0; t < n->nperiod; t++) {
            for (int i = 0; i < n->nbus; i++) {
                if (S->rect) {
                    xl[v_va(S, i, t)] = xl[v_vm(S, i, t)] = -n->vmax[i];
                    xu[v_va(S, i, t)] = xu[v_vm(S, i, t)] = n->vmax[i];
                    gl[row_of(S, G_VM, i, t)] = n->vmin[i] * n->vmin[i];
                    gu[row_of(S, G_VM, i, t)] = n->vmax[i] * n->vmax[i];
                    continue;
                }
                xl[v_va(S, i, t)] = -INFINITY;
                xu[v_va(S, i, t)] = INFINITY;
                xl[v_vm(S, i, t)] = n->vmin[i];
                xu[v_vm(S, i, t)] = n->vmax[i];
            }
            for (int g = 0; g < n->ngen; g++) {
                xl[v_pg(S, g, t)] = n->pmin[g];
                xu[v_pg(S, g, t)] = n->pmax[g];
                xl[v_qg(S, g, t)] = n->qmin[g];
                xu[v_qg(S, g, t)] = n->qmax[g];
            }
            for (int64_t a = 0; a < 2 * nl; a++) {
                double rate = n->rate_a[a % nl];
                xl[v_p(S, a, t)] = -rate;
                xu[v_p(S, a, t)] = rate;
                xl[v_q(S, a, t)] = -rate;
                xu[v_q(S, a, t)] = rate;
            }
            gl[row_of(S, G_REF, 0, t)] = gu[row_of(S, G_REF, 0, t)] = 0.0;
            for (int k = 0; k < nl; k++) {
                int grp[4] = {G_FPF, G_FQF, G_FPT, G_FQT};
                for (int r = 0; r < 4; r++)
                    gl[row_of(S, grp[r], k, t)] = gu[row_of(S, grp[r], k, t)] = 0.0;
                if (S->rect) {
                    gl[row_of(S, G_ANG, k, t)] = -INFINITY;
                    gu[row_of(S, G_ANG, k, t)] = 0.0;
                    gl[row_of(S, G_ANL, k, t)] = 0.0;
                    gu[row_of(S, G_ANL, k, t)] = INFINITY;
                } else {
                    gl[row_of(S, G_ANG, k, t)] = n->angmin[k];
                    gu[row_of(S, G_ANG, k, t)] = n->angmax[k];
                }
                gl[row_of(S, G_THF, k, t)] = -INFINITY;
                gu[row_of(S, G_THF, k, t)] = 0.0;
                gl[row_of(S, G_THT, k, t)] = -INFINITY;
                gu[row_of(S, G_THT, k, t)] = 0.0;
            }
            for (int i = 0; i < n->nbus; i++) {
                gl[row_of(S, G_PB, i, t)] = gu[row_of(S, G_PB, i, t)] = 0.0;
                gl[row_of(S, G_QB, i, t)] = gu[row_of(S, G_QB, i, t)] = 0.0;
            }
            if (S->ramp && t >= 1)
                for (int g = 0; g < n->ngen; g++) {
                    double d = n->ramp_ratio * n->pmax[g];
                    gl[row_of(S, G_RAMP, g, t)] = -d;
                    gu[row_of(S, G_RAMP, g, t)] = d;
                }
            for (int k = 0; k < S->ns; k++) {
                const ora_storage *st = &S->st;
                double S2 = st->thermal_rating[k];
                xl[v_st(S, V_PS, k, t)] = -S2;
                xu[v_st(S, V_PS, k, t)] = S2;
                xl[v_st(S, V_QS, k, t)] = st->qmin[k];
                xu[v_st(S, V_QS, k, t)] = st->qmax[k];
                xl[v_st(S, V_SC, k, t)] = 0.0;
                xu[v_st(S, V_SC, k, t)] = st->charge_rating[k];
                xl[v_st(S, V_SD, k, t)] = 0.0;
                xu[v_st(S, V_SD, k, t)] = st->discharge_rating[k];
                xl[v_st(S, V_SE, k, t)] = 0.0;
                xu[v_st(S, V_SE, k, t)] = st->energy_rating[k];
                gl[row_st(S, R_SOC, k, t)] = gu[row_st(S, R_SOC, k, t)] = t == 0 ? st->e_init[k] : 0.0;
                gl[row_st(S, R_LOSS, k, t)] = gu[row_st(S, R_LOSS, k, t)] = st->p_loss[k];
                gl[row_st(S, R_STH, k, t)] = -INFINITY;
                gu[row_st(S, R_STH, k, t)] = S2 * S2;
                if (S->compl) {
                    gl[row_st(S, R_CMP, k, t)] = -INFINITY;
                    gu[row_st(S, R_CMP, k, t)] = 0.0;
                }
            }
        }
    }
    if (C->link) {
        const ora_net *n0 = &C->in[0].net;
        for (int s = 1; s < C->ninst; s++)
            for (int g = 0; g < n0->ngen; g++) {
                int64_t row = C->link_row + g + (int64_t)n0->ngen * (s - 1);
                gl[row] = -C->link_ratios[s] * n0->pmax[g];
                gu[row] = C->link_ratios[s] * n0->pmax[g];
            }
    }
    if (C->reserve > 0.0) {
        int64_t row = C->res_row;
        for (int s = 0; s < C->ninst; s++) {
            const ora_net *n = &C->in[s].net;
            double cap = 0.0;
            for (int g = 0; g < n->ngen; g++)
                cap += n->pmax[g];
            for (int t = 0; t < n->nperiod; t++, row++) {
                double pd = 0.0;
                for (int l = 0; l < n->nload; l++)
                    pd += n->pd[(int64_t)t * n->nload + l];
                gl[row] = -INFINITY;
                gu[row] = cap - C->reserve * pd;
            }
        }
    }
}

/* ------------------------------------------------------------- objective -- */

double ora_obj(const ora_ctx *C, const double *x)
{
    double f = 0.0;
    for (int s = 0; s < C->ninst; s++) {
        const inst_t *S = &C->in[s];
        const ora_net *n = &S->net;
        for (int t = 0; t < n->nperiod; t++)
            for (int g = 0; g < n->ngen; g++) {
                double pg = x[v_pg(S, g, t)];
                f += n->c2[g] * pg * pg + n->c1[g] * pg + n->c0[g];
            }
    }
    return f;
}

/* Contribution scale of the objective: the sum of the magnitudes of its
 * terms, |c2 pg^2| + |c1 pg| + |c0| over generators and periods (the scale
 * against which a differently ordered sum of the same terms is judged). */
double ora_obj_scale(const ora_ctx *C, const double *x)
{
    double s_f = 0.0;
    for (int s = 0; s < C->ninst; s++) {
        const inst_t *S = &C->in[s];
        const ora_net *n = &S->net;
        for (int t = 0; t < n->nperiod; t++)
            for (int g = 0; g < n->ngen; g++) {
                double pg = x[v_pg(S, g, t)];
                s_f += fabs(n->c2[g] * pg * pg) + fabs(n->c1[g] * pg) + fabs(n->c0[g]);
            }
    }
    return s_f;
}

void ora_grad(const ora_ctx *C, const double *x, double *grad)
{
    memset(grad, 0, sizeof(double) * C->n);
    for (int s = 0; s < C->ninst; s++) {
        const inst_t *S = &C->in[s];
        const ora_net *n = &S->net;
        for (int t = 0; t < n->nperiod; t++)
            for (int g = 0; g < n->ngen; g++)
                grad[v_pg(S, g, t)] = 2.0 * n->c2[g] * x[v_pg(S, g, t)] + n->c1[g];
    }
}

/* ----------------------------------------------------------- constraints -- */

void ora_cons(const ora_ctx *C, const double *x, double *c, double *scale)
{
    memset(c, 0, sizeof(double) * C->m);
    if (scale)
        memset(scale, 0, sizeof(double) * C->m);
#define ADD(row, v, bnd)                \
    do {                                \
        c[row] += (v);                  \
        if (scale)                      \
            scale[row] += (bnd);        \
    } while (0)
    for (int s = 0; s < C->ninst; s++) {
        const inst_t *S = &C->in[s];
        const ora_net *n = &S->net;
        int64_t nl = n->nbranch, nb = n->nbus;
        for (int t = 0; t < n->nperiod; t++) {
            /* polar: va_ref; rectangular: vi_ref */
            double ref = x[S->rect ? v_vm(S, n->ref_bus, t) : v_va(S, n->ref_bus, t)];
            ADD(row_of(S, G_REF, 0, t), ref, fabs(ref));
            for (int k = 0; k < nl; k++) {
                end_t fr, to;
                ends_of(S, x, k, t, &fr, &to);
                double pf = x[fr.pvar], qf = x[fr.qvar], pt = x[to.pvar], qt = x[to.qvar];
                ADD(row_of(S, G_FPF, k, t), pf - creal(fr.e.S), fabs(pf) + fr.e.bS);
                ADD(row_of(S, G_FQF, k, t), qf - cimag(fr.e.S), fabs(qf) + fr.e.bS);
                ADD(row_of(S, G_FPT, k, t), pt - creal(to.e.S), fabs(pt) + to.e.bS);
                ADD(row_of(S, G_FQT, k, t), qt - cimag(to.e.S), fabs(qt) + to.e.bS);
                double vaf = x[v_va(S, n->f[k], t)], vat = x[v_va(S, n->t[k], t)];
                if (S->rect) {
                    double vif = x[v_vm(S, n->f[k], t)], vit = x[v_vm(S, n->t[k], t)];
                    double v, d[4], d2[4][4], bnd, db[4];
                    angle_rect(vaf, vat, vif, vit, tan(n->angmax[k]), &v, d, d2, &bnd, db);
                    ADD(row_of(S, G_ANG, k, t), v, bnd);
                    angle_rect(vaf, vat, vif, vit, tan(n->angmin[k]), &v, d, d2, &bnd, db);
                    ADD(row_of(S, G_ANL, k, t), v, bnd);
                } else
                    ADD(row_of(S, G_ANG, k, t), vaf - vat, fabs(vaf) + fabs(vat));
                double r2 = n->rate_a[k] * n->rate_a[k];
                ADD(row_of(S, G_THF, k, t), pf * pf + qf * qf - r2, pf * pf + qf * qf + r2);
                ADD(row_of(S, G_THT, k, t), pt * pt + qt * qt - r2, pt * pt + qt * qt + r2);
            }
            for (int i = 0; i < nb; i++) {
                double vm = x[v_vm(S, i, t)], vr = x[v_va(S, i, t)];
                double V2 = S->rect ? vr * vr + vm * vm : vm * vm; /* |V_i|^2 */
                double Pd = S->Pd[t * nb + i], Qd = S->Qd[t * nb + i];
                ADD(row_of(S, G_PB, i, t), Pd + n->gs[i] * V2, fabs(Pd) + fabs(n->gs[i]) * V2);
                ADD(row_of(S, G_QB, i, t), Qd - n->bs[i] * V2, fabs(Qd) + fabs(n->bs[i]) * V2);
                if (S->rect)
                    ADD(row_of(S, G_VM, i, t), V2, V2);
            }
            for (int64_t a = 0; a < 2 * nl; a++) { /* constraint! augmentation: +p[a] at a.bus */
                int i = arc_bus(S, a);
                double p = x[v_p(S, a, t)], q = x[v_q(S, a, t)];
                ADD(row_of(S, G_PB, i, t), p, fabs(p));
                ADD(row_of(S, G_QB, i, t), q, fabs(q));
            }
            for (int g = 0; g < n->ngen; g++) { /* -pg[g] at g.bus */
                int i = n->gen_bus[g];
                double pg = x[v_pg(S, g, t)], qg = x[v_qg(S, g, t)];
                ADD(row_of(S, G_PB, i, t), -pg, fabs(pg));
                ADD(row_of(S, G_QB, i, t), -qg, fabs(qg));
            }
            if (S->ramp && t >= 1)
                for (int g = 0; g < n->ngen; g++) {
                    double a = x[v_pg(S, g, t)], b = x[v_pg(S, g, t - 1)];
                    ADD(row_of(S, G_RAMP, g, t), a - b, fabs(a) + fabs(b));
                }
            for (int k = 0; k < S->ns; k++) {
                const ora_storage *st = &S->st;
                int bus = st->bus[k];
                double ps = x[v_st(S, V_PS, k, t)], qs = x[v_st(S, V_QS, k, t)];
                double sc = x[v_st(S, V_SC, k, t)], sd = x[v_st(S, V_SD, k, t)];
                double se = x[v_st(S, V_SE, k, t)], sp = t ? x[v_st(S, V_SE, k, t - 1)] : 0.0;
                double vm = x[v_vm(S, bus, t)];
                ADD(row_of(S, G_PB, bus, t), ps, fabs(ps)); /* drawn from the bus */
                ADD(row_of(S, G_QB, bus, t), qs, fabs(qs));
                double chg = st->dt * (st->eta_c[k] * sc - sd / st->eta_d[k]);
                ADD(row_st(S, R_SOC, k, t), se - sp - chg,
                    fabs(se) + fabs(sp) + st->dt * (st->eta_c[k] * fabs(sc) + fabs(sd) / st->eta_d[k]));
                double loss = st->r[k] * (ps * ps + qs * qs) / (vm * vm);
                ADD(row_st(S, R_LOSS, k, t), ps + sd - sc - loss, fabs(ps) + fabs(sd) + fabs(sc) + loss);
                ADD(row_st(S, R_STH, k, t), ps * ps + qs * qs, ps * ps + qs * qs);
                if (S->compl)
                    ADD(row_st(S, R_CMP, k, t), sc * sd, fabs(sc * sd));
            }
        }
    }
    if (C->link) {
        int ng = C->in[0].net.ngen;
        for (int s = 1; s < C->ninst; s++)
            for (int g = 0; g < ng; g++) {
                double a = x[v_pg(&C->in[s], g, 0)], b = x[v_pg(&C->in[0], g, 0)];
                ADD(C->link_row + g + (int64_t)ng * (s - 1), a - b, fabs(a) + fabs(b));
            }
    }
    if (C->reserve > 0.0) {
        int64_t row = C->res_row;
        for (int s = 0; s < C->ninst; s++)
            for (int t = 0; t < C->in[s].net.nperiod; t++, row++)
                for (int g = 0; g < C->in[s].net.ngen; g++) {
                    double a = x[v_pg(&C->in[s], g, t)];
                    ADD(row, a, fabs(a));
                }
    }
#undef ADD
}

/* ---------------------------------------------------------------- Jacobian -- */

typedef struct {
    const int64_t *keys;
    int64_t nnz, n;
    double *vals, *scale;
    int bad;
} acc_t;

static void acc(acc_t *A, int64_t r, int64_t c, double v, double bound)
{
    int64_t e = find(A->keys, A->nnz, r * A->n + c);
    if (e < 0) {
        if (!A->bad)
            set_err("entry (%lld, %lld) not in the pattern", (long long)r, (long long)c);
        A->bad = 1;
        return;
    }
    A->vals[e] += v;
    if (A->scale)
        A->scale[e] += bound;
}

/* Hessian accumulation into the lower triangle */
static void acc_sym(acc_t *A, int64_t r, int64_t c, double v, double bound)
{
    if (r >= c)
        acc(A, r, c, v, bound);
    else
        acc(A, c, r, v, bound);
}

int ora_jac(const ora_ctx *C, const double *x, double *vals, double *scale)
{
    acc_t A = {C->jkey, C->nnzj, C->n, vals, scale, 0};
    memset(vals, 0, sizeof(double) * C->nnzj);
    if (scale)
        memset(scale, 0, sizeof(double) * C->nnzj);
    for (int s = 0; s < C->ninst; s++) {
        const inst_t *S = &C->in[s];
        const ora_net *n = &S->net;
        int64_t nl = n->nbranch;
        for (int t = 0; t < n->nperiod; t++) {
            acc(&A, row_of(S, G_REF, 0, t), S->rect ? v_vm(S, n->ref_bus, t) : v_va(S, n->ref_bus, t),
                1.0, 1.0);
            for (int k = 0; k < nl; k++) {
                end_t fr, to;
                ends_of(S, x, k, t, &fr, &to);
                /* flow row = own variable - Re/Im S(u) */
                const end_t *ends[2] = {&fr, &to};
                int gP[2] = {G_FPF, G_FPT}, gQ[2] = {G_FQF, G_FQT};
                for (int side = 0; side < 2; side++) {
                    const end_t *E = ends[side];
                    int64_t rP = row_of(S, gP[side], k, t), rQ = row_of(S, gQ[side], k, t);
                    acc(&A, rP, E->pvar, 1.0, 1.0);
                    acc(&A, rQ, E->qvar, 1.0, 1.0);
                    for (int d = 0; d < 4; d++) {
                        acc(&A, rP, E->u[d], -creal(E->e.dS[d]), E->e.bdS[d]);
                        acc(&A, rQ, E->u[d], -cimag(E->e.dS[d]), E->e.bdS[d]);
                    }
                }
                if (S->rect) { /* local order of the from-end: (vr_f, vr_t, vi_f, vi_t) */
                    double v, d[4], d2[4][4], bnd, db[4];
                    double xv[4] = {x[fr.u[0]], x[fr.u[1]], x[fr.u[2]], x[fr.u[3]]};
                    angle_rect(xv[0], xv[1], xv[2], xv[3], tan(n->angmax[k]), &v, d, d2, &bnd, db);
                    for (int q = 0; q < 4; q++)
                        acc(&A, row_of(S, G_ANG, k, t), fr.u[q], d[q], db[q]);
                    angle_rect(xv[0], xv[1], xv[2], xv[3], tan(n->angmin[k]), &v, d, d2, &bnd, db);
                    for (int q = 0; q < 4; q++)
                        acc(&A, row_of(S, G_ANL, k, t), fr.u[q], d[q], db[q]);
                } else {
                    acc(&A, row_of(S, G_ANG, k, t), v_va(S, n->f[k], t), 1.0, 1.0);
                    acc(&A, row_of(S, G_ANG, k, t), v_va(S, n->t[k], t), -1.0, 1.0);
                }
                double pf = x[fr.pvar], qf = x[fr.qvar], pt = x[to.pvar], qt = x[to.qvar];
                acc(&A, row_of(S, G_THF, k, t), fr.pvar, 2.0 * pf, 2.0 * fabs(pf));
                acc(&A, row_of(S, G_THF, k, t), fr.qvar, 2.0 * qf, 2.0 * fabs(qf));
                acc(&A, row_of(S, G_THT, k, t), to.pvar, 2.0 * pt, 2.0 * fabs(pt));
                acc(&A, row_of(S, G_THT, k, t), to.qvar, 2.0 * qt, 2.0 * fabs(qt));
            }
            for (int i = 0; i < n->nbus; i++) {
                /* d|V|^2: polar 2 vm on vm; rectangular 2 vr on vr and 2 vi on vi */
                int nv = S->rect ? 2 : 1;
                int64_t col[2] = {v_vm(S, i, t), v_va(S, i, t)};
                for (int q = 0; q < nv; q++) {
                    double v = x[col[q]];
                    acc(&A, row_of(S, G_PB, i, t), col[q], 2.0 * n->gs[i] * v, 2.0 * fabs(n->gs[i] * v));
                    acc(&A, row_of(S, G_QB, i, t), col[q], -2.0 * n->bs[i] * v, 2.0 * fabs(n->bs[i] * v));
                    if (S->rect)
                        acc(&A, row_of(S, G_VM, i, t), col[q], 2.0 * v, 2.0 * fabs(v));
                }
            }
            for (int64_t a = 0; a < 2 * nl; a++) {
                int i = arc_bus(S, a);
                acc(&A, row_of(S, G_PB, i, t), v_p(S, a, t), 1.0, 1.0);
                acc(&A, row_of(S, G_QB, i, t), v_q(S, a, t), 1.0, 1.0);
            }
            for (int g = 0; g < n->ngen; g++) {
                int i = n->gen_bus[g];
                acc(&A, row_of(S, G_PB, i, t), v_pg(S, g, t), -1.0, 1.0);
                acc(&A, row_of(S, G_QB, i, t), v_qg(S, g, t), -1.0, 1.0);
            }
            if (S->ramp && t >= 1)
                for (int g = 0; g < n->ngen; g++) {
                    acc(&A, row_of(S, G_RAMP, g, t), v_pg(S, g, t), 1.0, 1.0);
                    acc(&A, row_of(S, G_RAMP, g, t), v_pg(S, g, t - 1), -1.0, 1.0);
                }
            for (int k = 0; k < S->ns; k++) {
                const ora_storage *st = &S->st;
                int bus = st->bus[k];
                int64_t ips = v_st(S, V_PS, k, t), iqs = v_st(S, V_QS, k, t);
                int64_t isc = v_st(S, V_SC, k, t), isd = v_st(S, V_SD, k, t), ise = v_st(S, V_SE, k, t);
                double ps = x[ips], qs = x[iqs], sc = x[isc], sd = x[isd];
                double vm = x[v_vm(S, bus, t)], r = st->r[k], s2 = ps * ps + qs * qs;
                acc(&A, row_of(S, G_PB, bus, t), ips, 1.0, 1.0);
                acc(&A, row_of(S, G_QB, bus, t), iqs, 1.0, 1.0);
                int64_t row = row_st(S, R_SOC, k, t);
                acc(&A, row, isc, -st->dt * st->eta_c[k], st->dt * st->eta_c[k]);
                acc(&A, row, isd, st->dt / st->eta_d[k], st->dt / st->eta_d[k]);
                acc(&A, row, ise, 1.0, 1.0);
                if (t >= 1)
                    acc(&A, row, v_st(S, V_SE, k, t - 1), -1.0, 1.0);
                /* d/dx of -r s2 vm^-2: -2 r ps vm^-2, -2 r qs vm^-2, 2 r s2 vm^-3 */
                row = row_st(S, R_LOSS, k, t);
                acc(&A, row, v_vm(S, bus, t), 2.0 * r * s2 / (vm * vm * vm), 2.0 * r * s2 / fabs(vm * vm * vm));
                acc(&A, row, ips, 1.0 - 2.0 * r * ps / (vm * vm), 1.0 + 2.0 * r * fabs(ps) / (vm * vm));
                acc(&A, row, iqs, -2.0 * r * qs / (vm * vm), 2.0 * r * fabs(qs) / (vm * vm));
                acc(&A, row, isc, -1.0, 1.0);
                acc(&A, row, isd, 1.0, 1.0);
                acc(&A, row_st(S, R_STH, k, t), ips, 2.0 * ps, 2.0 * fabs(ps));
                acc(&A, row_st(S, R_STH, k, t), iqs, 2.0 * qs, 2.0 * fabs(qs));
                if (S->compl) {
                    acc(&A, row_st(S, R_CMP, k, t), isc, sd, fabs(sd));
                    acc(&A, row_st(S, R_CMP, k, t), isd, sc, fabs(sc));
                }
            }
        }
    }
    if (C->link) {
        int ng = C->in[0].net.ngen;
        for (int s = 1; s < C->ninst; s++)
            for (int g = 0; g < ng; g++) {
                int64_t row = C->link_row + g + (int64_t)ng * (s - 1);
                acc(&A, row, v_pg(&C->in[s], g, 0), 1.0, 1.0);
                acc(&A, row, v_pg(&C->in[0], g, 0), -1.0, 1.0);
            }
    }
    if (C->reserve > 0.0) {
        int64_t row = C->res_row;
        for (int s = 0; s < C->ninst; s++)
            for (int t = 0; t < C->in[s].net.nperiod; t++, row++)
                for (int g = 0; g < C->in[s].net.ngen; g++)
                    acc(&A, row, v_pg(&C->in[s], g, t), 1.0, 1.0);
    }
    return A.bad ? -1 : 0;
}

/* ----------------------------------------------------------------- Hessian -- */

int ora_hess(const ora_ctx *C, const double *x, const double *lambda, double sigma, double *vals,
             double *scale)
{
    acc_t A = {C->hkey, C->nnzh, C->n, vals, scale, 0};
    memset(vals, 0, sizeof(double) * C->nnzh);
    if (scale)
        memset(scale, 0, sizeof(double) * C->nnzh);
    for (int s = 0; s < C->ninst; s++) {
        const inst_t *S = &C->in[s];
        const ora_net *n = &S->net;
        int64_t nl = n->nbranch;
        for (int t = 0; t < n->nperiod; t++) {
            /* sigma * cost: d2/dpg2 (c2 pg^2 + c1 pg + c0) = 2 c2 */
            for (int g = 0; g < n->ngen; g++)
                acc_sym(&A, v_pg(S, g, t), v_pg(S, g, t), sigma * 2.0 * n->c2[g],
                        fabs(sigma * 2.0 * n->c2[g]));
            /* flow rows: lambda_r * (own - Re/Im S) contributes -lambda_r Re/Im d2S */
            for (int k = 0; k < nl; k++) {
                end_t fr, to;
                ends_of(S, x, k, t, &fr, &to);
                const end_t *ends[2] = {&fr, &to};
                int gP[2] = {G_FPF, G_FPT}, gQ[2] = {G_FQF, G_FQT};
                for (int side = 0; side < 2; side++) {
                    const end_t *E = ends[side];
                    double lP = lambda[row_of(S, gP[side], k, t)];
                    double lQ = lambda[row_of(S, gQ[side], k, t)];
                    if (S->rect) { /* the structurally nonzero pairs only */
                        for (int q = 0; q < 6; q++) {
                            int a = RECT_D2[q][0], b = RECT_D2[q][1];
                            double v = -lP * creal(E->e.d2S[a][b]) - lQ * cimag(E->e.d2S[a][b]);
                            double bnd = (fabs(lP) + fabs(lQ)) * E->e.bd2S[a][b];
                            acc_sym(&A, E->u[a], E->u[b], v, bnd);
                        }
                        continue;
                    }
                    for (int a = 0; a < 4; a++)
                        for (int b = a; b < 4; b++) {
                            double v = -lP * creal(E->e.d2S[a][b]) - lQ * cimag(E->e.d2S[a][b]);
                            double bnd = (fabs(lP) + fabs(lQ)) * E->e.bd2S[a][b];
                            acc_sym(&A, E->u[a], E->u[b], v, bnd);
                        }
                }
                if (S->rect) { /* the two angle rows: constant second derivatives */
                    double v, d[4], dh[4][4], dl[4][4], bnd, db[4];
                    double lh = lambda[row_of(S, G_ANG, k, t)], ll = lambda[row_of(S, G_ANL, k, t)];
                    double xv[4] = {x[fr.u[0]], x[fr.u[1]], x[fr.u[2]], x[fr.u[3]]};
                    angle_rect(xv[0], xv[1], xv[2], xv[3], tan(n->angmax[k]), &v, d, dh, &bnd, db);
                    angle_rect(xv[0], xv[1], xv[2], xv[3], tan(n->angmin[k]), &v, d, dl, &bnd, db);
                    int pr[4][2] = {{0, 1}, {2, 3}, {0, 3}, {1, 2}};
                    for (int q = 0; q < 4; q++) {
                        int a = pr[q][0], b = pr[q][1];
                        acc_sym(&A, fr.u[a], fr.u[b], lh * dh[a][b] + ll * dl[a][b],
                                fabs(lh * dh[a][b]) + fabs(ll * dl[a][b]));
                    }
                }
                /* thermal rows: lambda * 2 on (p, p) and (q, q) of each arc */
                double lf = lambda[row_of(S, G_THF, k, t)], lt = lambda[row_of(S, G_THT, k, t)];
                acc_sym(&A, fr.pvar, fr.pvar, 2.0 * lf, 2.0 * fabs(lf));
                acc_sym(&A, fr.qvar, fr.qvar, 2.0 * lf, 2.0 * fabs(lf));
                acc_sym(&A, to.pvar, to.pvar, 2.0 * lt, 2.0 * fabs(lt));
                acc_sym(&A, to.qvar, to.qvar, 2.0 * lt, 2.0 * fabs(lt));
            }
            /* balance demand terms gs |V|^2 (P) and -bs |V|^2 (Q), and the
             * rectangular form's magnitude row |V|^2: d2|V|^2 = 2 on vm (polar),
             * on vr and on vi (rectangular) */
            for (int i = 0; i < n->nbus; i++) {
                double lP = lambda[row_of(S, G_PB, i, t)], lQ = lambda[row_of(S, G_QB, i, t)];
                double lV = S->rect ? lambda[row_of(S, G_VM, i, t)] : 0.0;
                double v = 2.0 * n->gs[i] * lP - 2.0 * n->bs[i] * lQ + 2.0 * lV;
                double bnd = 2.0 * fabs(n->gs[i] * lP) + 2.0 * fabs(n->bs[i] * lQ) + 2.0 * fabs(lV);
                acc_sym(&A, v_vm(S, i, t), v_vm(S, i, t), v, bnd);
                if (S->rect)
                    acc_sym(&A, v_va(S, i, t), v_va(S, i, t), v, bnd);
            }
            /* storage: mu (loss row) times the Hessian of -r (ps^2 + qs^2) vm^-2,
             * lambda (thermal) times 2 on (ps, ps), (qs, qs), and the
             * complementarity row's 1 on (sd, sc) */
            for (int k = 0; k < S->ns; k++) {
                const ora_storage *st = &S->st;
                int64_t ivm = v_vm(S, st->bus[k], t);
                int64_t ips = v_st(S, V_PS, k, t), iqs = v_st(S, V_QS, k, t);
                double ps = x[ips], qs = x[iqs], vm = x[ivm], r = st->r[k];
                double mu = lambda[row_st(S, R_LOSS, k, t)], lt = lambda[row_st(S, R_STH, k, t)];
                double v2 = vm * vm, v3 = v2 * vm, v4 = v2 * v2, s2 = ps * ps + qs * qs;
                acc_sym(&A, ips, ips, -2.0 * r * mu / v2 + 2.0 * lt, 2.0 * fabs(r * mu) / v2 + 2.0 * fabs(lt));
                acc_sym(&A, iqs, iqs, -2.0 * r * mu / v2 + 2.0 * lt, 2.0 * fabs(r * mu) / v2 + 2.0 * fabs(lt));
                acc_sym(&A, ips, ivm, 4.0 * r * mu * ps / v3, 4.0 * fabs(r * mu * ps / v3));
                acc_sym(&A, iqs, ivm, 4.0 * r * mu * qs / v3, 4.0 * fabs(r * mu * qs / v3));
                acc_sym(&A, ivm, ivm, -6.0 * r * mu * s2 / v4, 6.0 * fabs(r * mu) * s2 / v4);
                if (S->compl)
                    acc_sym(&A, v_st(S, V_SD, k, t), v_st(S, V_SC, k, t), lambda[row_st(S, R_CMP, k, t)],
                            fabs(lambda[row_st(S, R_CMP, k, t)]));
            }
        }
    }
    return A.bad ? -1 : 0;
}

/* ------------------------------------------------------------------ Cvio -- */

void ora_cvio(const ora_ctx *C, const double *x, double *cons_viol, double *var_viol)
{
    double *c = malloc(sizeof(double) * (C->m + 1));
    double *xl = malloc(sizeof(double) * (C->n + 1)), *xu = malloc(sizeof(double) * (C->n + 1));
    double *gl = malloc(sizeof(double) * (C->m + 1)), *gu = malloc(sizeof(double) * (C->m + 1));
    ora_cons(C, x, c, NULL);
    ora_bounds(C, xl, xu, gl, gu);
    double cv = 0.0, vv = 0.0;
    for (int64_t i = 0; i < C->m; i++) {
        if (gl[i] - c[i] > cv)
            cv = gl[i] - c[i];
        if (c[i] - gu[i] > cv)
            cv = c[i] - gu[i];
    }
    for (int64_t j = 0; j < C->n; j++) {
        if (xl[j] - x[j] > vv)
            vv = xl[j] - x[j];
        if (x[j] - xu[j] > vv)
            vv = x[j] - xu[j];
    }
    *cons_viol = cv;
    *var_viol = vv;
    free(c); free(xl); free(xu); free(gl); free(gu);
}

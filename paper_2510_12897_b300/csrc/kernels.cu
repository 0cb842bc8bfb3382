// Evaluation kernels of libopf (sm_103a, FP64).
//
// One evaluation is two kernels on the caller's stream:
//
//  branch phase  one thread per (instance, period, branch) item. Computes the
//                four flow rows of Listing 3 with their Jacobian rows, the
//                angle-difference and thermal rows, the thermal Hessian
//                diagonals, and the branch's second-order contributions to
//                its two end buses' Hessian rows, which it stores in the
//                per-arc scratch at the arc's slot in its bus's arc list.
//  bus phase     one thread per (instance, period, bus) item, then one per
//                (instance, period, generator) item. Sums the balance rows
//                (the constraint! augmentations of Listing 3), writes their
//                Jacobian rows, assembles the bus's Hessian rows va_i and vm_i
//                from its slots in a fixed order (no atomics), and evaluates
//                the cost, its gradient and Hessian, ramp rows (Listing 6) and
//                linking rows. The objective is reduced in a fixed order by the
//                last block to finish.
//
// Flow arithmetic (pi-model, real expansion): with d = va_f - va_t, the
// from-end power is S_fr = |V_f|^2 conj(Yff) + vm_f vm_t e^{jd} conj(Yft), so
//   P_fr =  Gff vm_f^2 + vm_f vm_t A_ft,   A_ft = Gft cos d + Bft sin d
//   Q_fr = -Bff vm_f^2 + vm_f vm_t B_ft,   B_ft = Gft sin d - Bft cos d
// and at the to-end, with e^{-jd},
//   P_to =  Gtt vm_t^2 + vm_f vm_t A_tf,   A_tf = Gtf cos d - Btf sin d
//   Q_to = -Btt vm_t^2 + vm_f vm_t B_tf,   B_tf = -Gtf sin d - Btf cos d.
// dA_ft/dd = -B_ft, dB_ft/dd = A_ft, dA_tf/dd = B_tf, dB_tf/dd = -A_tf, and
// every second derivative is a combination of these four and the constants.
#include <cstdio>

#include "model.h"

namespace opf {

namespace {

struct KParams {
    DevArrays d;
    int32_t ninst;
    int64_t nbr_items, nbus_items, ngen_items;
    const double *__restrict__ x;
    const double *__restrict__ lam;
    double sigma;
    double *obj, *grad, *c, *jac, *hess;
};

// largest s with prefix[s] <= item (instances with no items are skipped)
__device__ __forceinline__ int find_inst(const int64_t *__restrict__ prefix, int ninst, int64_t item)
{
    int lo = 0, hi = ninst - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(prefix + mid) <= item)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void split(int loc, int count, int T, int &t, int &e)
{
    if (T == 1) {
        t = 0;
        e = loc;
    } else {
        t = loc / count;
        e = loc - t * count;
    }
}

// five Jacobian entries of a flow row, columns ascending:
// (va_lo, va_hi, vm_lo, vm_hi, own) where lo/hi order the two end buses
__device__ __forceinline__ void put5(double *J, bool f_lo, double vaf, double vat, double vmf,
                                     double vmt)
{
    J[0] = f_lo ? vaf : vat;
    J[1] = f_lo ? vat : vaf;
    J[2] = f_lo ? vmf : vmt;
    J[3] = f_lo ? vmt : vmf;
    J[4] = 1.0;
}

template <bool CONS, bool JAC, bool HESS, bool GRAD>
__global__ void branch_kernel(const KParams P)
{
    const DevArrays &d = P.d;
    const double *__restrict__ x = P.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < P.nbr_items; it += stride) {
        const int s = P.ninst == 1 ? 0 : find_inst(d.br_items, P.ninst, it);
        const InstDev *I = d.inst + s;
        const int nl = __ldg(&I->nl), nb = __ldg(&I->nb), ng = __ldg(&I->ng), T = __ldg(&I->T);
        int t, k;
        split((int)(it - __ldg(d.br_items + s)), nl, T, t, k);
        const int64_t nbT = (int64_t)nb * T, ngT = (int64_t)ng * T, nlT = (int64_t)nl * T;
        const int64_t na = 2 * (int64_t)nl;
        const int64_t x0 = __ldg(&I->x0), c0 = __ldg(&I->c0);
        const int64_t rk = k + (int64_t)nl * t;  // element index inside each branch group
        const int kb = __ldg(&I->br0) + k;

        const int2 ft = __ldg(d.br_ft + kb);
        const int64_t xva = x0 + (int64_t)nb * t, xvm = xva + nbT;
        const int64_t xp = x0 + 2 * nbT + 2 * ngT + na * t, xq = xp + na * T;
        const double vaf = __ldg(x + xva + ft.x), vat = __ldg(x + xva + ft.y);
        const double vmf = __ldg(x + xvm + ft.x), vmt = __ldg(x + xvm + ft.y);
        const double2 Yff = __ldg(d.y_ff + kb), Yft = __ldg(d.y_ft + kb);
        const double2 Ytf = __ldg(d.y_tf + kb), Ytt = __ldg(d.y_tt + kb);

        double sn, cs;
        sincos(vaf - vat, &sn, &cs);
        const double vft = vmf * vmt;
        const double Aft = fma(Yft.x, cs, Yft.y * sn);
        const double Bft = fma(Yft.x, sn, -Yft.y * cs);
        const double Atf = fma(Ytf.x, cs, -Ytf.y * sn);
        const double Btf = -fma(Ytf.x, sn, Ytf.y * cs);

        double pf = 0, qf = 0, pt = 0, qt = 0;
        if (CONS || JAC || HESS) {
            pf = __ldg(x + xp + k);
            pt = __ldg(x + xp + nl + k);
            qf = __ldg(x + xq + k);
            qt = __ldg(x + xq + nl + k);
        }
        if (CONS) {
            const double vf2 = vmf * vmf, vt2 = vmt * vmt;
            double *c = P.c + c0 + T + rk;
            c[0] = pf - fma(Yff.x, vf2, vft * Aft);
            c[nlT] = qf - fma(-Yff.y, vf2, vft * Bft);
            c[2 * nlT] = pt - fma(Ytt.x, vt2, vft * Atf);
            c[3 * nlT] = qt - fma(-Ytt.y, vt2, vft * Btf);
            c[4 * nlT] = vaf - vat;
            const double r2 = __ldg(d.rate2 + kb);
            c[5 * nlT + 2 * nbT] = fma(pf, pf, qf * qf) - r2;
            c[6 * nlT + 2 * nbT] = fma(pt, pt, qt * qt) - r2;
        }
        if (JAC) {
            const int64_t j0 = __ldg(&I->j0), jP = __ldg(&I->jP);
            const bool f_lo = ft.x < ft.y;
            double *J = P.jac + j0 + T + 5 * rk;
            // row p_fr - P_fr
            put5(J, f_lo, vft * Bft, -vft * Bft, -fma(2.0 * Yff.x, vmf, vmt * Aft), -vmf * Aft);
            // row q_fr - Q_fr
            put5(J + 5 * nlT, f_lo, -vft * Aft, vft * Aft, fma(2.0 * Yff.y, vmf, -vmt * Bft), -vmf * Bft);
            // row p_to - P_to
            put5(J + 10 * nlT, f_lo, -vft * Btf, vft * Btf, -vmt * Atf, -fma(2.0 * Ytt.x, vmt, vmf * Atf));
            // row q_to - Q_to
            put5(J + 15 * nlT, f_lo, vft * Atf, -vft * Atf, -vmt * Btf, fma(2.0 * Ytt.y, vmt, -vmf * Btf));
            double *Ja = P.jac + j0 + T + 20 * nlT + 2 * rk;  // angle row va_f - va_t
            Ja[0] = f_lo ? 1.0 : -1.0;
            Ja[1] = f_lo ? -1.0 : 1.0;
            double *Jt = P.jac + j0 + T + 22 * nlT + 2 * jP * T + 2 * rk;  // thermal rows
            Jt[0] = 2.0 * pf;
            Jt[1] = 2.0 * qf;
            Jt[2 * nlT] = 2.0 * pt;
            Jt[2 * nlT + 1] = 2.0 * qt;
        }
        if (HESS || CONS) {
            const int2 pos = __ldg(d.br_pos + kb);
            ArcScratch *S = d.arcs + __ldg(&I->scr0) + na * t;
            if (HESS) {
                const double *L = P.lam + c0 + T + rk;
                const double m1 = __ldg(L), m2 = __ldg(L + nlT), m3 = __ldg(L + 2 * nlT),
                             m4 = __ldg(L + 3 * nlT);
                const double lf = __ldg(L + 5 * nlT + 2 * nbT), lt = __ldg(L + 6 * nlT + 2 * nbT);
                // U = sum_r mu_r val_r(d), V = dU/dd, W = weighted vm^2 coefficients
                const double U = fma(m1, Aft, fma(m2, Bft, fma(m3, Atf, m4 * Btf)));
                const double V = fma(-m1, Bft, fma(m2, Aft, fma(m3, Btf, -m4 * Atf)));
                const double Wf = fma(m1, Yff.x, -m2 * Yff.y);
                const double Wt = fma(m3, Ytt.x, -m4 * Ytt.y);
                const double vU = vft * U;
                double2 *sf = reinterpret_cast<double2 *>(S + pos.x);
                double2 *st = reinterpret_cast<double2 *>(S + pos.y);
                sf[0] = make_double2(pf, qf);
                sf[1] = make_double2(vU, -vmt * V);
                sf[2] = make_double2(-2.0 * Wf, vmt * V);
                sf[3] = make_double2(-vU, -U);
                st[0] = make_double2(pt, qt);
                st[1] = make_double2(vU, vmf * V);
                st[2] = make_double2(-2.0 * Wt, -vmf * V);
                st[3] = make_double2(-vU, -U);
                const int64_t hpq = __ldg(&I->h0) + (__ldg(&I->hva) + __ldg(&I->hvm)) * T + ngT;
                double *Hp = P.hess + hpq + k + na * t;
                Hp[0] = 2.0 * lf;         // (p_fr, p_fr)
                Hp[nl] = 2.0 * lt;        // (p_to, p_to)
                Hp[na * T] = 2.0 * lf;    // (q_fr, q_fr)
                Hp[na * T + nl] = 2.0 * lt;
            } else {
                reinterpret_cast<double2 *>(S + pos.x)[0] = make_double2(pf, qf);
                reinterpret_cast<double2 *>(S + pos.y)[0] = make_double2(pt, qt);
            }
        }
        if (GRAD) {
            P.grad[xp + k] = 0.0;
            P.grad[xp + nl + k] = 0.0;
            P.grad[xq + k] = 0.0;
            P.grad[xq + nl + k] = 0.0;
        }
    }
}

template <bool CONS, bool JAC, bool HESS, bool GRAD, bool OBJ>
__global__ void bus_kernel(const KParams P)
{
    const DevArrays &d = P.d;
    const double *__restrict__ x = P.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t total = P.nbus_items + P.ngen_items;
    double obj_acc = 0.0;
    for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < total; it += stride) {
        if (it < P.nbus_items) {
            const int s = P.ninst == 1 ? 0 : find_inst(d.bus_items, P.ninst, it);
            const InstDev *I = d.inst + s;
            const int nl = __ldg(&I->nl), nb = __ldg(&I->nb), ng = __ldg(&I->ng), T = __ldg(&I->T);
            int t, i;
            split((int)(it - __ldg(d.bus_items + s)), nb, T, t, i);
            const int64_t nbT = (int64_t)nb * T, ngT = (int64_t)ng * T, nlT = (int64_t)nl * T;
            const int64_t na = 2 * (int64_t)nl;
            const int64_t x0 = __ldg(&I->x0), c0 = __ldg(&I->c0);
            const int64_t xva = x0 + (int64_t)nb * t, xvm = xva + nbT;
            const int ib = __ldg(&I->bus0) + i, bp = __ldg(&I->bptr0) + i;
            const double vm = __ldg(x + xvm + i);
            const double2 gb = __ldg(d.gsbs + ib);
            const int a0 = __ldg(d.arc_ptr + bp), a1 = __ldg(d.arc_ptr + bp + 1);
            const ArcScratch *S = d.arcs + __ldg(&I->scr0) + na * t;
            if (GRAD) {
                P.grad[xva + i] = 0.0;
                P.grad[xvm + i] = 0.0;
            }
            if (i == __ldg(&I->ref)) {
                if (CONS)
                    P.c[c0 + t] = __ldg(x + xva + i);
                if (JAC)
                    P.jac[__ldg(&I->j0) + t] = 1.0;
            }
            const int g0 = __ldg(d.gen_ptr + bp), g1 = __ldg(d.gen_ptr + bp + 1);
            if (CONS) {
                const int64_t pd = __ldg(&I->pd0) + (int64_t)nb * t + i;
                double Pb = fma(gb.x, vm * vm, __ldg(d.Pd + pd));
                double Qb = fma(-gb.y, vm * vm, __ldg(d.Qd + pd));
                for (int a = a0; a < a1; a++) {
                    const double2 pq = __ldg(reinterpret_cast<const double2 *>(S + a));
                    Pb += pq.x;
                    Qb += pq.y;
                }
                const int gl0 = __ldg(&I->gl0);
                const int64_t xpg = x0 + 2 * nbT + (int64_t)ng * t, xqg = xpg + ngT;
                for (int gp = g0; gp < g1; gp++) {
                    const int g = __ldg(d.gen_list + gl0 + gp);
                    Pb -= __ldg(x + xpg + g);
                    Qb -= __ldg(x + xqg + g);
                }
                P.c[c0 + T + 5 * nlT + (int64_t)nb * t + i] = Pb;
                P.c[c0 + T + 5 * nlT + nbT + (int64_t)nb * t + i] = Qb;
            }
            if (JAC) {
                const int64_t jP = __ldg(&I->jP);
                double *JP = P.jac + __ldg(&I->j0) + T + 22 * nlT + jP * t + __ldg(d.jpos + ib);
                double *JQ = JP + jP * T;
                JP[0] = 2.0 * gb.x * vm;
                JQ[0] = -2.0 * gb.y * vm;
                int e = 1;
                for (int gp = g0; gp < g1; gp++, e++) {
                    JP[e] = -1.0;
                    JQ[e] = -1.0;
                }
                for (int a = a0; a < a1; a++, e++) {
                    JP[e] = 1.0;
                    JQ[e] = 1.0;
                }
            }
            if (HESS) {
                const double lP = __ldg(P.lam + c0 + T + 5 * nlT + (int64_t)nb * t + i);
                const double lQ = __ldg(P.lam + c0 + T + 5 * nlT + nbT + (int64_t)nb * t + i);
                double daa = 0.0, dma = 0.0, dmm = fma(2.0 * gb.x, lP, -2.0 * gb.y * lQ);
                for (int a = a0; a < a1; a++) {
                    const double2 v1 = __ldg(reinterpret_cast<const double2 *>(S + a) + 1);
                    const double2 v2 = __ldg(reinterpret_cast<const double2 *>(S + a) + 2);
                    daa += v1.x;
                    dma += v1.y;
                    dmm += v2.x;
                }
                const int64_t h0 = __ldg(&I->h0), hva = __ldg(&I->hva), hvm = __ldg(&I->hvm);
                double *Hvm = P.hess + h0 + hva * T + hvm * t + __ldg(d.hvm_pos + ib);
                if (a1 > a0) {
                    // far bus of each of this instance's slots (2 nl per instance)
                    const int32_t *far = d.arc_nbr + 2 * (int64_t)__ldg(&I->br0);
                    double *Hva = P.hess + h0 + hva * t + __ldg(d.hva_pos + ib);
                    // row va_i: (va_i, va_j) for far buses j < i, then (va_i, va_i)
                    int e = 0, a = a0;
                    while (a < a1) {
                        const int j = __ldg(far + a);
                        if (j > i)
                            break;
                        double acc = 0.0;
                        for (; a < a1 && __ldg(far + a) == j; a++)
                            acc += __ldg(&S[a].x_aa);
                        Hva[e++] = acc;
                    }
                    Hva[e] = daa;
                    // row vm_i: (vm_i, va_j) for j in far buses and i, ascending
                    e = 0;
                    a = a0;
                    bool self = false;
                    while (a < a1) {
                        const int j = __ldg(far + a);
                        if (!self && j > i) {
                            Hvm[e++] = dma;
                            self = true;
                        }
                        double acc = 0.0;
                        for (; a < a1 && __ldg(far + a) == j; a++)
                            acc += __ldg(&S[a].x_ma);
                        Hvm[e++] = acc;
                    }
                    if (!self)
                        Hvm[e++] = dma;
                    // then (vm_i, vm_j) for j < i, then (vm_i, vm_i)
                    a = a0;
                    while (a < a1) {
                        const int j = __ldg(far + a);
                        if (j > i)
                            break;
                        double acc = 0.0;
                        for (; a < a1 && __ldg(far + a) == j; a++)
                            acc += __ldg(&S[a].x_mm);
                        Hvm[e++] = acc;
                    }
                    Hvm[e] = dmm;
                } else {
                    Hvm[0] = dmm;
                }
            }
        } else {
            const int64_t gi = it - P.nbus_items;
            const int s = P.ninst == 1 ? 0 : find_inst(d.gen_items, P.ninst, gi);
            const InstDev *I = d.inst + s;
            const int nl = __ldg(&I->nl), nb = __ldg(&I->nb), ng = __ldg(&I->ng), T = __ldg(&I->T);
            int t, g;
            split((int)(gi - __ldg(d.gen_items + s)), ng, T, t, g);
            const int64_t nbT = (int64_t)nb * T, ngT = (int64_t)ng * T, nlT = (int64_t)nl * T;
            const int64_t x0 = __ldg(&I->x0);
            const int64_t xpg = x0 + 2 * nbT + (int64_t)ng * t + g;
            const int gg = __ldg(&I->gen0) + g;
            const double pg = __ldg(x + xpg);
            const double c2 = __ldg(d.c2 + gg), c1 = __ldg(d.c1 + gg);
            if (OBJ)
                obj_acc += fma(fma(c2, pg, c1), pg, __ldg(d.c0 + gg));
            if (GRAD) {
                P.grad[xpg] = fma(2.0 * c2, pg, c1);
                P.grad[xpg + ngT] = 0.0;
            }
            if (HESS) {
                const int64_t hpg = __ldg(&I->h0) + (__ldg(&I->hva) + __ldg(&I->hvm)) * T;
                P.hess[hpg + (int64_t)ng * t + g] = P.sigma * 2.0 * c2;
            }
            if ((CONS || JAC) && t >= 1 && __ldg(&I->ramp)) {
                const int64_t e = g + (int64_t)ng * (t - 1);
                if (CONS)
                    P.c[__ldg(&I->c0) + T + 7 * nlT + 2 * nbT + e] = pg - __ldg(x + xpg - ng);
                if (JAC) {
                    double *J = P.jac + __ldg(&I->j0) + T + 26 * nlT + 2 * __ldg(&I->jP) * T + 2 * e;
                    J[0] = -1.0;
                    J[1] = 1.0;
                }
            }
            const int64_t lc = __ldg(&I->link_c);
            if ((CONS || JAC) && lc >= 0) {
                if (CONS)
                    P.c[lc + g] = pg - __ldg(x + __ldg(&I->link_x0) + g);
                if (JAC) {
                    double *J = P.jac + __ldg(&I->link_j) + 2 * g;
                    J[0] = -1.0;
                    J[1] = 1.0;
                }
            }
        }
    }
    if (OBJ) {
        // fixed-order reduction: warp, block, then the last block over blocks
        __shared__ double wsum[32];
        __shared__ bool last;
        for (int off = 16; off; off >>= 1)
            obj_acc += __shfl_down_sync(0xffffffffu, obj_acc, off);
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if (lane == 0)
            wsum[warp] = obj_acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++)
                b += wsum[w];
            d.obj_part[blockIdx.x] = b;
            __threadfence();
            const unsigned prev = atomicAdd(d.ticket, 1u);
            last = prev == gridDim.x - 1;
        }
        __syncthreads();
        if (last && threadIdx.x == 0) {
            __threadfence();
            double tot = 0.0;
            for (unsigned b = 0; b < gridDim.x; b++)
                tot += __ldcg(d.obj_part + b);
            *P.obj = tot;
            *d.ticket = 0u;  // ready for the next launch
        }
    }
}

// Flat start: va = 0, vm = clamp(1), pg, qg at mid-bounds, p, q = flows at
// those voltages (d = 0: cos d = 1, sin d = 0).
__global__ void flat_kernel(const DevArrays d, int32_t ninst, int64_t nbr_items, int64_t nbus_items,
                            int64_t ngen_items, double *x)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t total = nbr_items + nbus_items + ngen_items;
    for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < total; it += stride) {
        if (it < nbr_items) {
            const int s = ninst == 1 ? 0 : find_inst(d.br_items, ninst, it);
            const InstDev *I = d.inst + s;
            const int nl = I->nl, nb = I->nb, ng = I->ng, T = I->T;
            int t, k;
            split((int)(it - d.br_items[s]), nl, T, t, k);
            const int kb = I->br0 + k;
            const int2 ft = d.br_ft[kb];
            const double2 bf = d.vbnd[I->bus0 + ft.x], bt = d.vbnd[I->bus0 + ft.y];
            const double vmf = fmin(fmax(1.0, bf.x), bf.y), vmt = fmin(fmax(1.0, bt.x), bt.y);
            const double2 Yff = d.y_ff[kb], Yft = d.y_ft[kb], Ytf = d.y_tf[kb], Ytt = d.y_tt[kb];
            const double vft = vmf * vmt;
            const int64_t nbT = (int64_t)nb * T, ngT = (int64_t)ng * T, na = 2 * (int64_t)nl;
            const int64_t xp = I->x0 + 2 * nbT + 2 * ngT + na * t, xq = xp + na * T;
            x[xp + k] = Yff.x * vmf * vmf + vft * Yft.x;
            x[xq + k] = -Yff.y * vmf * vmf - vft * Yft.y;
            x[xp + nl + k] = Ytt.x * vmt * vmt + vft * Ytf.x;
            x[xq + nl + k] = -Ytt.y * vmt * vmt - vft * Ytf.y;
        } else if (it < nbr_items + nbus_items) {
            const int64_t bi = it - nbr_items;
            const int s = ninst == 1 ? 0 : find_inst(d.bus_items, ninst, bi);
            const InstDev *I = d.inst + s;
            int t, i;
            split((int)(bi - d.bus_items[s]), I->nb, I->T, t, i);
            const double2 vb = d.vbnd[I->bus0 + i];
            const int64_t xva = I->x0 + (int64_t)I->nb * t;
            x[xva + i] = 0.0;
            x[xva + (int64_t)I->nb * I->T + i] = fmin(fmax(1.0, vb.x), vb.y);
        } else {
            const int64_t gi = it - nbr_items - nbus_items;
            const int s = ninst == 1 ? 0 : find_inst(d.gen_items, ninst, gi);
            const InstDev *I = d.inst + s;
            int t, g;
            split((int)(gi - d.gen_items[s]), I->ng, I->T, t, g);
            const int gg = I->gen0 + g;
            const int64_t xpg = I->x0 + 2 * (int64_t)I->nb * I->T + (int64_t)I->ng * t + g;
            x[xpg] = 0.5 * (d.pbnd[gg].x + d.pbnd[gg].y);
            x[xpg + (int64_t)I->ng * I->T] = 0.5 * (d.qbnd[gg].x + d.qbnd[gg].y);
        }
    }
}

int grid_for(int64_t items, int block, int ctas_per_sm, int num_sms, int cap)
{
    int64_t g = (items + block - 1) / block;
    if (ctas_per_sm > 0 && g > (int64_t)ctas_per_sm * num_sms)
        g = (int64_t)ctas_per_sm * num_sms;
    if (cap > 0 && g > cap)
        g = cap;
    if (g < 1)
        g = 1;
    return (int)g;
}

template <bool C, bool J, bool H, bool G>
void launch_branch(const KParams &P, int grid, int block, cudaStream_t s)
{
    branch_kernel<C, J, H, G><<<grid, block, 0, s>>>(P);
}

template <bool C, bool J, bool H, bool G, bool O>
void launch_bus(const KParams &P, int grid, int block, cudaStream_t s)
{
    bus_kernel<C, J, H, G, O><<<grid, block, 0, s>>>(P);
}

template <bool C, bool J, bool H>
void dispatch(const KParams &P, bool grad, bool obj, bool run_branch, bool run_bus, int gb, int bb,
              int gu, int bu, cudaStream_t s)
{
    if (run_branch) {
        if (grad)
            launch_branch<C, J, H, true>(P, gb, bb, s);
        else
            launch_branch<C, J, H, false>(P, gb, bb, s);
    }
    if (!run_bus)
        return;
    if (grad) {
        if (obj)
            launch_bus<C, J, H, true, true>(P, gu, bu, s);
        else
            launch_bus<C, J, H, true, false>(P, gu, bu, s);
    } else {
        if (obj)
            launch_bus<C, J, H, false, true>(P, gu, bu, s);
        else
            launch_bus<C, J, H, false, false>(P, gu, bu, s);
    }
}

}  // namespace

int launch_eval(Model &M, const EvalArgs &a, unsigned what, cudaStream_t s, int phases)
{
    KParams P;
    P.d = M.d;
    P.ninst = M.ninst;
    P.nbr_items = M.nbr_items;
    P.nbus_items = M.nbus_items;
    P.ngen_items = M.ngen_items;
    P.x = a.x;
    P.lam = a.lam;
    P.sigma = a.sigma;
    P.obj = a.obj;
    P.grad = a.grad;
    P.c = a.c;
    P.jac = a.jac;
    P.hess = a.hess;
    const bool C = what & W_CONS, J = what & W_JAC, H = what & W_HESS;
    const bool G = what & W_GRAD, O = what & W_OBJ;
    const opf_launch &L = M.launch;
    const int gb = grid_for(M.nbr_items, L.branch_block, L.branch_ctas_per_sm, M.num_sms, 0);
    const int gu = grid_for(M.nbus_items + M.ngen_items, L.bus_block, L.bus_ctas_per_sm, M.num_sms,
                            M.max_part);
    // the branch phase is needed for its rows and for the scratch the bus
    // phase reads (balance sums, Hessian), and to zero the p, q gradient
    const bool run_branch = (phases & 1) && (C || J || H || G) && M.nbr_items > 0;
    const bool run_bus = phases & 2;
    const int bb = L.branch_block, bu = L.bus_block;
    switch ((C ? 1 : 0) | (J ? 2 : 0) | (H ? 4 : 0)) {
    case 0: dispatch<false, false, false>(P, G, O, run_branch, run_bus, gb, bb, gu, bu, s); break;
    case 1: dispatch<true, false, false>(P, G, O, run_branch, run_bus, gb, bb, gu, bu, s); break;
    case 2: dispatch<false, true, false>(P, G, O, run_branch, run_bus, gb, bb, gu, bu, s); break;
    case 3: dispatch<true, true, false>(P, G, O, run_branch, run_bus, gb, bb, gu, bu, s); break;
    case 4: dispatch<false, false, true>(P, G, O, run_branch, run_bus, gb, bb, gu, bu, s); break;
    case 5: dispatch<true, false, true>(P, G, O, run_branch, run_bus, gb, bb, gu, bu, s); break;
    case 6: dispatch<false, true, true>(P, G, O, run_branch, run_bus, gb, bb, gu, bu, s); break;
    default: dispatch<true, true, true>(P, G, O, run_branch, run_bus, gb, bb, gu, bu, s); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("kernel launch failed: %s", cudaGetErrorString(e));
        return OPF_ECUDA;
    }
    return OPF_OK;
}

int launch_flat_start(Model &M, double *x, cudaStream_t s)
{
    const int64_t total = M.nbr_items + M.nbus_items + M.ngen_items;
    const int block = 256;
    const int grid = grid_for(total, block, 8, M.num_sms, 0);
    flat_kernel<<<grid, block, 0, s>>>(M.d, M.ninst, M.nbr_items, M.nbus_items, M.ngen_items, x);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("kernel launch failed: %s", cudaGetErrorString(e));
        return OPF_ECUDA;
    }
    return OPF_OK;
}

}  // namespace opf

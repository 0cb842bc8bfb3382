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
// Both kernels are launched with programmatic dependent launch: each block
// first loads the static network data of its first item (which no kernel
// writes), then waits for the previous kernel in the stream to complete
// (cudaGridDependencySynchronize), then reads x, lambda and the scratch. The
// static prologue and the launch therefore overlap the previous kernel.
//
// FP64 is the scarce resource on this GPU (about 2 FMA per clock per SM), so
// sign flips and selects are done on the integer pipe and every product
// shared between rows is computed once.
//
// Flow arithmetic (pi-model, real expansion): with d = va_f - va_t, the
// from-end power is S_fr = |V_f|^2 conj(Yff) + vm_f vm_t e^{jd} conj(Yft), so
//   P_fr =  Gff vm_f^2 + vm_f vm_t A_ft,   A_ft = Gft cos d + Bft sin d
//   Q_fr = -Bff vm_f^2 + vm_f vm_t B_ft,   B_ft = Gft sin d - Bft cos d
// and at the to-end, with e^{-jd},
//   P_to =  Gtt vm_t^2 + vm_f vm_t A_tf,   A_tf = Gtf cos d - Btf sin d
//   Q_to = -Btt vm_t^2 + vm_f vm_t B_tf,   B_tf = -Gtf sin d - Btf cos d.
// dA_ft/dd = -B_ft, dB_ft/dd = A_ft, dA_tf/dd = B_tf, dB_tf/dd = -A_tf, and
// every second derivative is a combination of these four and the constants:
// with multipliers m1..m4 of the rows p_fr - P_fr, q_fr - Q_fr, p_to - P_to,
// q_to - Q_to, U = m1 A_ft + m2 B_ft + m3 A_tf + m4 B_tf and V = dU/dd, the
// Lagrangian L = sum m_r (own_r - F_r) has
//   d2L/dva_f2 = d2L/dva_t2 = vm_f vm_t U = -d2L/dva_f dva_t,
//   d2L/dvm_f dvm_t = -U,  d2L/dvm_f dva_f = -vm_t V = -d2L/dvm_f dva_t,
//   d2L/dvm_t dva_t = vm_f V = -d2L/dvm_t dva_f,
//   d2L/dvm_f2 = -2 (m1 Gff - m2 Bff),  d2L/dvm_t2 = -2 (m3 Gtt - m4 Btt).
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

// -v on the integer pipe
__device__ __forceinline__ double neg(double v)
{
    return __longlong_as_double(__double_as_longlong(v) ^ (long long)0x8000000000000000ULL);
}

// v or -v on the integer pipe
__device__ __forceinline__ double flip(double v, bool f)
{
    return __longlong_as_double(__double_as_longlong(v) ^ (f ? (long long)0x8000000000000000ULL : 0LL));
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

// static (never written) data of one branch item
struct BrStatic {
    int4 br;  // f, t, slot of the from-arc, slot of the to-arc
    double2 yff, yft, ytf, ytt;
    double r2;
};

__device__ __forceinline__ BrStatic load_br(const DevArrays &d, int kb, bool need_r2)
{
    BrStatic s;
    s.br = __ldg(d.br + kb);
    s.yff = __ldg(d.y_ff + kb);
    s.yft = __ldg(d.y_ft + kb);
    s.ytf = __ldg(d.y_tf + kb);
    s.ytt = __ldg(d.y_tt + kb);
    s.r2 = need_r2 ? __ldg(d.rate2 + kb) : 0.0;
    return s;
}

template <bool CONS, bool JAC, bool HESS, bool GRAD>
__global__ void branch_kernel(const KParams P)
{
    cudaTriggerProgrammaticLaunchCompletion();
    const DevArrays &d = P.d;
    const double *__restrict__ x = P.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;

    auto locate = [&](int64_t item, int &s, int &t, int &k) {
        s = P.ninst == 1 ? 0 : find_inst(d.br_items, P.ninst, item);
        const InstDev *I = d.inst + s;
        split((int)(item - __ldg(d.br_items + s)), __ldg(&I->nl), __ldg(&I->T), t, k);
    };

    int s = 0, t = 0, k = 0;
    BrStatic st{};
    if (it < P.nbr_items) {
        locate(it, s, t, k);
        st = load_br(d, __ldg(&d.inst[s].br0) + k, CONS);
    }
    cudaGridDependencySynchronize();

    for (; it < P.nbr_items; it += stride) {
        const BrStatic cur = st;
        const int cs = s, ct = t, ck = k;
        if (it + stride < P.nbr_items) {  // prefetch the next item's static data
            locate(it + stride, s, t, k);
            st = load_br(d, __ldg(&d.inst[s].br0) + k, CONS);
        }
        const InstDev *I = d.inst + cs;
        const int nl = __ldg(&I->nl), nb = __ldg(&I->nb), ng = __ldg(&I->ng), T = __ldg(&I->T);
        const int64_t nbT = (int64_t)nb * T, ngT = (int64_t)ng * T, nlT = (int64_t)nl * T;
        const int64_t na = 2 * (int64_t)nl;
        const int64_t x0 = __ldg(&I->x0), c0 = __ldg(&I->c0);
        const int64_t rk = ck + (int64_t)nl * ct;  // element index inside each branch group
        const int f = cur.br.x, b = cur.br.y;

        const int64_t xva = x0 + (int64_t)nb * ct, xvm = xva + nbT;
        const int64_t xp = x0 + 2 * nbT + 2 * ngT + na * ct, xq = xp + na * T;
        const double vaf = __ldg(x + xva + f), vat = __ldg(x + xva + b);
        const double vmf = __ldg(x + xvm + f), vmt = __ldg(x + xvm + b);
        double pf = 0, qf = 0, pt = 0, qt = 0;
        if (CONS || JAC || HESS) {
            pf = __ldg(x + xp + ck);
            pt = __ldg(x + xp + nl + ck);
            qf = __ldg(x + xq + ck);
            qt = __ldg(x + xq + nl + ck);
        }
        double m1 = 0, m2 = 0, m3 = 0, m4 = 0, lf = 0, lt = 0;
        if (HESS) {
            const double *L = P.lam + c0 + T + rk;
            m1 = __ldg(L);
            m2 = __ldg(L + nlT);
            m3 = __ldg(L + 2 * nlT);
            m4 = __ldg(L + 3 * nlT);
            lf = __ldg(L + 5 * nlT + 2 * nbT);
            lt = __ldg(L + 6 * nlT + 2 * nbT);
        }
        const double2 Yff = cur.yff, Yft = cur.yft, Ytf = cur.ytf, Ytt = cur.ytt;

        const double dlt = vaf - vat;
        double sn, cs_;
        sincos(dlt, &sn, &cs_);
        const double vft = vmf * vmt;
        const double Aft = fma(Yft.x, cs_, Yft.y * sn);
        const double Bft = fma(Yft.x, sn, neg(Yft.y * cs_));
        const double Atf = fma(Ytf.x, cs_, neg(Ytf.y * sn));
        const double Btf = neg(fma(Ytf.x, sn, Ytf.y * cs_));

        if (CONS) {
            const double vf2 = vmf * vmf, vt2 = vmt * vmt;
            double *c = P.c + c0 + T + rk;
            c[0] = pf - fma(Yff.x, vf2, vft * Aft);
            c[nlT] = qf - fma(neg(Yff.y), vf2, vft * Bft);
            c[2 * nlT] = pt - fma(Ytt.x, vt2, vft * Atf);
            c[3 * nlT] = qt - fma(neg(Ytt.y), vt2, vft * Btf);
            c[4 * nlT] = dlt;
            c[5 * nlT + 2 * nbT] = fma(pf, pf, qf * qf) - cur.r2;
            c[6 * nlT + 2 * nbT] = fma(pt, pt, qt * qt) - cur.r2;
        }
        if (JAC) {
            const int64_t j0 = __ldg(&I->j0), jP = __ldg(&I->jP);
            const bool f_lo = f < b;
            const double v2f = vmf + vmf, v2t = vmt + vmt;
            const double uB = vft * Bft, uA = vft * Aft, wB = vft * Btf, wA = vft * Atf;
            double *J = P.jac + j0 + T + 5 * rk;
            // row p_fr - P_fr
            put5(J, f_lo, uB, neg(uB), neg(fma(Yff.x, v2f, vmt * Aft)), neg(vmf * Aft));
            // row q_fr - Q_fr
            put5(J + 5 * nlT, f_lo, neg(uA), uA, fma(Yff.y, v2f, neg(vmt * Bft)), neg(vmf * Bft));
            // row p_to - P_to
            put5(J + 10 * nlT, f_lo, neg(wB), wB, neg(vmt * Atf), neg(fma(Ytt.x, v2t, vmf * Atf)));
            // row q_to - Q_to
            put5(J + 15 * nlT, f_lo, wA, neg(wA), neg(vmt * Btf), fma(Ytt.y, v2t, neg(vmf * Btf)));
            double *Ja = P.jac + j0 + T + 20 * nlT + 2 * rk;  // angle row va_f - va_t
            Ja[0] = flip(1.0, !f_lo);
            Ja[1] = flip(1.0, f_lo);
            double *Jt = P.jac + j0 + T + 22 * nlT + 2 * jP * T + 2 * rk;  // thermal rows
            Jt[0] = pf + pf;
            Jt[1] = qf + qf;
            Jt[2 * nlT] = pt + pt;
            Jt[2 * nlT + 1] = qt + qt;
        }
        if (HESS || CONS) {
            ArcScratch *S = d.arcs + __ldg(&I->scr0) + na * ct;
            double2 *sf = reinterpret_cast<double2 *>(S + cur.br.z);
            double2 *sto = reinterpret_cast<double2 *>(S + cur.br.w);
            sf[0] = make_double2(pf, qf);
            sto[0] = make_double2(pt, qt);
            if (HESS) {
                const double U = fma(m1, Aft, fma(m2, Bft, fma(m3, Atf, m4 * Btf)));
                const double V = fma(m2, Aft, fma(m3, Btf, fma(neg(m1), Bft, neg(m4 * Atf))));
                const double Wf = fma(m1, Yff.x, neg(m2 * Yff.y));
                const double Wt = fma(m3, Ytt.x, neg(m4 * Ytt.y));
                const double vU = vft * U;
                sf[1] = make_double2(vU, neg(vmt * V));
                sf[2] = make_double2(neg(Wf + Wf), neg(U));
                sto[1] = make_double2(vU, vmf * V);
                sto[2] = make_double2(neg(Wt + Wt), neg(U));
                const int64_t hpq = __ldg(&I->h0) + (__ldg(&I->hva) + __ldg(&I->hvm)) * T + ngT;
                double *Hp = P.hess + hpq + ck + na * ct;
                const double l2f = lf + lf, l2t = lt + lt;
                Hp[0] = l2f;            // (p_fr, p_fr)
                Hp[nl] = l2t;           // (p_to, p_to)
                Hp[na * T] = l2f;       // (q_fr, q_fr)
                Hp[na * T + nl] = l2t;  // (q_to, q_to)
            }
        }
        if (GRAD) {
            P.grad[xp + ck] = 0.0;
            P.grad[xp + nl + ck] = 0.0;
            P.grad[xq + ck] = 0.0;
            P.grad[xq + nl + ck] = 0.0;
        }
    }
}

struct BusStatic {
    int4 a;  // first slot, end slot, first gen entry, end gen entry
    int4 b;  // balance-row offset, va-row offset, vm-row offset, nd | nlt << 16
    double2 gsbs;
};

template <bool CONS, bool JAC, bool HESS, bool GRAD, bool OBJ>
__global__ void bus_kernel(const KParams P)
{
    cudaTriggerProgrammaticLaunchCompletion();
    const DevArrays &d = P.d;
    const double *__restrict__ x = P.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t total = P.nbus_items + P.ngen_items;
    int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;

    auto locate = [&](int64_t item, int &s, int &t, int &e) {
        if (item < P.nbus_items) {
            s = P.ninst == 1 ? 0 : find_inst(d.bus_items, P.ninst, item);
            const InstDev *I = d.inst + s;
            split((int)(item - __ldg(d.bus_items + s)), __ldg(&I->nb), __ldg(&I->T), t, e);
        } else {
            const int64_t gi = item - P.nbus_items;
            s = P.ninst == 1 ? 0 : find_inst(d.gen_items, P.ninst, gi);
            const InstDev *I = d.inst + s;
            split((int)(gi - __ldg(d.gen_items + s)), __ldg(&I->ng), __ldg(&I->T), t, e);
        }
    };
    auto load = [&](int64_t item, int s, int e) {
        BusStatic b{};
        if (item < P.nbus_items) {
            const int ib = __ldg(&d.inst[s].bus0) + e;
            b.a = __ldg(d.bus_a + ib);
            b.b = __ldg(d.bus_b + ib);
            b.gsbs = __ldg(d.gsbs + ib);
        }
        return b;
    };

    int s = 0, t = 0, e = 0;
    BusStatic st{};
    if (it < total) {
        locate(it, s, t, e);
        st = load(it, s, e);
    }
    cudaGridDependencySynchronize();

    double obj_acc = 0.0;
    for (; it < total; it += stride) {
        const BusStatic cur = st;
        const int cs = s, ct = t, ce = e;
        if (it + stride < total) {
            locate(it + stride, s, t, e);
            st = load(it + stride, s, e);
        }
        const InstDev *I = d.inst + cs;
        const int nl = __ldg(&I->nl), nb = __ldg(&I->nb), ng = __ldg(&I->ng), T = __ldg(&I->T);
        const int64_t nbT = (int64_t)nb * T, ngT = (int64_t)ng * T, nlT = (int64_t)nl * T;
        const int64_t x0 = __ldg(&I->x0), c0 = __ldg(&I->c0);
        if (it < P.nbus_items) {
            const int i = ce;
            const int64_t na = 2 * (int64_t)nl;
            const int64_t xva = x0 + (int64_t)nb * ct, xvm = xva + nbT;
            const double vm = __ldg(x + xvm + i);
            const double2 gb = cur.gsbs;
            const int a0 = cur.a.x, a1 = cur.a.y, g0 = cur.a.z, g1 = cur.a.w;
            const ArcScratch *S = d.arcs + __ldg(&I->scr0) + na * ct;
            if (GRAD) {
                P.grad[xva + i] = 0.0;
                P.grad[xvm + i] = 0.0;
            }
            if (i == __ldg(&I->ref)) {
                if (CONS)
                    P.c[c0 + ct] = __ldg(x + xva + i);
                if (JAC)
                    P.jac[__ldg(&I->j0) + ct] = 1.0;
            }
            if (CONS) {
                const int64_t pd = __ldg(&I->pd0) + (int64_t)nb * ct + i;
                const double vm2 = vm * vm;
                double Pb = fma(gb.x, vm2, __ldg(d.Pd + pd));
                double Qb = fma(neg(gb.y), vm2, __ldg(d.Qd + pd));
                const int gl0 = __ldg(&I->gl0);
                const int64_t xpg = x0 + 2 * nbT + (int64_t)ng * ct, xqg = xpg + ngT;
                for (int gp = g0; gp < g1; gp++) {
                    const int g = __ldg(d.gen_list + gl0 + gp);
                    Pb -= __ldg(x + xpg + g);
                    Qb -= __ldg(x + xqg + g);
                }
#pragma unroll 4
                for (int a = a0; a < a1; a++) {
                    const double2 pq = __ldg(reinterpret_cast<const double2 *>(S + a));
                    Pb += pq.x;
                    Qb += pq.y;
                }
                P.c[c0 + T + 5 * nlT + (int64_t)nb * ct + i] = Pb;
                P.c[c0 + T + 5 * nlT + nbT + (int64_t)nb * ct + i] = Qb;
            }
            if (JAC) {
                const int64_t jP = __ldg(&I->jP);
                double *JP = P.jac + __ldg(&I->j0) + T + 22 * nlT + jP * ct + cur.b.x;
                double *JQ = JP + jP * T;
                const double v2 = vm + vm;
                JP[0] = gb.x * v2;
                JQ[0] = neg(gb.y * v2);
                int q = 1;
                for (int gp = g0; gp < g1; gp++, q++) {
                    JP[q] = -1.0;
                    JQ[q] = -1.0;
                }
                for (int a = a0; a < a1; a++, q++) {
                    JP[q] = 1.0;
                    JQ[q] = 1.0;
                }
            }
            if (HESS) {
                const int64_t lb = c0 + T + 5 * nlT + (int64_t)nb * ct + i;
                const double lP = __ldg(P.lam + lb), lQ = __ldg(P.lam + lb + nbT);
                const int64_t h0 = __ldg(&I->h0), hva = __ldg(&I->hva), hvm = __ldg(&I->hvm);
                double *Hvm = P.hess + h0 + hva * T + hvm * ct + cur.b.z;
                double dmm = fma(gb.x, lP, neg(gb.y * lQ));
                dmm = dmm + dmm;  // 2 gs lambda_P - 2 bs lambda_Q
                if (a1 > a0) {
                    double *Hva = P.hess + h0 + hva * ct + cur.b.y;
                    const int nd = cur.b.w & 0xffff, nlt = cur.b.w >> 16;
                    const uint8_t *code = d.slot_code + __ldg(&I->slot0);
                    // one pass over the slots, sorted by far bus: groups of
                    // parallel arcs are summed, then written in column order
                    double daa = 0.0, dma = 0.0, acc_ma = 0.0, acc_aa = 0.0, acc_mm = 0.0;
                    bool first = true;
                    int grp = 0;
                    for (int a = a0; a < a1; a++) {
                        const unsigned cd = __ldg(code + a);
                        const double2 v1 = __ldg(reinterpret_cast<const double2 *>(S + a) + 1);
                        const double2 v2 = __ldg(reinterpret_cast<const double2 *>(S + a) + 2);
                        daa += v1.x;
                        dma += v1.y;
                        dmm += v2.x;
                        if (first) {
                            acc_ma = neg(v1.y);
                            acc_aa = neg(v1.x);
                            acc_mm = v2.y;
                        } else {
                            acc_ma -= v1.y;
                            acc_aa -= v1.x;
                            acc_mm += v2.y;
                        }
                        first = (cd & SLOT_LAST) != 0;
                        if (first) {
                            Hvm[grp < nlt ? grp : grp + 1] = acc_ma;  // (vm_i, va_j)
                            if (cd & SLOT_LOWER) {
                                Hva[grp] = acc_aa;               // (va_i, va_j), j < i
                                Hvm[nd + 1 + grp] = acc_mm;      // (vm_i, vm_j), j < i
                            }
                            grp++;
                        }
                    }
                    Hva[nlt] = daa;
                    Hvm[nlt] = dma;
                    Hvm[nd + 1 + nlt] = dmm;
                } else {
                    Hvm[0] = dmm;
                }
            }
        } else {
            const int g = ce;
            const int64_t xpg = x0 + 2 * nbT + (int64_t)ng * ct + g;
            const int gg = __ldg(&I->gen0) + g;
            const double pg = __ldg(x + xpg);
            const double c2 = __ldg(d.c2 + gg), c1 = __ldg(d.c1 + gg);
            if (OBJ)
                obj_acc += fma(fma(c2, pg, c1), pg, __ldg(d.c0 + gg));
            if (GRAD) {
                P.grad[xpg] = fma(c2 + c2, pg, c1);
                P.grad[xpg + ngT] = 0.0;
            }
            if (HESS) {
                const int64_t hpg = __ldg(&I->h0) + (__ldg(&I->hva) + __ldg(&I->hvm)) * T;
                P.hess[hpg + (int64_t)ng * ct + g] = P.sigma * (c2 + c2);
            }
            if ((CONS || JAC) && ct >= 1 && __ldg(&I->ramp)) {
                const int64_t q = g + (int64_t)ng * (ct - 1);
                if (CONS)
                    P.c[c0 + T + 7 * nlT + 2 * nbT + q] = pg - __ldg(x + xpg - ng);
                if (JAC) {
                    double *J = P.jac + __ldg(&I->j0) + T + 26 * nlT + 2 * __ldg(&I->jP) * T + 2 * q;
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
            const int4 br = d.br[kb];
            const double2 bf = d.vbnd[I->bus0 + br.x], bt = d.vbnd[I->bus0 + br.y];
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

// launch with programmatic stream serialization (see the file comment)
template <class K>
cudaError_t launch_pdl(K kernel, int grid, int block, cudaStream_t s, const KParams &P)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, P);
}

template <bool C, bool J, bool H>
cudaError_t dispatch(const KParams &P, bool grad, bool obj, bool run_branch, bool run_bus, int gb,
                     int bb, int gu, int bu, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    if (run_branch)
        e = grad ? launch_pdl(branch_kernel<C, J, H, true>, gb, bb, s, P)
                 : launch_pdl(branch_kernel<C, J, H, false>, gb, bb, s, P);
    if (e != cudaSuccess || !run_bus)
        return e;
    if (grad)
        return obj ? launch_pdl(bus_kernel<C, J, H, true, true>, gu, bu, s, P)
                   : launch_pdl(bus_kernel<C, J, H, true, false>, gu, bu, s, P);
    return obj ? launch_pdl(bus_kernel<C, J, H, false, true>, gu, bu, s, P)
               : launch_pdl(bus_kernel<C, J, H, false, false>, gu, bu, s, P);
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
    cudaError_t e;
    switch ((C ? 1 : 0) | (J ? 2 : 0) | (H ? 4 : 0)) {
    case 0: e = dispatch<false, false, false>(P, G, O, run_branch, run_bus, gb, bb, gu, bu, s); break;
    case 1: e = dispatch<true, false, false>(P, G, O, run_branch, run_bus, gb, bb, gu, bu, s); break;
    case 2: e = dispatch<false, true, false>(P, G, O, run_branch, run_bus, gb, bb, gu, bu, s); break;
    case 3: e = dispatch<true, true, false>(P, G, O, run_branch, run_bus, gb, bb, gu, bu, s); break;
    case 4: e = dispatch<false, false, true>(P, G, O, run_branch, run_bus, gb, bb, gu, bu, s); break;
    case 5: e = dispatch<true, false, true>(P, G, O, run_branch, run_bus, gb, bb, gu, bu, s); break;
    case 6: e = dispatch<false, true, true>(P, G, O, run_branch, run_bus, gb, bb, gu, bu, s); break;
    default: e = dispatch<true, true, true>(P, G, O, run_branch, run_bus, gb, bb, gu, bu, s); break;
    }
    if (e == cudaSuccess)
        e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("kernel launch failed: %s", cudaGetErrorString(e));
        return OPF_ECUDA;
    }
    return OPF_OK;
}

// The fused evaluation with caller-chosen scratch (arc slots, objective
// partials, block counter) in place of the model's own; used by
// opf_eval_all_noalloc. Same kernels and launch shape as launch_eval.
int launch_eval_scratch(Model &M, const EvalArgs &a, unsigned what, cudaStream_t s,
                        ArcScratch *arcs, double *obj_part, int max_part, unsigned int *ticket)
{
    KParams P;
    P.d = M.d;
    P.d.arcs = arcs;
    P.d.obj_part = obj_part;
    P.d.ticket = ticket;
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
    const int cap = max_part < M.max_part ? max_part : M.max_part;
    const int gu = grid_for(M.nbus_items + M.ngen_items, L.bus_block, L.bus_ctas_per_sm, M.num_sms, cap);
    const bool run_branch = (C || J || H || G) && M.nbr_items > 0;
    const int bb = L.branch_block, bu = L.bus_block;
    cudaError_t e;
    switch ((C ? 1 : 0) | (J ? 2 : 0) | (H ? 4 : 0)) {
    case 0: e = dispatch<false, false, false>(P, G, O, run_branch, true, gb, bb, gu, bu, s); break;
    case 1: e = dispatch<true, false, false>(P, G, O, run_branch, true, gb, bb, gu, bu, s); break;
    case 2: e = dispatch<false, true, false>(P, G, O, run_branch, true, gb, bb, gu, bu, s); break;
    case 3: e = dispatch<true, true, false>(P, G, O, run_branch, true, gb, bb, gu, bu, s); break;
    case 4: e = dispatch<false, false, true>(P, G, O, run_branch, true, gb, bb, gu, bu, s); break;
    case 5: e = dispatch<true, false, true>(P, G, O, run_branch, true, gb, bb, gu, bu, s); break;
    case 6: e = dispatch<false, true, true>(P, G, O, run_branch, true, gb, bb, gu, bu, s); break;
    default: e = dispatch<true, true, true>(P, G, O, run_branch, true, gb, bb, gu, bu, s); break;
    }
    if (e == cudaSuccess)
        e = cudaGetLastError();
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

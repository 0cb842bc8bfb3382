// k_branch.cuh: the branch-phase kernels (polar and rectangular, one and two threads per branch item)
//
// Part of the translation unit of kernels.cu, which includes it inside
// namespace opf::(anonymous) after k_common.cuh; not a standalone header.

template <bool CONS, bool JAC, bool HESS, bool ONE, bool OCC, bool SETF = false>
__global__ void __launch_bounds__(OCC ? 256 : 512, OCC ? 3 : 1) branch_kernel(const KParams P)
{
    const DevArrays &d = P.d;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    __shared__ double stage[JAC ? 16 : 1][JAC ? 160 : 1];  // per warp: one flow-row group's Jacobian values

    auto locate = [&](int64_t item, int &s, int &t, int &k, int &kb) {
        if (ONE) {
            s = 0;
            split((int)item, P.inst0.nl, P.inst0.T, t, k);
            kb = k;
        } else {
            s = find_inst(d.br_items, P.ninst, item);
            const InstDev *I = d.inst + s;
            split((int)(item - __ldg(d.br_items + s)), __ldg(&I->nl), __ldg(&I->T), t, k);
            kb = __ldg(&I->br0) + k;
        }
    };

    int s = 0, t = 0, k = 0, kb = 0;
    BrStatic st{};
    if (it < P.nbr_items) {  // static prologue, overlaps the previous kernel
        locate(it, s, t, k, kb);
        st = load_br(d, kb, CONS, JAC);
    }
    cudaGridDependencySynchronize();
    cudaTriggerProgrammaticLaunchCompletion();  // the next kernel may launch now

    const int64_t first = it;
    for (; it < P.nbr_items; it += stride) {
        if (OCC && it != first) {  // the low-register build loads each item's static data here
            locate(it, s, t, k, kb);
            st = load_br(d, kb, CONS, JAC);
        }
        const BrStatic cur = st;
        const int cs = s, ct = t, ck = k;
        if (!OCC && it + stride < P.nbr_items) {  // prefetch the next item's static data
            locate(it + stride, s, t, k, kb);
            st = load_br(d, kb, CONS, JAC);
        }
        const InstDev I = inst_of<ONE>(P, cs);
        const int nl = I.nl, nb = I.nb, ng = I.ng, T = I.T;
        const int nbT = nb * T, ngT = ng * T, nlT = nl * T, na = 2 * nl;
        const int rk = ck + nl * ct;  // element index inside each branch group
        const int f = cur.br.x, b = cur.br.y;

        const double *__restrict__ xs = P.x + I.x0;
        const int iva = nb * ct, ivm = nbT + nb * ct;
        const int ip = 2 * nbT + 2 * ngT + na * ct, iq = ip + na * T;
        const double vaf = __ldg(xs + iva + f), vat = __ldg(xs + iva + b);
        const double vmf = __ldg(xs + ivm + f), vmt = __ldg(xs + ivm + b);
        double pf = 0, qf = 0, pt = 0, qt = 0;
        if ((CONS || JAC || HESS) && !SETF) {
            pf = __ldg(xs + ip + ck);
            pt = __ldg(xs + ip + nl + ck);
            qf = __ldg(xs + iq + ck);
            qt = __ldg(xs + iq + nl + ck);
        }
        double m1 = 0, m2 = 0, m3 = 0, m4 = 0, lf = 0, lt = 0;
        if (HESS) {
            const double *L = P.lam + I.c0 + (T + rk);
            m1 = __ldg(L);
            m2 = __ldg(L + nlT);
            m3 = __ldg(L + 2 * nlT);
            m4 = __ldg(L + 3 * nlT);
            lf = __ldg(L + (5 * nlT + 2 * nbT));
            lt = __ldg(L + (6 * nlT + 2 * nbT));
        }
        const double2 Yff = cur.yff, Yft = cur.yft, Ytf = cur.ytf, Ytt = cur.ytt;

        const double dlt = vaf - vat;
        double sn, cs_;
        sincos_tab(dlt, d.trig, &sn, &cs_);
        const double vft = vmf * vmt;
        const double Aft = fma(Yft.x, cs_, Yft.y * sn);
        const double Bft = fma(Yft.x, sn, neg(Yft.y * cs_));
        const double Atf = fma(Ytf.x, cs_, neg(Ytf.y * sn));
        const double Btf = neg(fma(Ytf.x, sn, Ytf.y * cs_));
        if (SETF) {  // p, q := the flows at the voltages (their rows become exactly zero)
            const double vf2 = vmf * vmf, vt2 = vmt * vmt;
            pf = fma(Yff.x, vf2, vft * Aft);
            qf = fma(neg(Yff.y), vf2, vft * Bft);
            pt = fma(Ytt.x, vt2, vft * Atf);
            qt = fma(neg(Ytt.y), vt2, vft * Btf);
            double *xw = P.xw + I.x0;
            xw[ip + ck] = pf;
            xw[ip + nl + ck] = pt;
            xw[iq + ck] = qf;
            xw[iq + nl + ck] = qt;
        }

        if (CONS) {
            const double vf2 = vmf * vmf, vt2 = vmt * vmt;
            double *c = P.c + I.c0 + (T + rk);
            if (SETF) {  // p, q were just set to these flows: the rows are exactly zero
                c[0] = 0.0;
                c[nlT] = 0.0;
                c[2 * nlT] = 0.0;
                c[3 * nlT] = 0.0;
            } else {
                c[0] = pf - fma(Yff.x, vf2, vft * Aft);
                c[nlT] = qf - fma(neg(Yff.y), vf2, vft * Bft);
                c[2 * nlT] = pt - fma(Ytt.x, vt2, vft * Atf);
                c[3 * nlT] = qt - fma(neg(Ytt.y), vt2, vft * Btf);
            }
            c[4 * nlT] = dlt;
            c[5 * nlT + 2 * nbT] = fma(pf, pf, qf * qf) - cur.r2;
            c[6 * nlT + 2 * nbT] = fma(pt, pt, qt * qt) - cur.r2;
        }
        if (JAC) {
            const int jP = (int)I.jP;
            const bool f_lo = f < b;
            const double v2f = twice(vmf), v2t = twice(vmt);
            const double uB = vft * Bft, uA = vft * Aft, wB = vft * Btf, wA = vft * Atf;
            double *J = P.jac + I.j0;
            double *Jf = J + (T + 5 * rk);
            // When the warp's 32 items are consecutive elements of one
            // instance, each flow-row group's 32 x 5 values are contiguous:
            // staged through shared memory and written coalesced (the
            // scattered 8-byte stores took a third of the batched phase)
            const unsigned am = __activemask();
            bool coal = false;
            if (am == 0xffffffffu) {  // every lane takes every shuffle (no short-circuit around them)
                const int lane = threadIdx.x & 31;
                const int rk0 = __shfl_sync(am, rk, 0), s0 = __shfl_sync(am, cs, 0);
                const bool mine = (rk == rk0 + lane) & (cs == s0);
                coal = __all_sync(am, mine);
            }
            if (coal) {
                const int lane = threadIdx.x & 31;
                double *stg = stage[threadIdx.x >> 5];
                double *J0 = Jf - 5 * lane;  // the warp's first row
                put5_warp(stg, J0, lane, f_lo, uB, neg(uB), neg(fma(Yff.x, v2f, vmt * Aft)), neg(vmf * Aft));
                put5_warp(stg, J0 + 5 * nlT, lane, f_lo, neg(uA), uA, fma(Yff.y, v2f, neg(vmt * Bft)),
                          neg(vmf * Bft));
                put5_warp(stg, J0 + 10 * nlT, lane, f_lo, neg(wB), wB, neg(vmt * Atf),
                          neg(fma(Ytt.x, v2t, vmf * Atf)));
                put5_warp(stg, J0 + 15 * nlT, lane, f_lo, wA, neg(wA), neg(vmt * Btf),
                          fma(Ytt.y, v2t, neg(vmf * Btf)));
            } else {
                // row p_fr - P_fr
                put5(Jf, f_lo, uB, neg(uB), neg(fma(Yff.x, v2f, vmt * Aft)), neg(vmf * Aft));
                // row q_fr - Q_fr
                put5(Jf + 5 * nlT, f_lo, neg(uA), uA, fma(Yff.y, v2f, neg(vmt * Bft)), neg(vmf * Bft));
                // row p_to - P_to
                put5(Jf + 10 * nlT, f_lo, neg(wB), wB, neg(vmt * Atf), neg(fma(Ytt.x, v2t, vmf * Atf)));
                // row q_to - Q_to
                put5(Jf + 15 * nlT, f_lo, wA, neg(wA), neg(vmt * Btf), fma(Ytt.y, v2t, neg(vmf * Btf)));
            }
            double *Ja = J + (T + 20 * nlT + 2 * rk);  // angle row va_f - va_t
            Ja[0] = flip(1.0, !f_lo);
            Ja[1] = flip(1.0, f_lo);
            double *Jb = J + (T + 22 * nlT + jP * ct);  // +1 of each arc in its bus's P and Q rows
            Jb[cur.jb.x] = 1.0;
            Jb[cur.jb.y] = 1.0;
            Jb[jP * T + cur.jb.x] = 1.0;
            Jb[jP * T + cur.jb.y] = 1.0;
            double *Jt = J + (T + 22 * nlT + 2 * jP * T + 2 * rk);  // thermal rows
            Jt[0] = twice(pf);
            Jt[1] = twice(qf);
            Jt[2 * nlT] = twice(pt);
            Jt[2 * nlT + 1] = twice(qt);
        }
        if (HESS || CONS) {
            ArcScratch *S = d.arcs + I.scr0 + na * ct;
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
                sf[2] = make_double2(neg(twice(Wf)), neg(U));
                sto[1] = make_double2(vU, vmf * V);
                sto[2] = make_double2(neg(twice(Wt)), neg(U));
                double *Hp = P.hess + I.h0 + ((int)(I.hva + I.hvm) * T + ngT + ck + na * ct);
                const double l2f = twice(lf), l2t = twice(lt);
                Hp[0] = l2f;            // (p_fr, p_fr)
                Hp[nl] = l2t;           // (p_to, p_to)
                Hp[na * T] = l2f;       // (q_fr, q_fr)
                Hp[na * T + nl] = l2t;  // (q_to, q_to)
            }
        }
        if (P.want_grad) {
            double *g = P.grad + I.x0;
            g[ip + ck] = 0.0;
            g[ip + nl + ck] = 0.0;
            g[iq + ck] = 0.0;
            g[iq + nl + ck] = 0.0;
        }
    }
}

// Branch phase with two threads per branch item (branch_occupancy 2, polar
// form): the lanes 2q and 2q + 1 of a warp take the from-end and the to-end
// of item q. Each computes the shared trigonometry and, for its own end,
// the two flow rows with their Jacobian rows, the thermal row and its
// Jacobian and Hessian entries, the balance +1 entries, the arc's scratch
// record and its gradient zeros; the from-end lane also writes the angle
// row. The Hessian's U and V (section above) are sums of one part per end,
// exchanged between the two lanes with one shuffle each and added in the
// same order in both. Every per-end formula is the from-end one with the
// ends swapped: at the to-end the angle is va_t - va_f.
template <bool CONS, bool JAC, bool HESS, bool ONE>
__global__ void __launch_bounds__(512, 1) branch2_kernel(const KParams P)
{
    const DevArrays &d = P.d;
    const int lane = threadIdx.x & 31;
    const int e = lane & 1;                                      // 0: from-end, 1: to-end
    const unsigned pair = 3u << (lane & ~1);                     // this pair's lanes
    const int64_t stride = ((int64_t)gridDim.x * blockDim.x) >> 1;
    int64_t it = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 1;

    auto locate = [&](int64_t item, int &s, int &t, int &k, int &kb) {
        if (ONE) {
            s = 0;
            split((int)item, P.inst0.nl, P.inst0.T, t, k);
            kb = k;
        } else {
            s = find_inst(d.br_items, P.ninst, item);
            const InstDev *I = d.inst + s;
            split((int)(item - __ldg(d.br_items + s)), __ldg(&I->nl), __ldg(&I->T), t, k);
            kb = __ldg(&I->br0) + k;
        }
    };
    int s = 0, t = 0, k = 0, kb = 0;
    int4 br = make_int4(0, 0, 0, 0);
    int jb = 0;
    double2 Yo = make_double2(0.0, 0.0), Yx = make_double2(0.0, 0.0);
    double r2 = 0.0;
    auto load = [&]() {  // this end's static data
        br = __ldg(d.br + kb);
        if (JAC) {
            const int2 j2 = __ldg(d.br_jb + kb);
            jb = e ? j2.y : j2.x;
        }
        Yo = __ldg((e ? d.y_tt : d.y_ff) + kb);
        Yx = __ldg((e ? d.y_tf : d.y_ft) + kb);
        if (CONS)
            r2 = __ldg(d.rate2 + kb);
    };
    if (it < P.nbr_items) {  // static prologue, overlaps the previous kernel
        locate(it, s, t, k, kb);
        load();
    }
    cudaGridDependencySynchronize();
    cudaTriggerProgrammaticLaunchCompletion();  // the next kernel may launch now

    const int64_t first = it;
    for (; it < P.nbr_items; it += stride) {
        if (it != first) {
            locate(it, s, t, k, kb);
            load();
        }
        const InstDev I = inst_of<ONE>(P, s);
        const int nl = I.nl, nb = I.nb, ng = I.ng, T = I.T;
        const int nbT = nb * T, ngT = ng * T, nlT = nl * T, na = 2 * nl;
        const int rk = k + nl * t;
        const int f = br.x, b = br.y;
        const int own = e ? b : f, far = e ? f : b;
        const double *__restrict__ xs = P.x + I.x0;
        const int iva = nb * t, ivm = nbT + nb * t;
        const int ip = 2 * nbT + 2 * ngT + na * t, iq = ip + na * T;
        const int arc = e ? nl + k : k;  // this end's arc
        const double vao = __ldg(xs + iva + own), vax = __ldg(xs + iva + far);
        const double vo = __ldg(xs + ivm + own), vx = __ldg(xs + ivm + far);
        double po = 0, qo = 0;
        if (CONS || JAC || HESS) {
            po = __ldg(xs + ip + arc);
            qo = __ldg(xs + iq + arc);
        }
        double mP = 0, mQ = 0, lth = 0;
        if (HESS) {
            const double *L = P.lam + I.c0 + (T + rk);
            mP = __ldg(L + (e ? 2 * nlT : 0));
            mQ = __ldg(L + (e ? 3 * nlT : nlT));
            lth = __ldg(L + ((e ? 6 : 5) * nlT + 2 * nbT));
        }
        const double dlt = vao - vax;  // this end's angle
        double sn, cs_;
        sincos_tab(dlt, d.trig, &sn, &cs_);
        const double vft = vo * vx;
        const double A = fma(Yx.x, cs_, Yx.y * sn);
        const double B = fma(Yx.x, sn, neg(Yx.y * cs_));
        if (CONS) {
            const double vo2 = vo * vo;
            double *c = P.c + I.c0 + (T + rk);
            c[e ? 2 * nlT : 0] = po - fma(Yo.x, vo2, vft * A);
            c[e ? 3 * nlT : nlT] = qo - fma(neg(Yo.y), vo2, vft * B);
            if (!e)
                c[4 * nlT] = dlt;
            c[(e ? 6 : 5) * nlT + 2 * nbT] = fma(po, po, qo * qo) - r2;
        }
        if (JAC) {
            const int jP = (int)I.jP;
            const bool o_lo = own < far;
            const double v2o = twice(vo);
            const double uB = vft * B, uA = vft * A;
            double *J = P.jac + I.j0;
            double *Jf = J + (T + 5 * rk + (e ? 10 * nlT : 0));
            // (va_own, va_far, vm_own, vm_far) of p - P and q - Q at this end
            put5(Jf, o_lo, uB, neg(uB), neg(fma(Yo.x, v2o, vx * A)), neg(vo * A));
            put5(Jf + 5 * nlT, o_lo, neg(uA), uA, fma(Yo.y, v2o, neg(vx * B)), neg(vo * B));
            if (!e) {  // angle row va_f - va_t
                double *Ja = J + (T + 20 * nlT + 2 * rk);
                Ja[0] = flip(1.0, !o_lo);
                Ja[1] = flip(1.0, o_lo);
            }
            double *Jb = J + (T + 22 * nlT + jP * t);  // +1 of the arc in its bus's P and Q rows
            Jb[jb] = 1.0;
            Jb[jP * T + jb] = 1.0;
            double *Jt = J + (T + 22 * nlT + 2 * jP * T + 2 * rk + (e ? 2 * nlT : 0));  // thermal row
            Jt[0] = twice(po);
            Jt[1] = twice(qo);
        }
        if (HESS || CONS) {
            ArcScratch *S = d.arcs + I.scr0 + na * t;
            double2 *so = reinterpret_cast<double2 *>(S + (e ? br.w : br.z));
            so[0] = make_double2(po, qo);
            if (HESS) {
                // U = (m1 Aft + m2 Bft) + (m3 Atf + m4 Btf), V = (m2 Aft - m1 Bft) + (m3 Btf - m4 Atf)
                const double Ue = fma(mP, A, mQ * B);
                const double Ve = flip(fma(mQ, A, neg(mP * B)), e);
                const double Uo = __shfl_xor_sync(pair, Ue, 1), Vo = __shfl_xor_sync(pair, Ve, 1);
                const double U = e ? Uo + Ue : Ue + Uo;  // from-end part first in both lanes
                const double V = e ? Vo + Ve : Ve + Vo;
                const double We = fma(mP, Yo.x, neg(mQ * Yo.y));
                so[1] = make_double2(vft * U, flip(vx * V, !e));
                so[2] = make_double2(neg(twice(We)), neg(U));
                double *Hp = P.hess + I.h0 + ((int)(I.hva + I.hvm) * T + ngT + arc + na * t);
                const double l2 = twice(lth);
                Hp[0] = l2;       // (p_arc, p_arc)
                Hp[na * T] = l2;  // (q_arc, q_arc)
            }
        }
        if (P.want_grad) {
            P.grad[I.x0 + ip + arc] = 0.0;
            P.grad[I.x0 + iq + arc] = 0.0;
        }
    }
}

// gradient of a rectangular row in the order (vr_f, vr_t, vi_f, vi_t)
struct Grad4 {
    double rf, rt, jf, jt;
};

// the Jacobian entries of a rectangular row, columns ascending:
// (vr_lo, vr_hi, vi_lo, vi_hi), then the own flow variable if `own`
__device__ __forceinline__ void put_rect(double *J, bool f_lo, const Grad4 &g, bool own)
{
    J[0] = f_lo ? g.rf : g.rt;
    J[1] = f_lo ? g.rt : g.rf;
    J[2] = f_lo ? g.jf : g.jt;
    J[3] = f_lo ? g.jt : g.jf;
    if (own)
        J[4] = 1.0;
}

// Branch phase of the rectangular form: the same items, rows and scratch
// slots as the polar branch kernel, without trigonometry. Row groups per
// instance: ref, four flow groups, upper angle rows, P and Q balance, two
// thermal groups, lower angle rows, magnitude rows, ramp rows.
template <bool CONS, bool JAC, bool HESS, bool ONE, bool OCC>
__global__ void __launch_bounds__(OCC ? 256 : 512, OCC ? 3 : 1) rect_branch_kernel(const KParams P)
{
    const DevArrays &d = P.d;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    __shared__ double stage[JAC ? 16 : 1][JAC ? 160 : 1];  // per warp: one flow-row group's Jacobian values

    auto locate = [&](int64_t item, int &s, int &t, int &k, int &kb) {
        if (ONE) {
            s = 0;
            split((int)item, P.inst0.nl, P.inst0.T, t, k);
            kb = k;
        } else {
            s = find_inst(d.br_items, P.ninst, item);
            const InstDev *I = d.inst + s;
            split((int)(item - __ldg(d.br_items + s)), __ldg(&I->nl), __ldg(&I->T), t, k);
            kb = __ldg(&I->br0) + k;
        }
    };

    int s = 0, t = 0, k = 0, kb = 0;
    BrStatic st{};
    double2 tb = make_double2(0.0, 0.0);
    if (it < P.nbr_items) {  // static prologue, overlaps the previous kernel
        locate(it, s, t, k, kb);
        st = load_br(d, kb, CONS, JAC);
        tb = __ldg(d.tanb + kb);
    }
    cudaGridDependencySynchronize();
    cudaTriggerProgrammaticLaunchCompletion();  // the next kernel may launch now

    const int64_t first = it;
    for (; it < P.nbr_items; it += stride) {
        if (OCC && it != first) {  // the low-register build loads each item's static data here
            locate(it, s, t, k, kb);
            st = load_br(d, kb, CONS, JAC);
            tb = __ldg(d.tanb + kb);
        }
        const BrStatic cur = st;
        const double2 tan_ = tb;
        const int cs = s, ct = t, ck = k;
        if (!OCC && it + stride < P.nbr_items) {  // prefetch the next item's static data
            locate(it + stride, s, t, k, kb);
            st = load_br(d, kb, CONS, JAC);
            tb = __ldg(d.tanb + kb);
        }
        const InstDev I = inst_of<ONE>(P, cs);
        const int nl = I.nl, nb = I.nb, ng = I.ng, T = I.T;
        const int nbT = nb * T, ngT = ng * T, nlT = nl * T, na = 2 * nl;
        const int rk = ck + nl * ct;
        const int f = cur.br.x, b = cur.br.y;

        const double *__restrict__ xs = P.x + I.x0;
        const int ivr = nb * ct, ivi = nbT + nb * ct;
        const int ip = 2 * nbT + 2 * ngT + na * ct, iq = ip + na * T;
        const double vrf = __ldg(xs + ivr + f), vrt = __ldg(xs + ivr + b);
        const double vif = __ldg(xs + ivi + f), vit = __ldg(xs + ivi + b);
        double pf = 0, qf = 0, pt = 0, qt = 0;
        if (CONS || JAC || HESS) {
            pf = __ldg(xs + ip + ck);
            pt = __ldg(xs + ip + nl + ck);
            qf = __ldg(xs + iq + ck);
            qt = __ldg(xs + iq + nl + ck);
        }
        double m1 = 0, m2 = 0, m3 = 0, m4 = 0, a1 = 0, a2 = 0, lf = 0, lt = 0;
        if (HESS) {
            const double *L = P.lam + I.c0 + (T + rk);
            m1 = __ldg(L);
            m2 = __ldg(L + nlT);
            m3 = __ldg(L + 2 * nlT);
            m4 = __ldg(L + 3 * nlT);
            a1 = __ldg(L + 4 * nlT);
            lf = __ldg(L + (5 * nlT + 2 * nbT));
            lt = __ldg(L + (6 * nlT + 2 * nbT));
            a2 = __ldg(L + (7 * nlT + 2 * nbT));
        }
        const double2 Yff = cur.yff, Yft = cur.yft, Ytf = cur.ytf, Ytt = cur.ytt;
        const double wR = fma(vrf, vrt, vif * vit);
        const double wI = fma(vif, vrt, neg(vrf * vit));

        if (CONS) {
            const double vf2 = fma(vrf, vrf, vif * vif), vt2 = fma(vrt, vrt, vit * vit);
            double *c = P.c + I.c0 + (T + rk);
            c[0] = pf - fma(Yff.x, vf2, fma(Yft.x, wR, Yft.y * wI));
            c[nlT] = qf - fma(neg(Yff.y), vf2, fma(Yft.x, wI, neg(Yft.y * wR)));
            c[2 * nlT] = pt - fma(Ytt.x, vt2, fma(Ytf.x, wR, neg(Ytf.y * wI)));
            c[3 * nlT] = qt - fma(neg(Ytt.y), vt2, neg(fma(Ytf.x, wI, Ytf.y * wR)));
            c[4 * nlT] = fma(neg(tan_.x), wR, wI);
            c[5 * nlT + 2 * nbT] = fma(pf, pf, qf * qf) - cur.r2;
            c[6 * nlT + 2 * nbT] = fma(pt, pt, qt * qt) - cur.r2;
            c[7 * nlT + 2 * nbT] = fma(neg(tan_.y), wR, wI);
        }
        if (JAC) {
            const int jP = (int)I.jP;
            const bool f_lo = f < b;
            double *J = P.jac + I.j0;
            double *Jf = J + (T + 5 * rk);
            // With z = c + j d the (c, d) part of a row's gradient is
            // (vr_f, vi_f) <- z V_t and (vr_t, -vi_t) <- z conj(V_f). The
            // rows p_fr - P_fr and q_fr - Q_fr have z = -Yft and -j Yft, the
            // rows p_to - P_to and q_to - Q_to z = -conj(Ytf) and j conj(Ytf):
            // two complex products per end serve both of its rows.
            const double y1r = fma(Yft.x, vrt, neg(Yft.y * vit)), y1i = fma(Yft.x, vit, Yft.y * vrt);  // Yft V_t
            const double y2r = fma(Yft.x, vrf, Yft.y * vif), y2i = fma(Yft.y, vrf, neg(Yft.x * vif));  // Yft conj(V_f)
            const double z1r = fma(Ytf.x, vrt, Ytf.y * vit), z1i = fma(Ytf.x, vit, neg(Ytf.y * vrt));  // conj(Ytf) V_t
            const double z2r = fma(Ytf.x, vrf, neg(Ytf.y * vif));                                     // conj(Ytf V_f)
            const double z2i = neg(fma(Ytf.x, vif, Ytf.y * vrf));
            const double pa = neg(twice(Yff.x)), qa = twice(Yff.y);  // the from-end's own |V_f|^2 terms
            const double pb = neg(twice(Ytt.x)), qb = twice(Ytt.y);
            // the four flow rows, staged per warp and written coalesced when
            // the warp's items are consecutive rows of one instance (as in
            // the polar branch kernel; every lane takes every shuffle)
            const unsigned am = __activemask();
            bool coal = false;
            if (am == 0xffffffffu) {
                const int lane = threadIdx.x & 31;
                const int rk0 = __shfl_sync(am, rk, 0), s0 = __shfl_sync(am, cs, 0);
                const bool mine = (rk == rk0 + lane) & (cs == s0);
                coal = __all_sync(am, mine);
            }
            const int lane = threadIdx.x & 31;
            double *J0 = Jf - 5 * lane;
            double *stg = stage[threadIdx.x >> 5];
            Grad4 g;
            g.rf = fma(pa, vrf, neg(y1r)); g.jf = fma(pa, vif, neg(y1i)); g.rt = neg(y2r); g.jt = y2i;
            if (coal)  // p_fr - P_fr
                put5_warp(stg, J0, lane, f_lo, g.rf, g.rt, g.jf, g.jt);
            else
                put_rect(Jf, f_lo, g, true);
            g.rf = fma(qa, vrf, y1i); g.jf = fma(qa, vif, neg(y1r)); g.rt = y2i; g.jt = y2r;
            if (coal)  // q_fr - Q_fr
                put5_warp(stg, J0 + 5 * nlT, lane, f_lo, g.rf, g.rt, g.jf, g.jt);
            else
                put_rect(Jf + 5 * nlT, f_lo, g, true);
            g.rf = neg(z1r); g.jf = neg(z1i); g.rt = fma(pb, vrt, neg(z2r)); g.jt = fma(pb, vit, z2i);
            if (coal)  // p_to - P_to
                put5_warp(stg, J0 + 10 * nlT, lane, f_lo, g.rf, g.rt, g.jf, g.jt);
            else
                put_rect(Jf + 10 * nlT, f_lo, g, true);
            g.rf = neg(z1i); g.jf = z1r; g.rt = fma(qb, vrt, neg(z2i)); g.jt = fma(qb, vit, neg(z2r));
            if (coal)  // q_to - Q_to
                put5_warp(stg, J0 + 15 * nlT, lane, f_lo, g.rf, g.rt, g.jf, g.jt);
            else
                put_rect(Jf + 15 * nlT, f_lo, g, true);
            // angle rows, z = -tan(limit) + j: one FMA per entry
            const double tu = neg(tan_.x), tl = neg(tan_.y);
            g.rf = fma(tu, vrt, neg(vit)); g.jf = fma(tu, vit, vrt); g.rt = fma(tu, vrf, vif); g.jt = fma(tu, vif, neg(vrf));
            put_rect(J + (T + 20 * nlT + 4 * rk), f_lo, g, false);
            g.rf = fma(tl, vrt, neg(vit)); g.jf = fma(tl, vit, vrt); g.rt = fma(tl, vrf, vif); g.jt = fma(tl, vif, neg(vrf));
            put_rect(J + (T + 28 * nlT + 2 * jP * T + 4 * rk), f_lo, g, false);
            double *Jb = J + (T + 24 * nlT + jP * ct);  // +1 of each arc in its bus's P and Q rows
            Jb[cur.jb.x] = 1.0;
            Jb[cur.jb.y] = 1.0;
            Jb[jP * T + cur.jb.x] = 1.0;
            Jb[jP * T + cur.jb.y] = 1.0;
            double *Jt = J + (T + 24 * nlT + 2 * jP * T + 2 * rk);  // thermal rows
            Jt[0] = twice(pf);
            Jt[1] = twice(qf);
            Jt[2 * nlT] = twice(pt);
            Jt[2 * nlT + 1] = twice(qt);
        }
        if (HESS || CONS) {
            ArcScratch *S = d.arcs + I.scr0 + na * ct;
            double2 *sf = reinterpret_cast<double2 *>(S + cur.br.z);
            double2 *sto = reinterpret_cast<double2 *>(S + cur.br.w);
            sf[0] = make_double2(pf, qf);
            sto[0] = make_double2(pt, qt);
            if (HESS) {
                // aR = -m1 Gft + m2 Bft - m3 Gtf + m4 Btf - a1 tan(angmax) - a2 tan(angmin)
                // aI = -m1 Bft - m2 Gft + m3 Btf + m4 Gtf + a1 + a2
                const double aR = neg(fma(m1, Yft.x, fma(neg(m2), Yft.y, fma(m3, Ytf.x,
                                  fma(neg(m4), Ytf.y, fma(a1, tan_.x, a2 * tan_.y))))));
                const double aI = fma(neg(m1), Yft.y, fma(neg(m2), Yft.x, fma(m3, Ytf.y, fma(m4, Ytf.x, a1 + a2))));
                const double Df = neg(twice(fma(m1, Yff.x, neg(m2 * Yff.y))));
                const double Dt = neg(twice(fma(m3, Ytt.x, neg(m4 * Ytt.y))));
                sf[1] = make_double2(Df, aR);
                sto[1] = make_double2(Dt, aR);
                reinterpret_cast<double *>(sf + 2)[0] = aI;
                reinterpret_cast<double *>(sto + 2)[0] = neg(aI);
                double *Hp = P.hess + I.h0 + ((int)(I.hva + I.hvm) * T + ngT + ck + na * ct);
                const double l2f = twice(lf), l2t = twice(lt);
                Hp[0] = l2f;            // (p_fr, p_fr)
                Hp[nl] = l2t;           // (p_to, p_to)
                Hp[na * T] = l2f;       // (q_fr, q_fr)
                Hp[na * T + nl] = l2t;  // (q_to, q_to)
            }
        }
        if (P.want_grad) {
            double *g = P.grad + I.x0;
            g[ip + ck] = 0.0;
            g[ip + nl + ck] = 0.0;
            g[iq + ck] = 0.0;
            g[iq + nl + ck] = 0.0;
        }
    }
}

// Branch phase of the rectangular form with two threads per branch item
// (branch_occupancy 2): lanes 2q and 2q + 1 take the from-end and the to-end
// of item q, as in the polar two-lane kernel. With the ends swapped,
// w' = V_t conj(V_f) = conj(w), and the to-end's flows P_to = Gtt |V_t|^2 +
// Gtf wR' + Btf wI', Q_to = -Btt |V_t|^2 + Gtf wI' - Btf wR' take the
// from-end's form with (Ytt, Ytf) for (Yff, Yft): each lane evaluates the
// from-end formulas on (own, far) = (f, t) or (t, f). The from-end lane writes
// the upper angle row, the to-end lane the lower one. The Hessian's aR and aI
// are sums of one part per end (plus the angle rows' parts), exchanged with
// one shuffle each and added from-end part first in both lanes.
template <bool CONS, bool JAC, bool HESS, bool ONE>
__global__ void __launch_bounds__(512, 1) rect_branch2_kernel(const KParams P)
{
    const DevArrays &d = P.d;
    const int lane = threadIdx.x & 31;
    const int e = lane & 1;                   // 0: from-end, 1: to-end
    const unsigned pair = 3u << (lane & ~1);  // this pair's lanes
    const int64_t stride = ((int64_t)gridDim.x * blockDim.x) >> 1;
    int64_t it = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 1;

    auto locate = [&](int64_t item, int &s, int &t, int &k, int &kb) {
        if (ONE) {
            s = 0;
            split((int)item, P.inst0.nl, P.inst0.T, t, k);
            kb = k;
        } else {
            s = find_inst(d.br_items, P.ninst, item);
            const InstDev *I = d.inst + s;
            split((int)(item - __ldg(d.br_items + s)), __ldg(&I->nl), __ldg(&I->T), t, k);
            kb = __ldg(&I->br0) + k;
        }
    };
    int s = 0, t = 0, k = 0, kb = 0;
    int4 br = make_int4(0, 0, 0, 0);
    int jb = 0;
    double2 Yo = make_double2(0.0, 0.0), Yx = make_double2(0.0, 0.0);
    double r2 = 0.0, tn = 0.0;
    auto load = [&]() {  // this end's static data
        br = __ldg(d.br + kb);
        if (JAC) {
            const int2 j2 = __ldg(d.br_jb + kb);
            jb = e ? j2.y : j2.x;
        }
        Yo = __ldg((e ? d.y_tt : d.y_ff) + kb);
        Yx = __ldg((e ? d.y_tf : d.y_ft) + kb);
        if (CONS)
            r2 = __ldg(d.rate2 + kb);
        const double2 tb = __ldg(d.tanb + kb);  // tan(angmax), tan(angmin)
        tn = e ? tb.y : tb.x;
    };
    if (it < P.nbr_items) {  // static prologue, overlaps the previous kernel
        locate(it, s, t, k, kb);
        load();
    }
    cudaGridDependencySynchronize();
    cudaTriggerProgrammaticLaunchCompletion();  // the next kernel may launch now

    const int64_t first = it;
    for (; it < P.nbr_items; it += stride) {
        if (it != first) {
            locate(it, s, t, k, kb);
            load();
        }
        const InstDev I = inst_of<ONE>(P, s);
        const int nl = I.nl, nb = I.nb, ng = I.ng, T = I.T;
        const int nbT = nb * T, ngT = ng * T, nlT = nl * T, na = 2 * nl;
        const int rk = k + nl * t;
        const int f = br.x, b = br.y;
        const int own = e ? b : f, far = e ? f : b;
        const double *__restrict__ xs = P.x + I.x0;
        const int ivr = nb * t, ivi = nbT + nb * t;
        const int ip = 2 * nbT + 2 * ngT + na * t, iq = ip + na * T;
        const int arc = e ? nl + k : k;  // this end's arc
        const double vro = __ldg(xs + ivr + own), vrx = __ldg(xs + ivr + far);
        const double vio = __ldg(xs + ivi + own), vix = __ldg(xs + ivi + far);
        double po = 0, qo = 0;
        if (CONS || JAC || HESS) {
            po = __ldg(xs + ip + arc);
            qo = __ldg(xs + iq + arc);
        }
        double mP = 0, mQ = 0, ma = 0, lth = 0;
        if (HESS) {
            const double *L = P.lam + I.c0 + (T + rk);
            mP = __ldg(L + (e ? 2 * nlT : 0));
            mQ = __ldg(L + (e ? 3 * nlT : nlT));
            ma = __ldg(L + (e ? 7 * nlT + 2 * nbT : 4 * nlT));  // this lane's angle row
            lth = __ldg(L + ((e ? 6 : 5) * nlT + 2 * nbT));
        }
        // w_e = V_own conj(V_far): w at the from-end, conj(w) at the to-end
        const double wR = fma(vro, vrx, vio * vix);
        const double wI = fma(vio, vrx, neg(vro * vix));
        if (CONS) {
            const double vo2 = fma(vro, vro, vio * vio);
            double *c = P.c + I.c0 + (T + rk);
            c[e ? 2 * nlT : 0] = po - fma(Yo.x, vo2, fma(Yx.x, wR, Yx.y * wI));
            c[e ? 3 * nlT : nlT] = qo - fma(neg(Yo.y), vo2, fma(Yx.x, wI, neg(Yx.y * wR)));
            // angle rows on the from-end's w: wI - tan(limit) wR
            c[e ? 7 * nlT + 2 * nbT : 4 * nlT] = fma(neg(tn), wR, flip(wI, e));
            c[(e ? 6 : 5) * nlT + 2 * nbT] = fma(po, po, qo * qo) - r2;
        }
        if (JAC) {
            const int jP = (int)I.jP;
            const bool o_lo = own < far;
            double *J = P.jac + I.j0;
            double *Jf = J + (T + 5 * rk + (e ? 10 * nlT : 0));
            // the from-end's products with (own, far) for (f, t):
            // Yx V_far and Yx conj(V_own)
            const double y1r = fma(Yx.x, vrx, neg(Yx.y * vix)), y1i = fma(Yx.x, vix, Yx.y * vrx);
            const double y2r = fma(Yx.x, vro, Yx.y * vio), y2i = fma(Yx.y, vro, neg(Yx.x * vio));
            const double pa = neg(twice(Yo.x)), qa = twice(Yo.y);
            Grad4 g;  // (own, far) in the places of (f, t)
            g.rf = fma(pa, vro, neg(y1r)); g.jf = fma(pa, vio, neg(y1i)); g.rt = neg(y2r); g.jt = y2i;
            put_rect(Jf, o_lo, g, true);            // p - P at this end
            g.rf = fma(qa, vro, y1i); g.jf = fma(qa, vio, neg(y1r)); g.rt = y2i; g.jt = y2r;
            put_rect(Jf + 5 * nlT, o_lo, g, true);  // q - Q at this end
            // this lane's angle row wI - tn wR, from-end w: its gradient in
            // (vr_f, vr_t, vi_f, vi_t) is (tu vr_t - vi_t, tu vr_f + vi_f,
            // tu vi_t + vr_t, tu vi_f - vr_f) with tu = -tn
            const double tu = neg(tn);
            const double vrf = e ? vrx : vro, vrt = e ? vro : vrx, vif = e ? vix : vio, vit = e ? vio : vix;
            g.rf = fma(tu, vrt, neg(vit)); g.jf = fma(tu, vit, vrt); g.rt = fma(tu, vrf, vif); g.jt = fma(tu, vif, neg(vrf));
            put_rect(J + (T + (e ? 28 * nlT + 2 * jP * T : 20 * nlT) + 4 * rk), f < b, g, false);
            double *Jb = J + (T + 24 * nlT + jP * t);  // +1 of the arc in its bus's P and Q rows
            Jb[jb] = 1.0;
            Jb[jP * T + jb] = 1.0;
            double *Jt = J + (T + 24 * nlT + 2 * jP * T + 2 * rk + (e ? 2 * nlT : 0));  // thermal row
            Jt[0] = twice(po);
            Jt[1] = twice(qo);
        }
        if (HESS || CONS) {
            ArcScratch *S = d.arcs + I.scr0 + na * t;
            double2 *so = reinterpret_cast<double2 *>(S + (e ? br.w : br.z));
            so[0] = make_double2(po, qo);
            if (HESS) {
                // aR = -(m1 Gft - m2 Bft + a1 tan(angmax)) - (m3 Gtf - m4 Btf + a2 tan(angmin))
                // aI = (-m1 Bft - m2 Gft + a1) + (m3 Btf + m4 Gtf + a2)
                const double Re = neg(fma(mP, Yx.x, fma(neg(mQ), Yx.y, ma * tn)));
                const double Ie = flip(fma(mP, Yx.y, mQ * Yx.x), !e) + ma;
                const double Ro = __shfl_xor_sync(pair, Re, 1), Io = __shfl_xor_sync(pair, Ie, 1);
                const double aR = e ? Ro + Re : Re + Ro;  // from-end part first in both lanes
                const double aI = e ? Io + Ie : Ie + Io;
                const double De = neg(twice(fma(mP, Yo.x, neg(mQ * Yo.y))));
                so[1] = make_double2(De, aR);
                reinterpret_cast<double *>(so + 2)[0] = flip(aI, e);
                double *Hp = P.hess + I.h0 + ((int)(I.hva + I.hvm) * T + ngT + arc + na * t);
                const double l2 = twice(lth);
                Hp[0] = l2;       // (p_arc, p_arc)
                Hp[na * T] = l2;  // (q_arc, q_arc)
            }
        }
        if (P.want_grad) {
            P.grad[I.x0 + ip + arc] = 0.0;
            P.grad[I.x0 + iq + arc] = 0.0;
        }
    }
}

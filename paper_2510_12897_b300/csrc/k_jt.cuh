// k_jt.cuh: J^T v (two-phase and fused) and the augmented Lagrangian's one-kernel gradient
//
// Part of the translation unit of kernels.cu, which includes it inside
// namespace opf::(anonymous) after k_bus.cuh; not a standalone header.

// ---------------------------------------------------------------- J^T v --

// entry i of the vector v of J^T v: the given v, or (AL) the augmented
// Lagrangian's multiplier estimate mu_i computed from the row's value
template <bool AL>
__device__ __forceinline__ double vrow(const KParams &P, int64_t i)
{
    if (!AL)
        return __ldg(P.lam + i);
    const double s = fma(__ldg(P.lam + i), P.inv_rho, __ldg(P.c + i));
    return P.rho * (s - fmin(fmax(s, __ldg(P.gl + i)), __ldg(P.gu + i)));
}
//
// out = J^T v, term by term (no Jacobian stored). Branch phase: the flow,
// angle and thermal rows of a branch give the p, q entries of its two arcs
// completely (with the +v of the arcs' balance rows) and their va, vm parts
// for the end buses, stored in the first 16 bytes of the arc's scratch
// record. Bus phase: va_i, vm_i sum their slots in a fixed order and add the
// reference and balance-row terms; generator items take their balance,
// ramp and linking rows.

template <bool ONE, bool RECT = false, bool AL = false>
__global__ void __launch_bounds__(512) jt_branch_kernel(const KParams P)
{
    const DevArrays &d = P.d;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int s = 0, t = 0, k = 0, kb = 0;
    BrStatic st{};
    auto locate = [&](int64_t item) {
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
    if (it < P.nbr_items) {
        locate(it);
        st = load_br(d, kb, false, false);
    }
    cudaGridDependencySynchronize();
    cudaTriggerProgrammaticLaunchCompletion();  // the next kernel may launch now
    for (; it < P.nbr_items; it += stride) {
        const BrStatic cur = st;
        const int cs = s, ct = t, ck = k;
        if (it + stride < P.nbr_items) {
            locate(it + stride);
            st = load_br(d, kb, false, false);
        }
        const InstDev I = inst_of<ONE>(P, cs);
        const int nl = I.nl, nb = I.nb, ng = I.ng, T = I.T;
        const int nbT = nb * T, ngT = ng * T, nlT = nl * T, na = 2 * nl;
        const int rk = ck + nl * ct;
        const int f = cur.br.x, b = cur.br.y;
        const double *__restrict__ xs = P.x + I.x0;
        const int iva = nb * ct, ivm = nbT + nb * ct;
        const int ip = 2 * nbT + 2 * ngT + na * ct, iq = ip + na * T;
        const double vaf = __ldg(xs + iva + f), vat = __ldg(xs + iva + b);
        const double vmf = __ldg(xs + ivm + f), vmt = __ldg(xs + ivm + b);
        const double pf = __ldg(xs + ip + ck), pt = __ldg(xs + ip + nl + ck);
        const double qf = __ldg(xs + iq + ck), qt = __ldg(xs + iq + nl + ck);
        const int64_t V = I.c0 + (T + rk);  // the vector v, indexed like the rows
        const double m1 = vrow<AL>(P, V), m2 = vrow<AL>(P, V + nlT), m3 = vrow<AL>(P, V + 2 * nlT),
                     m4 = vrow<AL>(P, V + 3 * nlT);
        const double va_ = vrow<AL>(P, V + 4 * nlT);
        const double tf = vrow<AL>(P, V + (5 * nlT + 2 * nbT)), tt = vrow<AL>(P, V + (6 * nlT + 2 * nbT));
        const int64_t VB = I.c0 + (T + 5 * nlT + nb * ct);  // balance rows, period ct
        const double bPf = vrow<AL>(P, VB + f), bPt = vrow<AL>(P, VB + b);
        const double bQf = vrow<AL>(P, VB + nbT + f), bQt = vrow<AL>(P, VB + nbT + b);
        const double2 Yff = cur.yff, Yft = cur.yft, Ytf = cur.ytf, Ytt = cur.ytt;
        double *o = P.grad + I.x0;  // P.grad carries `out`
        if constexpr (RECT) {
            // vr = the first block (vaf, vat), vi = the second (vmf, vmt);
            // v^T g over the branch's rows has the voltage part
            // (Df/2)|V_f|^2 + (Dt/2)|V_t|^2 + aR wR + aI wI (angle rows: v at
            // the upper row's and the lower row's places)
            const double a1 = va_;
            const double a2 = vrow<AL>(P, V + (7 * nlT + 2 * nbT));
            const double2 tn = __ldg(d.tanb + (I.br0 + ck));
            const double aR = neg(fma(m1, Yft.x, fma(neg(m2), Yft.y, fma(m3, Ytf.x,
                              fma(neg(m4), Ytf.y, fma(a1, tn.x, a2 * tn.y))))));
            const double aI = fma(neg(m1), Yft.y, fma(neg(m2), Yft.x, fma(m3, Ytf.y, fma(m4, Ytf.x, a1 + a2))));
            const double Df = neg(twice(fma(m1, Yff.x, neg(m2 * Yff.y))));
            const double Dt = neg(twice(fma(m3, Ytt.x, neg(m4 * Ytt.y))));
            o[ip + ck] = fma(twice(pf), tf, m1 + bPf);
            o[iq + ck] = fma(twice(qf), tf, m2 + bQf);
            o[ip + nl + ck] = fma(twice(pt), tt, m3 + bPt);
            o[iq + nl + ck] = fma(twice(qt), tt, m4 + bQt);
            const double drf = fma(Df, vaf, fma(aR, vat, neg(aI * vmt)));
            const double dif = fma(Df, vmf, fma(aR, vmt, aI * vat));
            const double drt = fma(Dt, vat, fma(aR, vaf, aI * vmf));
            const double dit = fma(Dt, vmt, fma(aR, vmf, neg(aI * vaf)));
            ArcScratch *S = d.arcs + I.scr0 + na * ct;
            reinterpret_cast<double2 *>(S + cur.br.z)[0] = make_double2(drf, dif);
            reinterpret_cast<double2 *>(S + cur.br.w)[0] = make_double2(drt, dit);
            continue;
        }
        double sn, cs_;
        sincos_tab(vaf - vat, d.trig, &sn, &cs_);
        const double vft = vmf * vmt;
        const double Aft = fma(Yft.x, cs_, Yft.y * sn);
        const double Bft = fma(Yft.x, sn, neg(Yft.y * cs_));
        const double Atf = fma(Ytf.x, cs_, neg(Ytf.y * sn));
        const double Btf = neg(fma(Ytf.x, sn, Ytf.y * cs_));
        // own variables: flow row, thermal row, balance row of the arc's bus
        o[ip + ck] = fma(twice(pf), tf, m1 + bPf);
        o[iq + ck] = fma(twice(qf), tf, m2 + bQf);
        o[ip + nl + ck] = fma(twice(pt), tt, m3 + bPt);
        o[iq + nl + ck] = fma(twice(qt), tt, m4 + bQt);
        // va: the flow rows' angle derivatives are +-vft (B_ft, A_ft, B_tf,
        // A_tf); the to-end gets exactly the negation of the from-end
        const double dva = fma(m1, Bft, fma(neg(m2), Aft, fma(neg(m3), Btf, m4 * Atf)));
        const double dva_f = fma(vft, dva, va_);
        // vm
        const double v2f = twice(vmf), v2t = twice(vmt);
        const double dvm_f = fma(neg(m1), fma(Yff.x, v2f, vmt * Aft),
                             fma(m2, fma(Yff.y, v2f, neg(vmt * Bft)),
                                 neg(vmt * fma(m3, Atf, m4 * Btf))));
        const double dvm_t = fma(neg(m3), fma(Ytt.x, v2t, vmf * Atf),
                             fma(m4, fma(Ytt.y, v2t, neg(vmf * Btf)),
                                 neg(vmf * fma(m1, Aft, m2 * Bft))));
        ArcScratch *S = d.arcs + I.scr0 + na * ct;
        reinterpret_cast<double2 *>(S + cur.br.z)[0] = make_double2(dva_f, dvm_f);
        reinterpret_cast<double2 *>(S + cur.br.w)[0] = make_double2(neg(dva_f), dvm_t);
    }
}

// J^T v at one (instance, period, generator): its balance, ramp, linking
// and reserve rows
template <bool RECT, bool AL>
__device__ __forceinline__ void jt_gen_item(const KParams &P, const InstDev &I, int s, int t, int g)
{
    const DevArrays &d = P.d;
    const int nl = I.nl, nb = I.nb, ng = I.ng, T = I.T;
    const int nbT = nb * T, ngT = ng * T, nlT = nl * T;
    const int64_t V = I.c0;  // the vector v, indexed like the rows
    double *o = P.grad + I.x0;
    const int bus = __ldg(d.gen_busid + I.gen0 + g);
    double vpg = neg(vrow<AL>(P, V + (T + 5 * nlT + nb * t + bus)));
    const double vqg = neg(vrow<AL>(P, V + (T + 5 * nlT + nbT + nb * t + bus)));
    if (I.ramp) {  // rows pg_t - pg_{t-1}, t = 1..T-1
        const int rb = T + (RECT ? 8 * nlT + 3 * nbT : 7 * nlT + 2 * nbT);
        if (t >= 1)
            vpg += vrow<AL>(P, V + (rb + g + ng * (t - 1)));
        if (t + 1 <= T - 1)
            vpg -= vrow<AL>(P, V + (rb + g + ng * t));
    }
    if (I.link_c >= 0)  // rows pg_s - pg_0 of instance s >= 1
        vpg += vrow<AL>(P, I.link_c + g);
    if (I.res_c >= 0)  // the instance's reserve row of this period
        vpg += vrow<AL>(P, I.res_c + t);
    if (P.link && s == 0)  // instance 0 appears in every linking row
        for (int q = 1; q < P.ninst; q++)
            vpg -= vrow<AL>(P, P.link_c0 + g + (int64_t)ng * (q - 1));
    o[2 * nbT + ng * t + g] = vpg;
    o[2 * nbT + ngT + ng * t + g] = vqg;
}

template <bool ONE, bool RECT = false, bool STOR = false, bool AL = false>
__global__ void __launch_bounds__(256) jt_bus_kernel(const KParams P)
{
    cudaGridDependencySynchronize();
    cudaTriggerProgrammaticLaunchCompletion();  // the next kernel may launch now
    if (AL && P.bp && blockIdx.x == 0 && threadIdx.x == 0) {  // the next Adam step's bias corrections
        P.bp[0] *= 0.9;
        P.bp[1] *= 0.999;
        P.bp[2] = 1.0 - P.bp[0];
        P.bp[3] = 1.0 - P.bp[1];
        P.bp[4] = 1.0 / P.bp[2];  // once here, not per Adam entry
        P.bp[5] = 1.0 / P.bp[3];
    }
    const DevArrays &d = P.d;
    const int64_t total = P.nbus_items + P.ngen_items;
    for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < total;
         it += (int64_t)gridDim.x * blockDim.x) {
        int s, t, e;
        if (it < P.nbus_items) {
            if (ONE) {
                s = 0;
                split((int)it, P.inst0.nb, P.inst0.T, t, e);
            } else {
                s = find_inst(d.bus_items, P.ninst, it);
                split((int)(it - __ldg(d.bus_items + s)), __ldg(&d.inst[s].nb), __ldg(&d.inst[s].T), t, e);
            }
        } else {
            const int64_t gi = it - P.nbus_items;
            if (ONE) {
                s = 0;
                split((int)gi, P.inst0.ng, P.inst0.T, t, e);
            } else {
                s = find_inst(d.gen_items, P.ninst, gi);
                split((int)(gi - __ldg(d.gen_items + s)), __ldg(&d.inst[s].ng), __ldg(&d.inst[s].T), t, e);
            }
        }
        const InstDev I = inst_of<ONE>(P, s);
        const int nl = I.nl, nb = I.nb, ng = I.ng, T = I.T;
        const int nbT = nb * T, ngT = ng * T, nlT = nl * T, na = 2 * nl;
        const double *__restrict__ xs = P.x + I.x0;
        const int64_t V = I.c0;  // the vector v, indexed like the rows
        double *o = P.grad + I.x0;
        if (it < P.nbus_items) {
            // buses in the arc-count order (lanes of a warp walk similar
            // slot counts); the bus's entries are its own wherever it lands
            const int i = __ldg(d.bus_order + I.bus0 + e), ib = I.bus0 + i;
            const int4 a = __ldg(d.bus_a + ib);
            const double2 gb = __ldg(d.gsbs + ib);
            const double vm = __ldg(xs + nbT + nb * t + i);
            const double vP = vrow<AL>(P, V + (T + 5 * nlT + nb * t + i)), vQ = vrow<AL>(P, V + (T + 5 * nlT + nbT + nb * t + i));
            const double2 *Sg = reinterpret_cast<const double2 *>(d.arcs + I.scr0 + (int64_t)na * t + a.x);
            double dva, dvm;
            if constexpr (RECT) {  // vr, vi: 2 V (gs vP - bs vQ + vV); the reference row is vi_ref
                const double vr = __ldg(xs + nb * t + i);
                const double vV = vrow<AL>(P, V + (T + 8 * nlT + 2 * nbT + nb * t + i));
                const double k = twice(fma(gb.x, vP, fma(neg(gb.y), vQ, vV)));
                dva = vr * k;
                dvm = fma(vm, k, i == I.ref ? vrow<AL>(P, V + t) : 0.0);
            } else {
                dva = i == I.ref ? vrow<AL>(P, V + t) : 0.0;
                dvm = twice(vm * fma(gb.x, vP, neg(gb.y * vQ)));  // 2 vm (gs vP - bs vQ)
            }
            // the slots' records four at a time (their loads together), added
            // in slot order; the warp leaves once no lane has another slot
            const int nsl = a.y - a.x;
            for (int q0 = 0; q0 < nsl; q0 += 4) {
                double2 w[4];
#pragma unroll
                for (int u = 0; u < 4; u++)
                    if (q0 + u < nsl)
                        w[u] = __ldcg(Sg + 3 * (q0 + u));
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    if (!__any_sync(__activemask(), q0 + u < nsl))
                        break;
                    if (q0 + u < nsl) {
                        dva += w[u].x;
                        dvm += w[u].y;
                    }
                }
            }
            if constexpr (STOR) {  // the bus's storage units: their five entries, the loss rows' vm part
                const int2 stb = __ldg(d.bus_st + ib);
                const int ns = I.ns, nsT = ns * T;
                const int ist = 2 * nbT + 2 * ngT + 2 * na * T;
                const double iv2 = 1.0 / (vm * vm);
                const int64_t Vs = V + I.st_c;
                for (int e = stb.x; e < stb.y; e++) {
                    const int k = __ldg(d.st_list + e);
                    const double4_16a par = ldg4(d.st_par + I.st0 + k);
                    const int r = k + ns * t, v = ist + r;
                    const double ps = __ldg(xs + v), qs = __ldg(xs + v + nsT);
                    const double sc = __ldg(xs + v + 2 * nsT), sd = __ldg(xs + v + 3 * nsT);
                    const double vs = vrow<AL>(P, Vs + r), vl = vrow<AL>(P, Vs + nsT + r), vt = vrow<AL>(P, Vs + 2 * nsT + r);
                    const double vc = I.st_compl ? vrow<AL>(P, Vs + 3 * nsT + r) : 0.0;
                    const double vn = t + 1 < T ? vrow<AL>(P, Vs + r + ns) : 0.0;  // next period's state of charge
                    const double rr = twice(par.z) * iv2;  // 2 r / vm^2
                    dvm = fma(vl * rr, fma(ps, ps, qs * qs) / vm, dvm);
                    o[v] = fma(twice(ps), vt, fma(vl, fma(neg(rr), ps, 1.0), vP));
                    o[v + nsT] = fma(twice(qs), vt, fma(vl, neg(rr * qs), vQ));
                    o[v + 2 * nsT] = fma(vc, sd, fma(neg(par.x), vs, neg(vl)));
                    o[v + 3 * nsT] = fma(vc, sc, fma(par.y, vs, vl));
                    o[v + 4 * nsT] = vs - vn;
                }
            }
            o[nb * t + i] = dva;
            o[nbT + nb * t + i] = dvm;
        } else {
            jt_gen_item<RECT, AL>(P, I, s, t, e);
        }
    }
}

// Fused J^T v (bus_order 3, models without storage): one kernel, the
// packed warps of the fused evaluation. Each slot lane takes its arc end: the
// p and q entries of its arc completely (flow row, thermal row, the balance
// rows of its bus, whose v it reads) and the va, vm (vr, vi) parts of its
// bus's entries from every row of its branch (its own end's flow rows, the
// far end's, the angle rows). The parts are summed per bus by a segmented
// scan and the bus's last lane adds the reference and balance-row terms.
// Generator items run in the blocks before the packed warps.
template <bool ONE, bool RECT, bool AL>
__device__ void fused_jt_warp(const KParams &P, const int64_t w)
{
    const DevArrays &d = P.d;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    if (w >= P.npack_items) {
        cudaGridDependencySynchronize();
        cudaTriggerProgrammaticLaunchCompletion();
        return;
    }
    int s = 0, t = 0, wl = 0;
    if (ONE) {
        split((int)w, P.inst0.npack, P.inst0.T, t, wl);
    } else {
        s = find_inst(d.pack_items, P.ninst, w);
        const InstDev *Ip = d.inst + s;
        split((int)(w - __ldg(d.pack_items + s)), __ldg(&Ip->npack), __ldg(&Ip->T), t, wl);
    }
    const InstDev I = inst_of<ONE>(P, s);
    const int4 ld = __ldg(d.pack + (((int64_t)I.pack0 + wl) << 5) + lane);  // (arc, bus, flags, group)
    const int fl = ld.z;
    const bool valid = (fl & PK_VALID) != 0, tail = (fl & PK_TAIL) != 0;
    const bool has = ld.x >= 0;
    const int nl = I.nl;
    const int e = has && ld.x >= nl ? 1 : 0;  // 0: from-end, 1: to-end
    const int k = has ? ld.x - e * nl : 0;
    const int kb = I.br0 + k;
    int4 br = make_int4(0, 0, 0, 0);
    double2 Yo = make_double2(0.0, 0.0), Yx = make_double2(0.0, 0.0), Yf = make_double2(0.0, 0.0);
    double2 gb = make_double2(0.0, 0.0);
    double tno = 0.0, tnf = 0.0;
    if (has) {
        br = __ldg(d.br + kb);
        Yo = __ldg((e ? d.y_tt : d.y_ff) + kb);
        Yx = __ldg((e ? d.y_tf : d.y_ft) + kb);
        Yf = __ldg((e ? d.y_ft : d.y_tf) + kb);
        if (RECT) {
            const double2 tb = __ldg(d.tanb + kb);
            tno = e ? tb.y : tb.x;
            tnf = e ? tb.x : tb.y;
        }
    }
    const int i = ld.y;
    if (valid && tail)
        gb = __ldg(d.gsbs + I.bus0 + i);
    cudaGridDependencySynchronize();
    cudaTriggerProgrammaticLaunchCompletion();  // the next kernel may launch now

    const int nb = I.nb, ng = I.ng, T = I.T;
    const int nbT = nb * T, ngT = ng * T, nlT = nl * T, na = 2 * nl;
    const int rk = k + nl * t;
    const int own = has ? (e ? br.y : br.x) : i, far = e ? br.x : br.y;
    const double *__restrict__ xs = P.x + I.x0;
    const int iva = nb * t, ivm = nbT + nb * t;
    const int ip = 2 * nbT + 2 * ngT + na * t, iq = ip + na * T;
    const int arc = e ? nl + k : k;
    double *o = P.grad + I.x0;  // P.grad carries `out`
    double vao = 0.0, vo = 0.0, bP = 0.0, bQ = 0.0;
    const int64_t VB = I.c0 + (T + 5 * nlT + nb * t);  // balance rows, period t
    if (valid) {
        vao = __ldg(xs + iva + own);
        vo = __ldg(xs + ivm + own);
        bP = vrow<AL>(P, VB + i);
        bQ = vrow<AL>(P, VB + nbT + i);
    }
    double dA = 0.0, dM = 0.0;  // this slot's va and vm (vr and vi) parts
    if (has) {
        const double vax = __ldg(xs + iva + far), vx = __ldg(xs + ivm + far);
        const double po = __ldg(xs + ip + arc), qo = __ldg(xs + iq + arc);
        const int64_t V = I.c0 + (T + rk);  // the vector v, indexed like the rows
        const double mP = vrow<AL>(P, V + (e ? 2 * nlT : 0)), mQ = vrow<AL>(P, V + (e ? 3 * nlT : nlT));
        const double fP = vrow<AL>(P, V + (e ? 0 : 2 * nlT)), fQ = vrow<AL>(P, V + (e ? nlT : 3 * nlT));
        const double th = vrow<AL>(P, V + ((e ? 6 : 5) * nlT + 2 * nbT));
        // own variables: flow row, thermal row, balance row of the arc's bus
        o[ip + arc] = fma(twice(po), th, mP + bP);
        o[iq + arc] = fma(twice(qo), th, mQ + bQ);
        if constexpr (RECT) {
            // v^T g over the branch's rows: (De/2)|V_own|^2 + ... + aR wR + aI wI
            const double ma = vrow<AL>(P, V + (e ? 7 * nlT + 2 * nbT : 4 * nlT));
            const double fa = vrow<AL>(P, V + (e ? 4 * nlT : 7 * nlT + 2 * nbT));
            const double Re = neg(fma(mP, Yx.x, fma(neg(mQ), Yx.y, ma * tno)));
            const double Ie = flip(fma(mP, Yx.y, mQ * Yx.x), !e) + ma;
            const double Rf = neg(fma(fP, Yf.x, fma(neg(fQ), Yf.y, fa * tnf)));
            const double If = flip(fma(fP, Yf.y, fQ * Yf.x), e) + fa;
            const double aR = e ? Rf + Re : Re + Rf;  // from-end part first
            const double sI = flip(e ? If + Ie : Ie + If, e);
            const double De = neg(twice(fma(mP, Yo.x, neg(mQ * Yo.y))));
            dA = fma(De, vao, fma(aR, vax, neg(sI * vx)));
            dM = fma(De, vo, fma(aR, vx, sI * vax));
        } else {
            const double va_ = vrow<AL>(P, V + 4 * nlT);  // the angle row
            double sn, cs_;
            sincos_tab(vao - vax, d.trig, &sn, &cs_);
            const double vft = vo * vx;
            const double A = fma(Yx.x, cs_, Yx.y * sn), B = fma(Yx.x, sn, neg(Yx.y * cs_));
            const double Af = fma(Yf.x, cs_, neg(Yf.y * sn)), Bf = neg(fma(Yf.x, sn, Yf.y * cs_));
            const double dva = fma(mP, B, fma(neg(mQ), A, fma(neg(fP), Bf, fQ * Af)));
            dA = fma(vft, dva, flip(va_, e));
            dM = fma(neg(mP), fma(Yo.x, twice(vo), vx * A), fma(mQ, fma(Yo.y, twice(vo), neg(vx * B)),
                                                                  neg(vx * fma(fP, Af, fQ * Bf))));
        }
    }
    // per-bus sums of the slots' parts
    const unsigned upto = (2u << lane) - 1u;
    const unsigned bheads = __ballot_sync(full, (fl & PK_HEAD) || !valid);
    const int bhead = 31 - __clz(bheads & upto);
    const int bmax = __reduce_max_sync(full, (unsigned)(lane - bhead + 1));
    for (int dd = 1; dd < bmax; dd <<= 1) {
        const double ya = __shfl_up_sync(full, dA, dd), ym = __shfl_up_sync(full, dM, dd);
        if (lane - dd >= bhead) {
            dA += ya;
            dM += ym;
        }
    }
    if (!(valid && tail))
        return;
    const double vref = i == I.ref ? vrow<AL>(P, I.c0 + t) : 0.0;
    if constexpr (RECT) {  // vr, vi: 2 V (gs vP - bs vQ + vV); the reference row is vi_ref
        const double vV = vrow<AL>(P, I.c0 + (T + 8 * nlT + 2 * nbT + nb * t + i));
        const double kk = twice(fma(gb.x, bP, fma(neg(gb.y), bQ, vV)));
        o[iva + i] = fma(vao, kk, dA);
        o[ivm + i] = fma(vo, kk, dM) + vref;
    } else {
        o[iva + i] = dA + vref;
        o[ivm + i] = fma(twice(vo), fma(gb.x, bP, neg(gb.y * bQ)), dM);  // 2 vm (gs vP - bs vQ)
    }
}

template <bool ONE, bool RECT, bool AL>
__global__ void __launch_bounds__(256) jt_fused_kernel(const KParams P)
{
    if ((int)blockIdx.x >= P.split_tblocks) {  // the packed warps
        fused_jt_warp<ONE, RECT, AL>(P, (int64_t)(blockIdx.x - P.split_tblocks) * (blockDim.x >> 5) +
                                            (threadIdx.x >> 5));
        return;
    }
    cudaGridDependencySynchronize();
    cudaTriggerProgrammaticLaunchCompletion();  // the next kernel may launch now
    if (AL && P.bp && blockIdx.x == 0 && threadIdx.x == 0) {  // the next Adam step's bias corrections
        P.bp[0] *= 0.9;
        P.bp[1] *= 0.999;
        P.bp[2] = 1.0 - P.bp[0];
        P.bp[3] = 1.0 - P.bp[1];
        P.bp[4] = 1.0 / P.bp[2];  // once here, not per Adam entry
        P.bp[5] = 1.0 / P.bp[3];
    }
    const DevArrays &d = P.d;
    for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < P.ngen_items;
         it += (int64_t)P.split_tblocks * blockDim.x) {
        int s, t, g;
        if (ONE) {
            s = 0;
            split((int)it, P.inst0.ng, P.inst0.T, t, g);
        } else {
            s = find_inst(d.gen_items, P.ninst, it);
            split((int)(it - __ldg(d.gen_items + s)), __ldg(&d.inst[s].ng), __ldg(&d.inst[s].T), t, g);
        }
        jt_gen_item<RECT, AL>(P, inst_of<ONE>(P, s), s, t, g);
    }
}

// The augmented Lagrangian's gradient in one kernel (fused layout, polar,
// without linking or reserve rows): out = grad f + J^T mu with mu_r =
// rho (s_r - clip(s_r, gl_r, gu_r)), s_r = c_r + lambda_r / rho, where every
// row value c_r is formed where it is needed instead of being read: each
// slot lane forms its own end's flow and thermal rows, the far end's flow
// rows and the angle row, and their multipliers; the bus's last lane forms
// the balance rows from the scanned p and q sums, and hands their
// multipliers back to the bus's slot lanes by shuffles for the p and q
// entries; it also writes its generators' entries (cost gradient, balance
// and ramp rows). Advances the Adam step state bp like the J^T kernels.
__device__ __forceinline__ double al_mu(const KParams &P, int64_t row, double c)
{
    const double s = fma(__ldg(P.lam + row), P.inv_rho, c);
    return P.rho * (s - fmin(fmax(s, __ldg(P.gl + row)), __ldg(P.gu + row)));
}

template <bool ONE>
__global__ void __launch_bounds__(256) al_grad_kernel(const KParams P)
{
    const DevArrays &d = P.d;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= P.npack_items) {
        cudaGridDependencySynchronize();
        cudaTriggerProgrammaticLaunchCompletion();
        return;
    }
    int s = 0, t = 0, wl = 0;
    if (ONE) {
        split((int)w, P.inst0.npack, P.inst0.T, t, wl);
    } else {
        s = find_inst(d.pack_items, P.ninst, w);
        const InstDev *Ip = d.inst + s;
        split((int)(w - __ldg(d.pack_items + s)), __ldg(&Ip->npack), __ldg(&Ip->T), t, wl);
    }
    const InstDev I = inst_of<ONE>(P, s);
    const int4 ld = __ldg(d.pack + (((int64_t)I.pack0 + wl) << 5) + lane);  // (arc, bus, flags, group)
    const int fl = ld.z;
    const bool valid = (fl & PK_VALID) != 0, tail = (fl & PK_TAIL) != 0;
    const bool has = ld.x >= 0;
    const int nl = I.nl;
    const int e = has && ld.x >= nl ? 1 : 0;  // 0: from-end, 1: to-end
    const int k = has ? ld.x - e * nl : 0;
    const int kb = I.br0 + k;
    int4 br = make_int4(0, 0, 0, 0), a = make_int4(0, 0, 0, 0);
    double2 Yo = make_double2(0.0, 0.0), Yx = make_double2(0.0, 0.0);
    double2 Yfo = make_double2(0.0, 0.0), Yf = make_double2(0.0, 0.0), gb = make_double2(0.0, 0.0);
    double r2 = 0.0;
    if (has) {
        br = __ldg(d.br + kb);
        Yo = __ldg((e ? d.y_tt : d.y_ff) + kb);
        Yx = __ldg((e ? d.y_tf : d.y_ft) + kb);
        Yfo = __ldg((e ? d.y_ff : d.y_tt) + kb);  // the far end's own and transfer admittances
        Yf = __ldg((e ? d.y_ft : d.y_tf) + kb);
        r2 = __ldg(d.rate2 + kb);
    }
    const int i = ld.y;
    if (valid && tail) {
        a = __ldg(d.bus_a + I.bus0 + i);
        gb = __ldg(d.gsbs + I.bus0 + i);
    }
    cudaGridDependencySynchronize();
    cudaTriggerProgrammaticLaunchCompletion();  // the next kernel may launch now
    if (P.bp && w == 0 && lane == 0) {  // the next Adam step's bias corrections
        P.bp[0] *= 0.9;
        P.bp[1] *= 0.999;
        P.bp[2] = 1.0 - P.bp[0];
        P.bp[3] = 1.0 - P.bp[1];
        P.bp[4] = 1.0 / P.bp[2];  // once here, not per Adam entry
        P.bp[5] = 1.0 / P.bp[3];
    }

    const int nb = I.nb, ng = I.ng, T = I.T;
    const int nbT = nb * T, ngT = ng * T, nlT = nl * T, na = 2 * nl;
    const int rk = k + nl * t;
    const int own = has ? (e ? br.y : br.x) : i, far = e ? br.x : br.y;
    const double *__restrict__ xs = P.x + I.x0;
    const int iva = nb * t, ivm = nbT + nb * t;
    const int ip = 2 * nbT + 2 * ngT + na * t, iq = ip + na * T;
    const int arc = e ? nl + k : k, farc = e ? k : nl + k;
    double *o = P.grad + I.x0;  // P.grad carries `out`
    const int64_t R = I.c0 + T + rk;  // this branch's first flow row
    double vao = 0.0, vo = 0.0, po = 0.0, qo = 0.0;
    if (valid) {
        vao = __ldg(xs + iva + own);
        vo = __ldg(xs + ivm + own);
    }
    double dA = 0.0, dM = 0.0, mP = 0.0, mQ = 0.0, mth = 0.0;
    if (has) {
        const double vax = __ldg(xs + iva + far), vx = __ldg(xs + ivm + far);
        po = __ldg(xs + ip + arc);
        qo = __ldg(xs + iq + arc);
        const double pf = __ldg(xs + ip + farc), qf = __ldg(xs + iq + farc);
        const double dlt = vao - vax;
        double sn, cs_;
        sincos_tab(dlt, d.trig, &sn, &cs_);
        const double vft = vo * vx;
        const double A = fma(Yx.x, cs_, Yx.y * sn), B = fma(Yx.x, sn, neg(Yx.y * cs_));
        const double Af = fma(Yf.x, cs_, neg(Yf.y * sn)), Bf = neg(fma(Yf.x, sn, Yf.y * cs_));
        // the branch's rows at this lane: own and far flow rows, the angle row, own thermal row
        mP = al_mu(P, R + (e ? 2 * nlT : 0), po - fma(Yo.x, vo * vo, vft * A));
        mQ = al_mu(P, R + (e ? 3 * nlT : nlT), qo - fma(neg(Yo.y), vo * vo, vft * B));
        const double fP = al_mu(P, R + (e ? 0 : 2 * nlT), pf - fma(Yfo.x, vx * vx, vft * Af));
        const double fQ = al_mu(P, R + (e ? nlT : 3 * nlT), qf - fma(neg(Yfo.y), vx * vx, vft * Bf));
        const double mang = al_mu(P, R + 4 * nlT, flip(dlt, e));  // va_f - va_t
        mth = al_mu(P, R + ((e ? 6 : 5) * nlT + 2 * nbT), fma(po, po, qo * qo) - r2);
        const double dva = fma(mP, B, fma(neg(mQ), A, fma(neg(fP), Bf, fQ * Af)));
        dA = fma(vft, dva, flip(mang, e));
        dM = fma(neg(mP), fma(Yo.x, twice(vo), vx * A), fma(mQ, fma(Yo.y, twice(vo), neg(vx * B)),
                                                              neg(vx * fma(fP, Af, fQ * Bf))));
    }
    // per-bus sums: p, q (for the balance rows) and the voltage parts
    const unsigned upto = (2u << lane) - 1u;
    const unsigned bheads = __ballot_sync(full, (fl & PK_HEAD) || !valid);
    const int bhead = 31 - __clz(bheads & upto);
    const int bmax = __reduce_max_sync(full, (unsigned)(lane - bhead + 1));
    double tp = po, tq = qo;
    for (int dd = 1; dd < bmax; dd <<= 1) {
        const double yp = __shfl_up_sync(full, tp, dd), yq = __shfl_up_sync(full, tq, dd);
        const double ya = __shfl_up_sync(full, dA, dd), ym = __shfl_up_sync(full, dM, dd);
        if (lane - dd >= bhead) {
            tp += yp;
            tq += yq;
            dA += ya;
            dM += ym;
        }
    }
    // the bus's last lane: its balance rows and their multipliers
    double mbP = 0.0, mbQ = 0.0;
    const int64_t RB = I.c0 + (T + 5 * nlT + nb * t + i);  // balance P row of the bus
    if (valid && tail) {
        const double vm2 = vo * vo;
        double Pb = fma(gb.x, vm2, __ldg(d.Pd + I.pd0 + (nb * t + i)));
        double Qb = fma(neg(gb.y), vm2, __ldg(d.Qd + I.pd0 + (nb * t + i)));
        for (int gp = a.z; gp < a.w; gp++) {
            const int g = __ldg(d.gen_list + I.gl0 + gp);
            Pb -= __ldg(xs + 2 * nbT + ng * t + g);
            Qb -= __ldg(xs + 2 * nbT + ngT + ng * t + g);
        }
        mbP = al_mu(P, RB, Pb + tp);
        mbQ = al_mu(P, RB + nbT, Qb + tq);
    }
    // hand them to the bus's slot lanes (the first tail lane at or above this one)
    const unsigned tails = __ballot_sync(full, tail || !valid);
    const int mytail = __ffs(tails & ~(upto >> 1)) - 1;
    mbP = __shfl_sync(full, mbP, mytail);
    mbQ = __shfl_sync(full, mbQ, mytail);
    if (has) {  // own variables: flow row, thermal row, balance row of the arc's bus
        o[ip + arc] = fma(twice(po), mth, mP + mbP);
        o[iq + arc] = fma(twice(qo), mth, mQ + mbQ);
    }
    if (!(valid && tail))
        return;
    const double mref = i == I.ref ? al_mu(P, I.c0 + t, vao) : 0.0;
    o[iva + i] = dA + mref;
    o[ivm + i] = fma(twice(vo), fma(gb.x, mbP, neg(gb.y * mbQ)), dM);  // 2 vm (gs muP - bs muQ)
    const int rb = T + 7 * nlT + 2 * nbT;  // ramp rows
    for (int gp = a.z; gp < a.w; gp++) {  // the bus's generators: cost, balance and ramp rows
        const int g = __ldg(d.gen_list + I.gl0 + gp);
        const int ipg = 2 * nbT + ng * t + g;
        const double pg = __ldg(xs + ipg);
        const int gg = I.gen0 + g;
        double upg = fma(twice(__ldg(d.c2 + gg)), pg, __ldg(d.c1 + gg)) - mbP;
        if (I.ramp) {  // rows pg_t - pg_{t-1}, t = 1..T-1
            if (t >= 1)
                upg += al_mu(P, I.c0 + (rb + g + ng * (t - 1)), pg - __ldg(xs + ipg - ng));
            if (t + 1 <= T - 1)
                upg -= al_mu(P, I.c0 + (rb + g + ng * t), __ldg(xs + ipg + ng) - pg);
        }
        o[ipg] = upg;
        o[ipg + ngT] = neg(mbQ);
    }
}

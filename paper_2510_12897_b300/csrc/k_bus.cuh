// k_bus.cuh: the bus-phase kernel, the split bus phase's heavy-bus warps and the fused evaluation
//
// Part of the translation unit of kernels.cu, which includes it inside
// namespace opf::(anonymous) after k_branch.cuh; not a standalone header.

constexpr int kBusBlockMax = 256;

// Split bus phase, heavy buses: one warp per (instance, period, bus) with
// kLightSlots < slots <= 32, one lane per slot. A segmented inclusive scan
// (shuffles, fixed order) sums each group of parallel arcs, whose last lane
// writes the group's off-diagonal Hessian entries; butterfly sums (fixed
// order) give the bus totals, and lane 0 finishes the bus exactly as a
// light bus's thread does (models without storage; both forms).
__device__ __forceinline__ double seg_scan(double v, int lane, int head)
{
#pragma unroll
    for (int dd = 1; dd < 32; dd <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, v, dd);
        if (lane - dd >= head)
            v += y;
    }
    return v;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int dd = 16; dd; dd >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, dd);
    return v;
}

template <bool CONS, bool JAC, bool HESS, bool ONE, bool RECT>
__device__ void heavy_bus_warp(const KParams &P)
{
    const DevArrays &d = P.d;
    const int lane = threadIdx.x & 31;
    const int64_t hw = (int64_t)(blockIdx.x - P.split_tblocks) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (hw >= P.nheavy_items) {
        cudaGridDependencySynchronize();
        cudaTriggerProgrammaticLaunchCompletion();
        return;
    }
    int s = 0, t = 0, h = 0;
    if (ONE) {
        split((int)hw, P.inst0.nheavy, P.inst0.T, t, h);
    } else {
        s = find_inst(d.heavy_items, P.ninst, hw);
        const InstDev *Ip = d.inst + s;
        split((int)(hw - __ldg(d.heavy_items + s)), __ldg(&Ip->nheavy), __ldg(&Ip->T), t, h);
    }
    const InstDev I = inst_of<ONE>(P, s);
    const int i = __ldg(d.heavy_list + I.heavy0 + h);
    const int ib = I.bus0 + i;
    const int4 a = __ldg(d.bus_a + ib), b = __ldg(d.bus_b + ib);
    const int2 m = __ldg(d.bus_c + ib);
    const double2 gb = __ldg(d.gsbs + ib);
    const int nsl = a.y - a.x;  // kLightSlots < nsl <= 32
    const bool has = lane < nsl;
    const unsigned code = has ? ((((unsigned)m.x >> lane) & 1u) | (lane < m.y ? 2u : 0u)) : 0u;
    int gfirst = -1;
    if (CONS && a.z < a.w)
        gfirst = __ldg(d.gen_list + I.gl0 + a.z);
    cudaGridDependencySynchronize();
    cudaTriggerProgrammaticLaunchCompletion();

    const int nl = I.nl, nb = I.nb, ng = I.ng, T = I.T;
    const int nbT = nb * T, ngT = ng * T, nlT = nl * T, na = 2 * nl;
    const double *__restrict__ xs = P.x + I.x0;
    double2 v0 = make_double2(0.0, 0.0), v1 = make_double2(0.0, 0.0), v2 = make_double2(0.0, 0.0);
    if (has) {
        const double2 *S = reinterpret_cast<const double2 *>(d.arcs + I.scr0 + (int64_t)na * t + a.x + lane);
        if (CONS)
            v0 = __ldcg(S);
        if (HESS) {
            v1 = __ldcg(S + 1);
            v2 = __ldcg(S + 2);
        }
    }
    const int iva = nb * t, ivm = nbT + nb * t;
    // polar: vm; rectangular: vi (and vr below)
    const double vm = __ldg(xs + ivm + i);
    const int hva = (int)I.hva, hvm = (int)I.hvm;
    double *Hvm = P.hess + I.h0 + (hva * T + hvm * t + b.z);
    double *Hva = P.hess + I.h0 + (hva * t + b.y);
    const int nd = b.w & 0xffff, nlt = b.w >> 16;
    double taa = 0.0, tma = 0.0, tmm = 0.0, tp = 0.0, tq = 0.0;
    if (HESS) {  // groups of parallel arcs end at SLOT_LAST slots
        const unsigned below = (1u << lane) - 1u;
        const unsigned tails = __ballot_sync(0xffffffffu, has && (code & SLOT_LAST));
        const unsigned tb = tails & below;
        const int ghead = tb ? 32 - __clz(tb) : 0;
        if constexpr (RECT) {
            // slots hold (diagonal part, aR) and the signed aI: the group sums
            // of aR give (vr_i, vr_j) = (vi_i, vi_j), those of aI (vi_i, vr_j)
            const double gaa = seg_scan(v1.y, lane, ghead);
            const double gma = seg_scan(v2.x, lane, ghead);
            if (has && (code & SLOT_LAST)) {
                const int grp = __popc(tb);
                Hvm[grp] = gma;  // (vi_i, vr_j)
                if (code & SLOT_LOWER) {
                    Hva[grp] = gaa;       // (vr_i, vr_j), j < i
                    Hvm[nd + grp] = gaa;  // (vi_i, vi_j), j < i
                }
            }
            tmm = warp_sum(v1.x);
        } else {
            const double gaa = seg_scan(v1.x, lane, ghead);
            const double gma = seg_scan(v1.y, lane, ghead);
            const double gmm = seg_scan(v2.y, lane, ghead);
            if (has && (code & SLOT_LAST)) {
                const int grp = __popc(tb);
                Hvm[grp < nlt ? grp : grp + 1] = neg(gma);  // (vm_i, va_j)
                if (code & SLOT_LOWER) {
                    Hva[grp] = neg(gaa);         // (va_i, va_j), j < i
                    Hvm[nd + 1 + grp] = gmm;     // (vm_i, vm_j), j < i
                }
            }
            taa = warp_sum(v1.x);
            tma = warp_sum(v1.y);
            tmm = warp_sum(v2.x);
        }
    }
    if (CONS) {
        tp = warp_sum(v0.x);
        tq = warp_sum(v0.y);
    }
    if (lane != 0)
        return;
    // lane 0: the bus's own terms, as for a light bus
    const double vr = RECT ? __ldg(xs + iva + i) : 0.0;
    const int ng_here = a.w - a.z;
    if (P.want_grad) {
        P.grad[I.x0 + iva + i] = 0.0;
        P.grad[I.x0 + ivm + i] = 0.0;
    }
    if (i == I.ref) {  // va_ref, or vi_ref (rectangular)
        if (CONS)
            P.c[I.c0 + t] = RECT ? vm : __ldg(xs + iva + i);
        if (JAC)
            P.jac[I.j0 + t] = 1.0;
    }
    if (JAC) {
        const int jP = (int)I.jP;
        double *JP = P.jac + I.j0 + (T + (RECT ? 24 : 22) * nlT + jP * t + b.x);
        double *JQ = JP + jP * T;
        const double v2m = twice(vm);
        if constexpr (RECT) {  // d|V|^2 = (2 vr, 2 vi); the magnitude row
            const double r2 = twice(vr);
            JP[0] = gb.x * r2;
            JP[1] = gb.x * v2m;
            JQ[0] = neg(gb.y * r2);
            JQ[1] = neg(gb.y * v2m);
            double *JV = P.jac + I.j0 + (T + 32 * nlT + 2 * jP * T + 2 * (nb * t + i));
            JV[0] = r2;
            JV[1] = v2m;
        } else {
            JP[0] = gb.x * v2m;
            JQ[0] = neg(gb.y * v2m);
        }
        for (int e = RECT ? 2 : 1; e <= ng_here + (RECT ? 1 : 0); e++) {
            JP[e] = -1.0;
            JQ[e] = -1.0;
        }
    }
    if (CONS) {
        const double vm2 = RECT ? fma(vr, vr, vm * vm) : vm * vm;  // |V|^2
        double Pb = fma(gb.x, vm2, __ldg(d.Pd + I.pd0 + (nb * t + i)));
        double Qb = fma(neg(gb.y), vm2, __ldg(d.Qd + I.pd0 + (nb * t + i)));
        for (int gp = a.z; gp < a.w; gp++) {
            const int g = gp == a.z ? gfirst : __ldg(d.gen_list + I.gl0 + gp);
            Pb -= __ldg(xs + 2 * nbT + ng * t + g);
            Qb -= __ldg(xs + 2 * nbT + ngT + ng * t + g);
        }
        double *c = P.c + I.c0 + (T + 5 * nlT + nb * t + i);
        c[0] = Pb + tp;
        c[nbT] = Qb + tq;
        if (RECT)
            c[3 * nlT + 2 * nbT] = vm2;  // the magnitude row
    }
    if (HESS) {
        const double *L = P.lam + I.c0 + (T + 5 * nlT + nb * t + i);
        // 2 gs lP - 2 bs lQ (+ 2 lV, the magnitude row, rectangular)
        const double lV = RECT ? __ldg(L + (3 * nlT + 2 * nbT)) : 0.0;
        const double dmm = twice(fma(gb.x, __ldg(L), fma(neg(gb.y), __ldg(L + nbT), lV))) + tmm;
        if (RECT) {  // diagonals (vr_i, vr_i) and (vi_i, vi_i)
            Hva[nlt] = dmm;
            Hvm[nd + nlt] = dmm;
        } else {
            Hva[nlt] = taa;
            Hvm[nlt] = tma;
            Hvm[nd + 1 + nlt] = dmm;
        }
    }
}


// One arc end of the fused evaluation in rectangular form: the rows, the
// Jacobian, the flow Hessian diagonals and the gradient zeros of one lane of
// the rectangular two-lane branch kernel, with the far end's parts of aR and
// aI formed here from the far multipliers, admittance and angle limit.
// Returns the slot's Hessian parts: h1 the diagonal part, h2 aR, h3 the
// signed aI.
template <bool CONS, bool JAC, bool HESS>
__device__ __forceinline__ void fused_rect_arc(const KParams &P, const InstDev &I, int e, int k, int t, int own,
                                               int far, int4 br, int jb, double2 Yo, double2 Yx, double2 Yf,
                                               double r2, double tno, double tnf, double vro, double vrx,
                                               double vio, double vix, double po, double qo, double mP, double mQ,
                                               double ma, double lth, double fP, double fQ, double fa,
                                               bool grad_here, double &h1, double &h2, double &h3)
{
    const int nl = I.nl, nb = I.nb, ng = I.ng, T = I.T;
    const int nbT = nb * T, ngT = ng * T, nlT = nl * T, na = 2 * nl;
    const int rk = k + nl * t;
    const int f = br.x, b = br.y;
    const int ip = 2 * nbT + 2 * ngT + na * t, iq = ip + na * T;
    const int arc = e ? nl + k : k;
    // w_e = V_own conj(V_far): w at the from-end, conj(w) at the to-end
    const double wR = fma(vro, vrx, vio * vix);
    const double wI = fma(vio, vrx, neg(vro * vix));
    if (CONS) {
        const double vo2 = fma(vro, vro, vio * vio);
        double *c = P.c + I.c0 + (T + rk);
        c[e ? 2 * nlT : 0] = po - fma(Yo.x, vo2, fma(Yx.x, wR, Yx.y * wI));
        c[e ? 3 * nlT : nlT] = qo - fma(neg(Yo.y), vo2, fma(Yx.x, wI, neg(Yx.y * wR)));
        c[e ? 7 * nlT + 2 * nbT : 4 * nlT] = fma(neg(tno), wR, flip(wI, e));  // this lane's angle row
        c[(e ? 6 : 5) * nlT + 2 * nbT] = fma(po, po, qo * qo) - r2;
    }
    if (JAC) {
        const int jP = (int)I.jP;
        const bool o_lo = own < far;
        double *J = P.jac + I.j0;
        double *Jf = J + (T + 5 * rk + (e ? 10 * nlT : 0));
        const double y1r = fma(Yx.x, vrx, neg(Yx.y * vix)), y1i = fma(Yx.x, vix, Yx.y * vrx);
        const double y2r = fma(Yx.x, vro, Yx.y * vio), y2i = fma(Yx.y, vro, neg(Yx.x * vio));
        const double pa = neg(twice(Yo.x)), qa = twice(Yo.y);
        Grad4 g;  // (own, far) in the places of (f, t)
        g.rf = fma(pa, vro, neg(y1r)); g.jf = fma(pa, vio, neg(y1i)); g.rt = neg(y2r); g.jt = y2i;
        put_rect(Jf, o_lo, g, true);
        g.rf = fma(qa, vro, y1i); g.jf = fma(qa, vio, neg(y1r)); g.rt = y2i; g.jt = y2r;
        put_rect(Jf + 5 * nlT, o_lo, g, true);
        const double tu = neg(tno);
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
    if (HESS) {
        // aR = -(m1 Gft - m2 Bft + a1 tan(angmax)) - (m3 Gtf - m4 Btf + a2 tan(angmin))
        // aI = (-m1 Bft - m2 Gft + a1) + (m3 Btf + m4 Gtf + a2): one part per end
        const double Re = neg(fma(mP, Yx.x, fma(neg(mQ), Yx.y, ma * tno)));
        const double Ie = flip(fma(mP, Yx.y, mQ * Yx.x), !e) + ma;
        const double Rf = neg(fma(fP, Yf.x, fma(neg(fQ), Yf.y, fa * tnf)));
        const double If = flip(fma(fP, Yf.y, fQ * Yf.x), e) + fa;
        const double aR = e ? Rf + Re : Re + Rf;  // from-end part first
        const double aI = e ? If + Ie : Ie + If;
        h1 = neg(twice(fma(mP, Yo.x, neg(mQ * Yo.y))));
        h2 = aR;
        h3 = flip(aI, e);
        double *Hp = P.hess + I.h0 + ((int)(I.hva + I.hvm) * T + ngT + arc + na * t);
        const double l2 = twice(lth);
        Hp[0] = l2;       // (p_arc, p_arc)
        Hp[na * T] = l2;  // (q_arc, q_arc)
    }
    if (P.want_grad && grad_here) {
        P.grad[I.x0 + ip + arc] = 0.0;
        P.grad[I.x0 + iq + arc] = 0.0;
    }
}

// Fused evaluation (bus_order 3, models without storage): the whole
// evaluation in one kernel, without the arc scratch. Buses are packed whole
// into warps, one lane per arc slot (a bus without arcs takes one lane), so
// a bus's arcs sit in consecutive lanes of one warp. Each slot lane does the
// work of one lane of the two-lane branch kernel for its arc's end at its
// bus (the end's flow rows, Jacobian rows, thermal row, balance +1 entries,
// flow Hessian diagonals and gradient zeros; the from-end lane also the
// angle row), and forms the far end's part of U and V itself (the far
// multipliers and admittance; the far angle is -d, so sin changes sign)
// instead of receiving it. The slot's second-order parts are then summed
// per bus and per group of parallel arcs by segmented inclusive scans over
// the lanes (fixed order; only as many steps as the warp's longest bus or
// group needs, and no group scan in warps whose groups are single arcs),
// and the last lane of each bus writes the bus's own rows, as the bus phase
// does. Generator items run in the blocks before the packed warps. In
// rectangular form the slot lane does one lane of the rectangular two-lane
// kernel (fused_rect_arc), and the scans sum the diagonal parts per bus and
// aR and the signed aI per group.
//
// With two roles (branch_occupancy 2 in this mode) each packed warp of buses
// is taken by two warps, one writing the rows and the Jacobian (and the
// gradient zeros), the other the Hessian, so the dependent chain of each is
// shorter. In blocks of one warp both evaluate the shared trigonometry.
// Two-role exchange (polar, blocks of two warps or more, where both warps of
// a pair are in one block): the rows warp of a pair publishes each lane's
// sine and cosine in shared memory and raises the pair's flag; the Hessian
// warp waits for the flag (bounded: on a timeout it computes them itself,
// with the same result) instead of recomputing them. One slot per pair of a
// block (at most kBusBlockMax / 64 pairs); the flags are cleared at the
// block's start.
__shared__ double2 g_role_sc[kBusBlockMax / 64][32];
__shared__ int g_role_flag[kBusBlockMax / 64];
constexpr int kRoleWaitPolls = 1 << 20;

template <bool CONS, bool JAC, bool HESS, bool ONE, bool RECT = false, int ROLE = 0>
__device__ void fused_bus_warp(const KParams &P, const int64_t w, const bool grad_here)
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
    const bool has = ld.x >= 0;  // an arc end (else a bus without arcs, or padding)
    const int nl = I.nl;
    const int e = has && ld.x >= nl ? 1 : 0;  // 0: from-end, 1: to-end
    const int k = has ? ld.x - e * nl : 0;
    const int kb = I.br0 + k;
    // static data: this end's branch, the bus's offsets (and, at the bus's
    // last lane, its slots, generators and shunt)
    int4 br = make_int4(0, 0, 0, 0), a = make_int4(0, 0, 0, 0), b = make_int4(0, 0, 0, 0);
    int jb = 0, gfirst = -1;
    double2 Yo = make_double2(0.0, 0.0), Yx = make_double2(0.0, 0.0), Yf = make_double2(0.0, 0.0);
    double2 gb = make_double2(0.0, 0.0);
    double r2 = 0.0, tno = 0.0, tnf = 0.0;
    if (has) {
        br = __ldg(d.br + kb);
        if (JAC) {
            const int2 j2 = __ldg(d.br_jb + kb);
            jb = e ? j2.y : j2.x;
        }
        Yo = __ldg((e ? d.y_tt : d.y_ff) + kb);
        Yx = __ldg((e ? d.y_tf : d.y_ft) + kb);
        if (HESS)
            Yf = __ldg((e ? d.y_ft : d.y_tf) + kb);  // the far end's
        if (CONS)
            r2 = __ldg(d.rate2 + kb);
        if (RECT) {  // this lane's angle row limit and the far lane's
            const double2 tb = __ldg(d.tanb + kb);  // tan(angmax), tan(angmin)
            tno = e ? tb.y : tb.x;
            tnf = e ? tb.x : tb.y;
        }
    }
    const int i = ld.y;
    if (valid) {
        const int ib = I.bus0 + i;
        b = __ldg(d.bus_b + ib);
        if (tail) {
            a = __ldg(d.bus_a + ib);
            gb = __ldg(d.gsbs + ib);
            if (CONS && a.z < a.w)
                gfirst = __ldg(d.gen_list + I.gl0 + a.z);
        }
    }
    cudaGridDependencySynchronize();
    cudaTriggerProgrammaticLaunchCompletion();  // the next kernel may launch now

    const int nb = I.nb, ng = I.ng, T = I.T;
    const int nbT = nb * T, ngT = ng * T, nlT = nl * T, na = 2 * nl;
    const int rk = k + nl * t;
    const int f = br.x, bt = br.y;
    const int own = has ? (e ? bt : f) : i, far = e ? f : bt;
    const double *__restrict__ xs = P.x + I.x0;
    const int iva = nb * t, ivm = nbT + nb * t;
    const int ip = 2 * nbT + 2 * ngT + na * t, iq = ip + na * T;
    const int arc = e ? nl + k : k;  // this end's arc
    double vao = 0.0, vax = 0.0, vo = 0.0, vx = 0.0, po = 0.0, qo = 0.0;
    if (valid) {
        vao = __ldg(xs + iva + own);
        vo = __ldg(xs + ivm + own);
    }
    if (has) {
        vax = __ldg(xs + iva + far);
        vx = __ldg(xs + ivm + far);
        if (CONS || JAC || HESS) {
            po = __ldg(xs + ip + arc);
            qo = __ldg(xs + iq + arc);
        }
    }
    double mP = 0, mQ = 0, lth = 0, fP = 0, fQ = 0, ma = 0, fa = 0;
    if (HESS && has) {
        const double *L = P.lam + I.c0 + (T + rk);
        mP = __ldg(L + (e ? 2 * nlT : 0));
        mQ = __ldg(L + (e ? 3 * nlT : nlT));
        lth = __ldg(L + ((e ? 6 : 5) * nlT + 2 * nbT));
        fP = __ldg(L + (e ? 0 : 2 * nlT));  // the far end's flow rows
        fQ = __ldg(L + (e ? nlT : 3 * nlT));
        if (RECT) {  // the angle rows: upper (from-end lane's), lower (to-end lane's)
            ma = __ldg(L + (e ? 7 * nlT + 2 * nbT : 4 * nlT));
            fa = __ldg(L + (e ? 4 * nlT : 7 * nlT + 2 * nbT));
        }
    }
    double lP = 0.0, lQ = 0.0, lV = 0.0, Pd = 0.0, Qd = 0.0, pg1 = 0.0, qg1 = 0.0;
    if (valid && tail) {  // the bus's own dynamic scalars
        if (HESS) {
            const double *L = P.lam + I.c0 + (T + 5 * nlT + nb * t + i);
            lP = __ldg(L);
            lQ = __ldg(L + nbT);
            if (RECT)  // the magnitude row
                lV = __ldg(L + (3 * nlT + 2 * nbT));
        }
        if (CONS) {
            Pd = __ldg(d.Pd + I.pd0 + (nb * t + i));
            Qd = __ldg(d.Qd + I.pd0 + (nb * t + i));
            if (gfirst >= 0) {
                pg1 = __ldg(xs + 2 * nbT + ng * t + gfirst);
                qg1 = __ldg(xs + 2 * nbT + ngT + ng * t + gfirst);
            }
        }
    }

    // the arc end: as one lane of the two-lane branch kernel
    double h1 = 0.0, h2 = 0.0, h3 = 0.0, h4 = 0.0;  // the slot's Hessian parts (the scratch record's)
    if constexpr (RECT) {
        if (has)
            fused_rect_arc<CONS, JAC, HESS>(P, I, e, k, t, own, far, br, jb, Yo, Yx, Yf, r2, tno, tnf, vao, vax, vo,
                                            vx, po, qo, mP, mQ, ma, lth, fP, fQ, fa, grad_here, h1, h2, h3);
    } else {
        const double dlt = vao - vax;  // this end's angle
        double sn = 0.0, cs_ = 1.0;
        if (ROLE == 1) {  // rows warp of a pair: compute and publish
            if (has)
                sincos_tab(dlt, d.trig, &sn, &cs_);
            const int pair = (int)(threadIdx.x >> 6);
            g_role_sc[pair][lane] = make_double2(sn, cs_);
            __syncwarp();
            if (lane == 0)
                cuda::atomic_ref<int, cuda::thread_scope_block>(g_role_flag[pair]).store(1, cuda::memory_order_release);
        } else if (ROLE == 2) {  // Hessian warp of a pair: wait for the rows warp's
            const int pair = (int)(threadIdx.x >> 6);
            int ok = 0;
            if (lane == 0) {
                cuda::atomic_ref<int, cuda::thread_scope_block> f(g_role_flag[pair]);
                for (int i = 0; i < kRoleWaitPolls && !ok; i++)
                    ok = f.load(cuda::memory_order_acquire);
            }
            ok = __shfl_sync(full, ok, 0);
            __syncwarp();  // orders the lanes' reads after lane 0's acquire
            if (ok) {
                const double2 v = g_role_sc[pair][lane];
                sn = v.x;
                cs_ = v.y;
            } else if (has) {
                sincos_tab(dlt, d.trig, &sn, &cs_);
            }
        } else if (has) {
            sincos_tab(dlt, d.trig, &sn, &cs_);
        }
        if (has) {
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
        if (HESS) {
            // U = mP A + mQ B + fP A' + fQ B' (A', B' the far end's, at angle
            // -d) = alpha cos d + beta sin d in this end's angle d, with
            // alpha, beta from the multipliers and admittances only (formed
            // while the sine and cosine are computed); dU/dd = beta cos d -
            // alpha sin d, and d2L/dvm_own dva_own = -vm_far dU/dd
            const double alpha = fma(mP, Yx.x, fma(neg(mQ), Yx.y, fma(fP, Yf.x, neg(fQ * Yf.y))));
            const double beta = fma(mP, Yx.y, fma(mQ, Yx.x, fma(neg(fP), Yf.y, neg(fQ * Yf.x))));
            const double U = fma(alpha, cs_, beta * sn);
            const double Vn = fma(alpha, sn, neg(beta * cs_));  // -dU/dd
            const double We = fma(mP, Yo.x, neg(mQ * Yo.y));
            h1 = vft * U;
            h2 = vx * Vn;
            h3 = neg(twice(We));
            h4 = neg(U);
            double *Hp = P.hess + I.h0 + ((int)(I.hva + I.hvm) * T + ngT + arc + na * t);
            const double l2 = twice(lth);
            Hp[0] = l2;       // (p_arc, p_arc)
            Hp[na * T] = l2;  // (q_arc, q_arc)
        }
        if (P.want_grad && grad_here) {
            P.grad[I.x0 + ip + arc] = 0.0;
            P.grad[I.x0 + iq + arc] = 0.0;
        }
        }  // has
    }

    // segmented sums over the lanes: buses (a bus starts at its head lane;
    // padding lanes are single segments) and groups of parallel arcs (a
    // group starts after a group's last slot; a bus's last slot closes its
    // last group)
    const unsigned upto = (2u << lane) - 1u;  // this lane and the ones below
    const unsigned bheads = __ballot_sync(full, (fl & PK_HEAD) || !valid);
    const int bhead = 31 - __clz(bheads & upto);
    const int bmax = __reduce_max_sync(full, (unsigned)(lane - bhead + 1));
    // bus sums: p, q; polar: the (va, va), (vm, va), (vm, vm) parts;
    // rectangular: the diagonal part
    double tp = po, tq = qo, taa = h1, tma = h2, tmm = RECT ? h1 : h3;
    for (int dd = 1; dd < bmax; dd <<= 1) {
        const bool in = lane - dd >= bhead;
        if (CONS) {
            const double yp = __shfl_up_sync(full, tp, dd), yq = __shfl_up_sync(full, tq, dd);
            if (in) {
                tp += yp;
                tq += yq;
            }
        }
        if (HESS && !RECT) {
            const double ya = __shfl_up_sync(full, taa, dd), ym = __shfl_up_sync(full, tma, dd);
            if (in) {
                taa += ya;
                tma += ym;
            }
        }
        if (HESS) {
            const double yv = __shfl_up_sync(full, tmm, dd);
            if (in)
                tmm += yv;
        }
    }
    const int nd = b.w & 0xffff, nlt = b.w >> 16;
    const int hva = (int)I.hva, hvm = (int)I.hvm;
    double *Hvm = P.hess + I.h0 + (hva * T + hvm * t + b.z);
    double *Hva = P.hess + I.h0 + (hva * t + b.y);
    if (HESS) {
        // group sums: polar (va, va), (vm, va), (vm, vm) parts; rectangular aR, signed aI
        double gaa = RECT ? h2 : h1, gma = RECT ? h3 : h2, gmm = h4;
        const unsigned multi = __ballot_sync(full, has && !(fl & PK_GTAIL));
        if (multi) {  // some group of parallel arcs has more than one slot
            const unsigned gtails = __ballot_sync(full, (fl & PK_GTAIL) || !valid);
            const int ghead = 31 - __clz(((gtails << 1) | 1u) & upto);
            const int gmax = __reduce_max_sync(full, (unsigned)(lane - ghead + 1));
            for (int dd = 1; dd < gmax; dd <<= 1) {
                const double ya = __shfl_up_sync(full, gaa, dd), ym = __shfl_up_sync(full, gma, dd);
                const double yv = RECT ? 0.0 : __shfl_up_sync(full, gmm, dd);
                if (lane - dd >= ghead) {
                    gaa += ya;
                    gma += ym;
                    if (!RECT)
                        gmm += yv;
                }
            }
        }
        if (has && (fl & PK_GTAIL)) {  // the group's off-diagonal entries
            const int grp = ld.w;
            if (RECT) {
                Hvm[grp] = gma;  // (vi_i, vr_j)
                if (fl & PK_LOWER) {
                    Hva[grp] = gaa;       // (vr_i, vr_j), j < i
                    Hvm[nd + grp] = gaa;  // (vi_i, vi_j), j < i
                }
            } else {
                Hvm[grp < nlt ? grp : grp + 1] = neg(gma);  // (vm_i, va_j)
                if (fl & PK_LOWER) {
                    Hva[grp] = neg(gaa);      // (va_i, va_j), j < i
                    Hvm[nd + 1 + grp] = gmm;  // (vm_i, vm_j), j < i
                }
            }
        }
    }
    if (!(valid && tail))
        return;
    // the bus's last lane: its own terms, as in the bus phase (rectangular:
    // vr, vi in the places of va, vm, and the magnitude row)
    const int nsl = a.y - a.x, ng_here = a.w - a.z;
    if (P.want_grad && grad_here) {
        P.grad[I.x0 + iva + i] = 0.0;
        P.grad[I.x0 + ivm + i] = 0.0;
    }
    if (i == I.ref) {  // va_ref, or vi_ref
        if (CONS)
            P.c[I.c0 + t] = RECT ? vo : vao;
        if (JAC)
            P.jac[I.j0 + t] = 1.0;
    }
    if (JAC) {
        const int jP = (int)I.jP;
        double *JP = P.jac + I.j0 + (T + (RECT ? 24 : 22) * nlT + jP * t + b.x);
        double *JQ = JP + jP * T;
        const double v2m = twice(vo);
        if constexpr (RECT) {  // d|V|^2 = (2 vr, 2 vi); the magnitude row
            const double r2m = twice(vao);
            JP[0] = gb.x * r2m;
            JP[1] = gb.x * v2m;
            JQ[0] = neg(gb.y * r2m);
            JQ[1] = neg(gb.y * v2m);
            double *JV = P.jac + I.j0 + (T + 32 * nlT + 2 * jP * T + 2 * (nb * t + i));
            JV[0] = r2m;
            JV[1] = v2m;
        } else {
            JP[0] = gb.x * v2m;
            JQ[0] = neg(gb.y * v2m);
        }
        for (int g = RECT ? 2 : 1; g <= ng_here + (RECT ? 1 : 0); g++) {
            JP[g] = -1.0;
            JQ[g] = -1.0;
        }
    }
    if (CONS) {
        const double vm2 = RECT ? fma(vao, vao, vo * vo) : vo * vo;  // |V|^2
        double Pb = fma(gb.x, vm2, Pd), Qb = fma(neg(gb.y), vm2, Qd);
        if (gfirst >= 0) {
            Pb -= pg1;
            Qb -= qg1;
            for (int gp = a.z + 1; gp < a.w; gp++) {
                const int g = __ldg(d.gen_list + I.gl0 + gp);
                Pb -= __ldg(xs + 2 * nbT + ng * t + g);
                Qb -= __ldg(xs + 2 * nbT + ngT + ng * t + g);
            }
        }
        double *c = P.c + I.c0 + (T + 5 * nlT + nb * t + i);
        c[0] = Pb + tp;
        c[nbT] = Qb + tq;
        if (RECT)
            c[3 * nlT + 2 * nbT] = vm2;  // the magnitude row
    }
    if (HESS && RECT) {  // diagonals (vr_i, vr_i) and (vi_i, vi_i)
        const double dmm = twice(fma(gb.x, lP, fma(neg(gb.y), lQ, lV))) + tmm;
        Hva[nlt] = dmm;
        Hvm[nd + nlt] = dmm;
    } else if (HESS) {
        const double dmm = twice(fma(gb.x, lP, neg(gb.y * lQ))) + tmm;
        if (nsl > 0) {
            Hva[nlt] = taa;
            Hvm[nlt] = tma;
            Hvm[nd + 1 + nlt] = dmm;
        } else {
            Hvm[0] = dmm;
        }
    }
}


template <bool CONS, bool JAC, bool HESS, bool ONE, bool RECT = false, bool STOR = false, bool SPLIT = false,
          bool FUSED = false>
__global__ void __launch_bounds__(kBusBlockMax) bus_kernel(const KParams P)
{
    __shared__ double wsum[32];
    __shared__ bool last;
    if constexpr (SPLIT) {  // the blocks after the thread items take the heavy buses, a warp each
        if ((int)blockIdx.x >= P.split_tblocks) {
            if constexpr (FUSED) {  // or, fused, the packed warps of whole buses
                const int64_t wr = (int64_t)(blockIdx.x - P.split_tblocks) * (blockDim.x >> 5) + (threadIdx.x >> 5);
                if constexpr (HESS && (CONS || JAC)) {
                    if (P.fuse_roles) {  // even warps: rows and Jacobian; odd warps: Hessian
                        // blocks of at least two warps hold both warps of a pair: the
                        // Hessian warp takes the rows warp's sine and cosine (polar)
                        if (!RECT && blockDim.x >= 64) {
                            if (threadIdx.x < kBusBlockMax / 64)
                                g_role_flag[threadIdx.x] = 0;
                            __syncthreads();
                            if (wr & 1)
                                fused_bus_warp<false, false, true, ONE, RECT, 2>(P, wr >> 1, false);
                            else
                                fused_bus_warp<CONS, JAC, false, ONE, RECT, 1>(P, wr >> 1, true);
                        } else if (wr & 1) {
                            fused_bus_warp<false, false, true, ONE, RECT>(P, wr >> 1, false);
                        } else {
                            fused_bus_warp<CONS, JAC, false, ONE, RECT>(P, wr >> 1, true);
                        }
                        return;
                    }
                }
                fused_bus_warp<CONS, JAC, HESS, ONE, RECT>(P, wr, true);
            } else
                heavy_bus_warp<CONS, JAC, HESS, ONE, RECT>(P);
            return;
        }
    }
    const DevArrays &d = P.d;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned tblocks = SPLIT ? (unsigned)P.split_tblocks : gridDim.x;
    const int64_t stride = (int64_t)tblocks * blockDim.x;
    // generator items fill whole blocks when they fit in one pass, so that
    // the blocks holding them (which reduce the objective) hold no bus and
    // finish early: padding items after them do nothing
    const int64_t gpad = P.ngen_items < stride ? (P.ngen_items + blockDim.x - 1) / blockDim.x * blockDim.x
                                               : P.ngen_items;
    const int64_t nbg = (FUSED ? 0 : SPLIT ? P.nlight_items : P.nbus_items) + gpad;
    const int64_t total = nbg + (STOR ? P.nst_items : 0);
    int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;

    struct Item {
        int s, t, e;    // instance, period, bus or generator
        int4 a, b;      // bus: slots, generator entries, row offsets
        int2 m;         // bus: group-closing mask of its slots, number of lower slots
        int2 st;        // bus: (first, end) entry of its storage units (STOR)
        double2 gsbs;
        int gfirst;     // first generator id at the bus, or -1
    };
    // items: generators first (the few blocks holding them do the objective
    // reduction and finish early), then buses, then storage units (unit
    // index in e, its bus in a.x)
    auto load = [&](int64_t item) {
        Item q{};
        q.gfirst = -1;
        if (STOR && item >= nbg && item < total) {
            item -= nbg;
            q.s = ONE ? 0 : find_inst(d.st_items, P.ninst, item);
            const InstDev *I = d.inst + q.s;
            split((int)(item - (ONE ? 0 : __ldg(d.st_items + q.s))), __ldg(&I->ns), __ldg(&I->T), q.t, q.e);
            q.a.x = __ldg(d.st_busid + __ldg(&I->st0) + q.e);
        } else if (item >= gpad && item < nbg) {
            item -= gpad;
            int r, bus0;
            if (SPLIT) {  // the light buses, in id order
                q.s = ONE ? 0 : find_inst(d.light_items, P.ninst, item);
                const InstDev *I = d.inst + q.s;
                split((int)(item - (ONE ? 0 : __ldg(d.light_items + q.s))), __ldg(&I->nlight), __ldg(&I->T), q.t, r);
                bus0 = ONE ? 0 : __ldg(&I->bus0);
                q.e = __ldg(d.light_list + __ldg(&I->light0) + r);
            } else if (ONE) {
                q.s = 0;
                split((int)item, P.inst0.nb, P.inst0.T, q.t, r);
                bus0 = 0;
            } else {
                q.s = find_inst(d.bus_items, P.ninst, item);
                const InstDev *I = d.inst + q.s;
                split((int)(item - __ldg(d.bus_items + q.s)), __ldg(&I->nb), __ldg(&I->T), q.t, r);
                bus0 = __ldg(&I->bus0);
            }
            if (!SPLIT)
                q.e = P.order ? __ldg(P.order + bus0 + r) : r;
            const int ib = bus0 + q.e;
            q.a = __ldg(d.bus_a + ib);
            q.b = __ldg(d.bus_b + ib);
            q.m = __ldg(d.bus_c + ib);
            q.gsbs = __ldg(d.gsbs + ib);
            if (STOR)
                q.st = __ldg(d.bus_st + ib);
            if (CONS && q.a.z < q.a.w)
                q.gfirst = __ldg(d.gen_list + (ONE ? P.inst0.gl0 : __ldg(&d.inst[q.s].gl0)) + q.a.z);
        } else if (item < P.ngen_items) {
            const int64_t gi = item;
            if (ONE) {
                q.s = 0;
                split((int)gi, P.inst0.ng, P.inst0.T, q.t, q.e);
            } else {
                q.s = find_inst(d.gen_items, P.ninst, gi);
                const InstDev *I = d.inst + q.s;
                split((int)(gi - __ldg(d.gen_items + q.s)), __ldg(&I->ng), __ldg(&I->T), q.t, q.e);
            }
        }
        return q;
    };

    Item cur{};
    if (it < total)  // static prologue, overlaps the previous kernel
        cur = load(it);
    cudaGridDependencySynchronize();
    cudaTriggerProgrammaticLaunchCompletion();  // the next kernel may launch now

    double obj_acc = 0.0;
    for (; it < total; it += stride) {
        const Item q = cur;
        if (it + stride < total)
            cur = load(it + stride);
        const InstDev I = inst_of<ONE>(P, q.s);
        const int nl = I.nl, nb = I.nb, ng = I.ng, T = I.T;
        const int nbT = nb * T, ngT = ng * T, nlT = nl * T, na = 2 * nl;
        const double *__restrict__ xs = P.x + I.x0;
        if (STOR && it >= nbg) {
            // one storage unit in one period: its state-of-charge, loss,
            // thermal and complementarity rows, their Jacobian entries, its
            // Hessian entries except the bus's (vm, vm), zero gradient
            const int k = q.e, ns = I.ns, nsT = ns * T, r = k + ns * q.t;
            const int v = 2 * nbT + 2 * ngT + 2 * na * T + r;  // ps of the unit
            const double4_16a par = ldg4(d.st_par + I.st0 + k);  // (dt eta_c, dt / eta_d, r, e_init)
            const double vm = __ldg(xs + nbT + nb * q.t + q.a.x);
            const double ps = __ldg(xs + v), qs = __ldg(xs + v + nsT);
            const double sc = __ldg(xs + v + 2 * nsT), sd = __ldg(xs + v + 3 * nsT);
            const double s2 = fma(ps, ps, qs * qs);
            const double iv2 = 1.0 / (vm * vm);
            if (CONS) {
                const double se = __ldg(xs + v + 4 * nsT);
                const double sp = q.t ? __ldg(xs + v + 4 * nsT - ns) : 0.0;
                double *c = P.c + I.c0 + I.st_c + r;
                c[0] = se - sp - fma(par.x, sc, neg(par.y * sd));
                c[nsT] = ps + sd - sc - par.z * s2 * iv2;
                c[2 * nsT] = s2;
                if (I.st_compl)
                    c[3 * nsT] = sc * sd;
            }
            if (JAC) {
                double *J = P.jac + I.j0 + I.st_j;
                double *Js = J + (q.t ? 3 * ns + 4 * (r - ns) : 3 * k);
                Js[0] = neg(par.x);
                Js[1] = par.y;
                if (q.t) {
                    Js[2] = -1.0;
                    Js[3] = 1.0;
                } else {
                    Js[2] = 1.0;
                }
                double *Jl = J + ns * (4 * T - 1) + 5 * r;
                const double rr = twice(par.z) * iv2;  // 2 r / vm^2
                Jl[0] = rr * s2 / vm;
                Jl[1] = fma(neg(rr), ps, 1.0);
                Jl[2] = neg(rr * qs);
                Jl[3] = -1.0;
                Jl[4] = 1.0;
                double *Jt = J + ns * (4 * T - 1) + 5 * nsT + 2 * r;
                Jt[0] = twice(ps);
                Jt[1] = twice(qs);
                if (I.st_compl) {
                    Jt[2 * nsT] = sd;  // d(sc sd)/dsc
                    Jt[2 * nsT + 1] = sc;
                }
            }
            if (HESS) {
                const double *L = P.lam + I.c0 + I.st_c + r;
                const double rm = par.z * __ldg(L + nsT), lt = __ldg(L + 2 * nsT);
                const double iv3 = iv2 / vm;
                double *Hs = P.hess + I.h0 + I.st_h + 2 * r;
                const double dg = fma(-2.0 * rm, iv2, twice(lt));
                Hs[0] = 4.0 * rm * ps * iv3;  // (ps, vm)
                Hs[1] = dg;                   // (ps, ps)
                Hs[2 * nsT] = 4.0 * rm * qs * iv3;
                Hs[2 * nsT + 1] = dg;
                if (I.st_compl)
                    P.hess[I.h0 + I.st_h + 4 * nsT + r] = __ldg(L + 3 * nsT);  // (sd, sc)
            }
            if (P.want_grad) {
                double *g = P.grad + I.x0 + v;
                for (int w = 0; w < 5; w++)
                    g[w * nsT] = 0.0;
            }
        } else if (it >= gpad) {
            const int i = q.e;
            const int iva = nb * q.t, ivm = nbT + nb * q.t;
            // every dynamic scalar of the bus, issued together (rectangular:
            // vr, vi in the places of va, vm)
            const double vm = __ldg(xs + ivm + i);
            const double vr = RECT ? __ldg(xs + iva + i) : 0.0;
            double lP = 0.0, lQ = 0.0, lV = 0.0, Pd = 0.0, Qd = 0.0, pg1 = 0.0, qg1 = 0.0;
            if (HESS) {
                const double *L = P.lam + I.c0 + (T + 5 * nlT + nb * q.t + i);
                lP = __ldg(L);
                lQ = __ldg(L + nbT);
                if (RECT)  // the magnitude row
                    lV = __ldg(L + (3 * nlT + 2 * nbT));
            }
            if (CONS) {
                Pd = __ldg(d.Pd + I.pd0 + (nb * q.t + i));
                Qd = __ldg(d.Qd + I.pd0 + (nb * q.t + i));
                if (q.gfirst >= 0) {
                    pg1 = __ldg(xs + 2 * nbT + ng * q.t + q.gfirst);
                    qg1 = __ldg(xs + 2 * nbT + ngT + ng * q.t + q.gfirst);
                }
            }
            const double2 gb = q.gsbs;
            const int nsl = q.a.y - q.a.x;
            const int ng_here = q.a.w - q.a.z;
            const double2 *__restrict__ Sg =
                reinterpret_cast<const double2 *>(d.arcs + I.scr0 + (int64_t)na * q.t + q.a.x);
            if (P.want_grad) {
                P.grad[I.x0 + iva + i] = 0.0;
                P.grad[I.x0 + ivm + i] = 0.0;
            }
            if (i == I.ref) {  // va_ref, or vi_ref (rectangular)
                if (CONS)
                    P.c[I.c0 + q.t] = RECT ? vm : __ldg(xs + iva + i);
                if (JAC)
                    P.jac[I.j0 + q.t] = 1.0;
            }
            if (JAC) {  // the arcs' +1 entries are written by the branch phase
                const int jP = (int)I.jP;
                double *JP = P.jac + I.j0 + (T + (RECT ? 24 : 22) * nlT + jP * q.t + q.b.x);
                double *JQ = JP + jP * T;
                const double v2 = twice(vm);
                if constexpr (RECT) {  // d|V|^2 = (2 vr, 2 vi); the magnitude row
                    const double r2 = twice(vr);
                    JP[0] = gb.x * r2;
                    JP[1] = gb.x * v2;
                    JQ[0] = neg(gb.y * r2);
                    JQ[1] = neg(gb.y * v2);
                    double *JV = P.jac + I.j0 + (T + 32 * nlT + 2 * jP * T + 2 * (nb * q.t + i));
                    JV[0] = r2;
                    JV[1] = v2;
                } else {
                    JP[0] = gb.x * v2;
                    JQ[0] = neg(gb.y * v2);
                }
                for (int e = RECT ? 2 : 1; e <= ng_here + (RECT ? 1 : 0); e++) {
                    JP[e] = -1.0;
                    JQ[e] = -1.0;
                }
            }
            double sP = 0.0, sQ = 0.0, sH = 0.0;  // storage: drawn P, Q; (vm, vm) part
            if constexpr (STOR) {
                // storage units at the bus (ascending id): ps and qs are drawn
                // from the bus (balance sums and +1 entries), and each unit's
                // loss term -r (ps^2 + qs^2) / vm^2 adds -6 r mu (ps^2 + qs^2)
                // / vm^4 to the bus's (vm, vm); the rest of a unit's terms is
                // its own item's
                const int ns = I.ns, nsT = ns * T, rt = ns * q.t;
                const int ist = 2 * nbT + 2 * ngT + 2 * na * T;  // first ps
                for (int e = q.st.x; e < q.st.y; e++) {
                    const int k = __ldg(d.st_list + e);
                    if (CONS || HESS) {
                        const double ps = __ldg(xs + ist + k + rt), qs = __ldg(xs + ist + nsT + k + rt);
                        if (CONS) {
                            sP += ps;
                            sQ += qs;
                        }
                        if (HESS) {
                            const double r = __ldg(&d.st_par[I.st0 + k].z);
                            const double mu = __ldg(P.lam + I.c0 + I.st_c + nsT + k + rt);
                            const double iv2 = 1.0 / (vm * vm);
                            sH = fma(-6.0 * r * mu * fma(ps, ps, qs * qs), iv2 * iv2, sH);
                        }
                    }
                    if (JAC) {
                        const int u = 1 + ng_here + nsl + (e - q.st.x);  // after vm, generators, arcs
                        double *JP = P.jac + I.j0 + (T + 22 * nlT + (int)I.jP * q.t + q.b.x);
                        JP[u] = 1.0;
                        JP[(int)I.jP * T + u] = 1.0;
                    }
                }
            }
            if (CONS || HESS) {
                const double vm2 = RECT ? fma(vr, vr, vm * vm) : vm * vm;  // |V|^2
                double Pb = fma(gb.x, vm2, Pd), Qb = fma(neg(gb.y), vm2, Qd);
                if (CONS && q.gfirst >= 0) {
                    Pb -= pg1;
                    Qb -= qg1;
                    for (int gp = q.a.z + 1; gp < q.a.w; gp++) {
                        const int g = __ldg(d.gen_list + I.gl0 + gp);
                        Pb -= __ldg(xs + 2 * nbT + ng * q.t + g);
                        Qb -= __ldg(xs + 2 * nbT + ngT + ng * q.t + g);
                    }
                }
                const int hva = (int)I.hva, hvm = (int)I.hvm;
                double *Hvm = P.hess + I.h0 + (hva * T + hvm * q.t + q.b.z);
                double *Hva = P.hess + I.h0 + (hva * q.t + q.b.y);
                const int nd = q.b.w & 0xffff, nlt = q.b.w >> 16;
                const uint8_t *code = d.slot_code + I.slot0 + q.a.x;
                double daa = 0.0, dma = 0.0, acc_ma = 0.0, acc_aa = 0.0, acc_mm = 0.0;
                // 2 gs lP - 2 bs lQ (+ 2 lV, the magnitude row, rectangular)
                double dmm = HESS ? twice(fma(gb.x, lP, fma(neg(gb.y), lQ, lV))) : 0.0;
                bool first = true;
                int grp = 0;
                // the bus's slots (sorted by far bus), four at a time: the loads
                // of a chunk are all in flight before its arithmetic
                for (int a0 = 0; a0 < nsl; a0 += 4) {
                    double2 v0[4], v1[4], v2[4];
#pragma unroll
                    for (int u = 0; u < 4; u++)
                        if (a0 + u < nsl) {
                            if (CONS)
                                v0[u] = __ldcg(Sg + 3 * (a0 + u));
                            if (HESS) {
                                v1[u] = __ldcg(Sg + 3 * (a0 + u) + 1);
                                v2[u] = __ldcg(Sg + 3 * (a0 + u) + 2);
                            }
                        }
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        const int a = a0 + u;
                        // a warp-uniform exit once no lane has slot a: the
                        // FP64 work of absent slots is then not issued (an
                        // FP64 warp instruction costs the same with any
                        // number of active lanes)
                        if (!__any_sync(__activemask(), a < nsl))
                            break;
                        if (a >= nsl)
                            continue;
                        if (CONS) {
                            Pb += v0[u].x;
                            Qb += v0[u].y;
                        }
                        if (HESS && RECT) {
                            // v1 = (diagonal part, aR), v2.x = signed aI
                            const unsigned cd = nsl <= 32
                                ? (((unsigned)q.m.x >> a) & 1u) | (a < q.m.y ? 2u : 0u)
                                : (unsigned)__ldg(code + a);
                            dmm += v1[u].x;
                            if (__any_sync(__activemask(), !first)) {
                                if (first) {
                                    acc_aa = v1[u].y;
                                    acc_ma = v2[u].x;
                                } else {
                                    acc_aa += v1[u].y;
                                    acc_ma += v2[u].x;
                                }
                            } else {
                                acc_aa = v1[u].y;
                                acc_ma = v2[u].x;
                            }
                            first = (cd & SLOT_LAST) != 0;
                            if (first) {  // a group of parallel arcs ends
                                Hvm[grp] = acc_ma;  // (vi_i, vr_j)
                                if (cd & SLOT_LOWER) {
                                    Hva[grp] = acc_aa;           // (vr_i, vr_j), j < i
                                    Hvm[nd + grp] = acc_aa;      // (vi_i, vi_j), j < i
                                }
                                grp++;
                            }
                        } else if (HESS) {
                            const unsigned cd = nsl <= 32
                                ? (((unsigned)q.m.x >> a) & 1u) | (a < q.m.y ? 2u : 0u)
                                : (unsigned)__ldg(code + a);
                            daa += v1[u].x;
                            dma += v1[u].y;
                            dmm += v2[u].x;
                            // a slot that continues a group of parallel arcs
                            // adds to its sums; the additions issue only in
                            // warps that have such a slot
                            if (__any_sync(__activemask(), !first)) {
                                if (first) {
                                    acc_ma = neg(v1[u].y);
                                    acc_aa = neg(v1[u].x);
                                    acc_mm = v2[u].y;
                                } else {
                                    acc_ma -= v1[u].y;
                                    acc_aa -= v1[u].x;
                                    acc_mm += v2[u].y;
                                }
                            } else {
                                acc_ma = neg(v1[u].y);
                                acc_aa = neg(v1[u].x);
                                acc_mm = v2[u].y;
                            }
                            first = (cd & SLOT_LAST) != 0;
                            if (first) {  // a group of parallel arcs ends: write its entries
                                Hvm[grp < nlt ? grp : grp + 1] = acc_ma;  // (vm_i, va_j)
                                if (cd & SLOT_LOWER) {
                                    Hva[grp] = acc_aa;               // (va_i, va_j), j < i
                                    Hvm[nd + 1 + grp] = acc_mm;      // (vm_i, vm_j), j < i
                                }
                                grp++;
                            }
                        }
                    }
                }
                if (CONS) {
                    double *c = P.c + I.c0 + (T + 5 * nlT + nb * q.t + i);
                    if (STOR) {
                        Pb += sP;
                        Qb += sQ;
                    }
                    c[0] = Pb;
                    c[nbT] = Qb;
                    if (RECT)
                        c[3 * nlT + 2 * nbT] = vm2;  // the magnitude row
                }
                if (HESS && RECT) {  // diagonals (vr_i, vr_i) and (vi_i, vi_i)
                    Hva[nlt] = dmm;
                    Hvm[nd + nlt] = dmm;
                } else if (HESS) {
                    if (STOR)
                        dmm += sH;
                    if (nsl > 0) {
                        Hva[nlt] = daa;
                        Hvm[nlt] = dma;
                        Hvm[nd + 1 + nlt] = dmm;
                    } else {
                        Hvm[0] = dmm;
                    }
                }
            }
        } else if (it < P.ngen_items) {  // (padding items after the generators do nothing)
            const int g = q.e;
            const int ipg = 2 * nbT + ng * q.t + g;
            const int gg = I.gen0 + g;
            const double pg = __ldg(xs + ipg);
            const double c2 = __ldg(d.c2 + gg), c1 = __ldg(d.c1 + gg);
            if (P.want_obj)
                obj_acc += fma(fma(c2, pg, c1), pg, __ldg(d.c0 + gg));
            if (P.want_grad) {
                P.grad[I.x0 + ipg] = fma(twice(c2), pg, c1);
                P.grad[I.x0 + ipg + ngT] = 0.0;
            }
            if (HESS)
                P.hess[I.h0 + ((int)(I.hva + I.hvm) * T + ng * q.t + g)] = P.sigma * twice(c2);
            if ((CONS || JAC) && q.t >= 1 && I.ramp) {
                const int r = g + ng * (q.t - 1);
                if (CONS)
                    P.c[I.c0 + (T + (RECT ? 8 * nlT + 3 * nbT : 7 * nlT + 2 * nbT) + r)] = pg - __ldg(xs + ipg - ng);
                if (JAC) {
                    double *J = P.jac + I.j0 + (T + (RECT ? 32 * nlT + 2 * nbT : 26 * nlT) + 2 * (int)I.jP * T + 2 * r);
                    J[0] = -1.0;
                    J[1] = 1.0;
                }
            }
            if ((CONS || JAC) && I.link_c >= 0) {
                if (CONS)
                    P.c[I.link_c + g] = pg - __ldg(P.x + I.link_x0 + g);
                if (JAC) {
                    double *J = P.jac + I.link_j + 2 * g;
                    J[0] = -1.0;
                    J[1] = 1.0;
                }
            }
        }
    }
    // Objective: fixed-order reduction (warp, block, then the last of the
    // blocks that can hold generator items sums their partials). Only those
    // blocks take part; they come first in the grid.
    const int64_t per_pass = stride;
    unsigned gblocks = P.ngen_items >= per_pass
        ? tblocks : (unsigned)((P.ngen_items + blockDim.x - 1) / blockDim.x);
    if (gblocks == 0)
        gblocks = 1;  // no generators: block 0 still writes the (zero) objective
    if (P.want_obj && blockIdx.x < gblocks) {
        for (int off = 16; off; off >>= 1)
            obj_acc += __shfl_down_sync(0xffffffffu, obj_acc, off);
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
            last = prev == gblocks - 1;
        }
        __syncthreads();
        if (last) {  // the whole last block sums the partials, in a fixed order
            __threadfence();
            double tot = 0.0;
            for (unsigned b = threadIdx.x; b < gblocks; b += blockDim.x)
                tot += __ldcg(d.obj_part + b);
            for (int off = 16; off; off >>= 1)
                tot += __shfl_down_sync(0xffffffffu, tot, off);
            __syncthreads();
            if (lane == 0)
                wsum[warp] = tot;
            __syncthreads();
            if (threadIdx.x == 0) {
                double all = 0.0;
                for (int w = 0; w < (int)(blockDim.x >> 5); w++)
                    all += wsum[w];
                *P.obj = all;
                *d.ticket = 0u;  // ready for the next launch
            }
        }
    }
}

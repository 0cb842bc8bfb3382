// k_aux.cuh: flows, loads, flat start, reserve rows and the table sincos kernel
//
// Part of the translation unit of kernels.cu, which includes it inside
// namespace opf::(anonymous) after k_jt.cuh; not a standalone header.

// p, q of every arc := the flows at the point's voltages (flow rows exactly
// zero), one thread per branch item.
template <bool ONE, bool RECT = false>
__global__ void flows_kernel(const KParams P, double *x)
{
    const DevArrays &d = P.d;
    for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < P.nbr_items;
         it += (int64_t)gridDim.x * blockDim.x) {
        int s, t, k, kb;
        if (ONE) {
            s = 0;
            split((int)it, P.inst0.nl, P.inst0.T, t, k);
            kb = k;
        } else {
            s = find_inst(d.br_items, P.ninst, it);
            split((int)(it - __ldg(d.br_items + s)), __ldg(&d.inst[s].nl), __ldg(&d.inst[s].T), t, k);
            kb = __ldg(&d.inst[s].br0) + k;
        }
        const InstDev I = inst_of<ONE>(P, s);
        const int nl = I.nl, nb = I.nb, ng = I.ng, T = I.T;
        const int nbT = nb * T, ngT = ng * T, na = 2 * nl;
        const BrStatic br = load_br(d, kb, false, false);
        double *xs = x + I.x0;
        const int iva = nb * t, ivm = nbT + nb * t;
        const int ip = 2 * nbT + 2 * ngT + na * t, iq = ip + na * T;
        const double vaf = xs[iva + br.br.x], vat = xs[iva + br.br.y];
        const double vmf = xs[ivm + br.br.x], vmt = xs[ivm + br.br.y];
        if constexpr (RECT) {  // (vr, vi) in the places of (va, vm)
            const double wR = fma(vaf, vat, vmf * vmt), wI = fma(vmf, vat, neg(vaf * vmt));
            const double vf2 = fma(vaf, vaf, vmf * vmf), vt2 = fma(vat, vat, vmt * vmt);
            xs[ip + k] = fma(br.yff.x, vf2, fma(br.yft.x, wR, br.yft.y * wI));
            xs[iq + k] = fma(neg(br.yff.y), vf2, fma(br.yft.x, wI, neg(br.yft.y * wR)));
            xs[ip + nl + k] = fma(br.ytt.x, vt2, fma(br.ytf.x, wR, neg(br.ytf.y * wI)));
            xs[iq + nl + k] = fma(neg(br.ytt.y), vt2, neg(fma(br.ytf.x, wI, br.ytf.y * wR)));
            continue;
        }
        double sn, cs_;
        sincos_tab(vaf - vat, d.trig, &sn, &cs_);
        const double vft = vmf * vmt;
        const double Aft = fma(br.yft.x, cs_, br.yft.y * sn);
        const double Bft = fma(br.yft.x, sn, neg(br.yft.y * cs_));
        const double Atf = fma(br.ytf.x, cs_, neg(br.ytf.y * sn));
        const double Btf = neg(fma(br.ytf.x, sn, br.ytf.y * cs_));
        xs[ip + k] = fma(br.yff.x, vmf * vmf, vft * Aft);
        xs[iq + k] = fma(neg(br.yff.y), vmf * vmf, vft * Bft);
        xs[ip + nl + k] = fma(br.ytt.x, vmt * vmt, vft * Atf);
        xs[iq + nl + k] = fma(neg(br.ytt.y), vmt * vmt, vft * Btf);
    }
}

// Demand per bus and period from per-load values [T][nload] (instance-major):
// the sum over the bus's loads in ascending id, as at model creation.
template <bool ONE>
__global__ void set_loads_kernel(const KParams P, const double *pd, const double *qd)
{
    const DevArrays &d = P.d;
    for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < P.nbus_items;
         it += (int64_t)gridDim.x * blockDim.x) {
        int s, t, i;
        if (ONE) {
            s = 0;
            split((int)it, P.inst0.nb, P.inst0.T, t, i);
        } else {
            s = find_inst(d.bus_items, P.ninst, it);
            split((int)(it - __ldg(d.bus_items + s)), __ldg(&d.inst[s].nb), __ldg(&d.inst[s].T), t, i);
        }
        const InstDev I = inst_of<ONE>(P, s);
        const int l0 = __ldg(d.load_ptr + I.lp0 + i), l1 = __ldg(d.load_ptr + I.lp0 + i + 1);
        const double *ps = pd + I.ld0 + (int64_t)I.nload * t, *qs = qd + I.ld0 + (int64_t)I.nload * t;
        double P_ = 0.0, Q_ = 0.0;
        for (int q = l0; q < l1; q++) {
            const int l = __ldg(d.load_list + I.ll0 + q);
            P_ += ps[l];
            Q_ += qs[l];
        }
        d.Pd[I.pd0 + (int64_t)I.nb * t + i] = P_;
        d.Qd[I.pd0 + (int64_t)I.nb * t + i] = Q_;
    }
}

// Flat start: va = 0, vm = clamp(1), pg, qg at mid-bounds, p, q = flows at
// those voltages (d = 0: cos d = 1, sin d = 0). Rectangular: vr = clamp(1),
// vi = 0, the same point and flows.
__global__ void flat_kernel(const DevArrays d, int32_t ninst, int64_t nbr_items, int64_t nbus_items,
                            int64_t ngen_items, int rect, double *x)
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
            const double v1 = fmin(fmax(1.0, vb.x), vb.y);
            x[xva + i] = rect ? v1 : 0.0;
            x[xva + (int64_t)I->nb * I->T + i] = rect ? 0.0 : v1;
            if (d.bus_st) {  // storage at the bus: idle (ps = qs = sc = sd = 0), se at its initial energy
                const int2 stb = d.bus_st[I->bus0 + i];
                const int64_t ns = I->ns, nsT = ns * I->T;
                const int64_t ist = I->x0 + 2 * ((int64_t)I->nb + I->ng + 2 * (int64_t)I->nl) * I->T;
                for (int e = stb.x; e < stb.y; e++) {
                    const int k = d.st_list[e];
                    const int64_t v = ist + k + ns * t;
                    x[v] = x[v + nsT] = x[v + 2 * nsT] = x[v + 3 * nsT] = 0.0;
                    x[v + 4 * nsT] = d.st_par[I->st0 + k].w;
                }
            }
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

// Reserve rows (sum over an instance's generators of pg in one period), one
// warp per row: lane-strided partial sums, then a fixed shuffle tree; their
// Jacobian entries (+1 for each generator) lane-strided.
__global__ void reserve_kernel(const DevArrays d, int64_t nres, int64_t res_c0, const double *__restrict__ x,
                               double *c, double *jac)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nres; r += warps) {
        const int2 st = __ldg(d.res_st + r);
        const InstDev *I = d.inst + st.x;
        const int ng = __ldg(&I->ng), T = __ldg(&I->T), nb = __ldg(&I->nb);
        if (c) {
            const double *pg = x + __ldg(&I->x0) + 2 * (int64_t)nb * T + (int64_t)ng * st.y;
            double acc = 0.0;
            for (int g = lane; g < ng; g += 32)
                acc += __ldg(pg + g);
            for (int off = 16; off; off >>= 1)
                acc += __shfl_down_sync(0xffffffffu, acc, off);
            if (lane == 0)
                c[res_c0 + r] = acc;
        }
        if (jac) {
            double *J = jac + __ldg(&I->res_j) + (int64_t)ng * st.y;
            for (int g = lane; g < ng; g += 32)
                J[g] = 1.0;
        }
    }
}

__global__ void sincos_tab_kernel(const double2 *__restrict__ tab, const double *__restrict__ d,
                                  int64_t n, double *sn, double *cs)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        sincos_tab(d[i], tab, sn + i, cs + i);
}

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
//  bus phase     one thread per (instance, period, generator) item, then
//                one per (instance, period, bus) item, then (storage models)
//                one per (instance, period, storage unit). Sums the balance
//                rows (the constraint! augmentations of Listing 3), writes
//                their Jacobian rows, assembles the bus's Hessian rows va_i
//                and vm_i from its slots in a fixed order (no atomics), and
//                evaluates the cost, its gradient and Hessian, ramp rows
//                (Listing 6) and linking rows; storage items write their
//                unit's rows and derivatives. The objective is reduced in a
//                fixed order by the last block to finish. A reserve kernel
//                adds the reserve rows of batches that have them.
//
// The rectangular form (vr, vi in the places of va, vm) has its own branch
// kernel and a template variant of the bus kernel; J^T v runs the same two
// phases term by term (and, for the augmented-Lagrangian loop, forms each
// multiplier from its row's value where it reads it).
//
// The fused evaluation (bus_order 3) is one kernel instead of two: whole
// buses packed into warps, one lane per arc end, per-bus sums by segmented
// warp scans (fused_bus_warp); J^T v (fused_jt_warp) and the augmented
// Lagrangian's gradient (al_grad_kernel) have one-kernel forms on the same
// packed warps.
//
// Both kernels are launched with programmatic dependent launch: each block
// first loads the static network data of its first item (which no kernel
// writes), then waits for the previous kernel in the stream to complete
// (cudaGridDependencySynchronize), then reads x, lambda and the scratch. The
// static prologue and the launch therefore overlap the previous kernel. A
// kernel lets the next one launch (cudaTriggerProgrammaticLaunchCompletion)
// only once its own wait is over: triggered at the start, the next kernel's
// blocks took SM slots while this one still waited (16.4 vs 14.7 us per
// fused evaluation of the 10k grid). The trigger only lets the next grid be
// scheduled; its own wait still covers all of this kernel's writes.
//
// FP64 is the scarce resource on the B300 (about 2 FMA per clock per SM), so
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
//
// Rectangular form (form = :rect): with V = vr + j vi and w = V_f conj(V_t),
//   wR = vr_f vr_t + vi_f vi_t,  wI = vi_f vr_t - vr_f vi_t,
//   P_fr =  Gff |V_f|^2 + Gft wR + Bft wI,   Q_fr = -Bff |V_f|^2 + Gft wI - Bft wR,
//   P_to =  Gtt |V_t|^2 + Gtf wR - Btf wI,   Q_to = -Btt |V_t|^2 - Gtf wI - Btf wR,
// and the angle rows are wI - tan(angmax) wR and wI - tan(angmin) wR. Every
// row is a |V_e|^2 + c wR + d wI, whose gradient in (vr_f, vr_t, vi_f, vi_t)
// is (c vr_t - d vi_t, c vr_f + d vi_f, c vi_t + d vr_t, c vi_f - d vr_f)
// plus 2 a V_e on the end's own pair; the Lagrangian of a branch's rows is
// (Df/2) |V_f|^2 + (Dt/2) |V_t|^2 + aR wR + aI wI + linear terms, so its
// Hessian is constant: Df on (vr_f, vr_f) and (vi_f, vi_f), Dt likewise at
// the to-end, aR on (vr_f, vr_t) and (vi_f, vi_t), aI on (vi_f, vr_t) and
// -aI on (vr_f, vi_t).
#include "model.h"

namespace opf {

namespace {

struct KParams {
    DevArrays d;
    InstDev inst0;  // instance 0: the only one when ninst == 1
    int32_t ninst;
    int32_t link;       // linking rows present (J^T v of instance 0's generators)
    int64_t link_c0;    // first linking row
    int32_t want_grad, want_obj;
    int64_t nbr_items, nbus_items, ngen_items;
    int64_t nst_items;  // storage unit items (bus kernel with storage)
    int64_t nlight_items, nheavy_items;  // split bus phase: light-bus items, heavy-bus items
    int64_t npack_items = 0;             // fused evaluation: packed-warp items
    int32_t fuse_roles = 0;              // fused evaluation: two warps (rows, Hessian) per packed warp
    int32_t split_tblocks = 0;  // split bus phase: blocks of generator and light-bus items
    const int32_t *order = nullptr;  // bus-phase order within an instance, or null for id order
    double *xw = nullptr;            // x, writable (branch phase that sets the flows)
    // J^T mu of the augmented Lagrangian: v_i = mu_i = rho (s_i - clip(s_i, gl_i, gu_i)),
    // s_i = c_i + lambda_i / rho, from the rows c (in P.c) and lambda (in P.lam)
    const double *gl = nullptr, *gu = nullptr;
    double rho = 1.0, inv_rho = 1.0;
    double *bp = nullptr;            // the AL step count's bias corrections, advanced once
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

// the descriptor of instance s (kernel parameter for a single instance)
template <bool ONE>
__device__ __forceinline__ InstDev inst_of(const KParams &P, int s)
{
    if (ONE)
        return P.inst0;
    InstDev I;
    const int4 *src = reinterpret_cast<const int4 *>(P.d.inst + s);
    int4 *dst = reinterpret_cast<int4 *>(&I);
#pragma unroll
    for (int w = 0; w < (int)(sizeof(InstDev) / 16); w++)
        dst[w] = __ldg(src + w);
    return I;
}

// -v on the integer pipe (an opaque XOR of the sign bit: a plain negation
// could be rematerialised as an FP64 instruction, the scarce unit here)
__device__ __forceinline__ double neg(double v)
{
    long long r;
    asm("xor.b64 %0, %1, 0x8000000000000000;" : "=l"(r) : "l"(__double_as_longlong(v)));
    return __longlong_as_double(r);
}

// v or -v on the integer pipe
__device__ __forceinline__ double flip(double v, bool f)
{
    long long r;
    asm("xor.b64 %0, %1, %2;"
        : "=l"(r)
        : "l"(__double_as_longlong(v)), "l"(f ? (long long)0x8000000000000000ULL : 0LL));
    return __longlong_as_double(r);
}

// 2 v exactly, on the integer pipe: a normal v gets one more in its exponent
// field; zero and subnormals shift their magnitude left by one (carrying into
// the exponent field where the result becomes normal); the largest binade
// overflows to infinity; infinities and NaNs are returned unchanged.
__device__ __forceinline__ double twice(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned long long sign = b & 0x8000000000000000ULL;
    const unsigned long long mag = b & 0x7fffffffffffffffULL;
    const unsigned ex = (unsigned)(mag >> 52);
    unsigned long long r = b + (1ULL << 52);
    r = ex == 0u ? (sign | (mag << 1)) : r;
    r = ex == 0x7feu ? (sign | 0x7ff0000000000000ULL) : r;
    r = ex == 0x7ffu ? b : r;
    return __longlong_as_double((long long)r);
}

// Table-driven sine and cosine (the table-lookup method of Gal and Bachelis,
// 1991, and of Tang, 1989): d = k h + e with h = 1/kTrigScale, k = rint(d/h)
// (by adding 1.5 * 2^52), e = d - k h (exact, Sterbenz); sin(k h), cos(k h)
// from the table; sin e = e - e^3/6 + e^5/120 and cos e = 1 - e^2/2 + e^4/24,
// whose truncation errors are below 1e-20 for |e| <= 1/256; then
// sin d = sin(kh) cos e + cos(kh) sin e, cos d = cos(kh) cos e - sin(kh) sin e.
// Thirteen FP64 operations. |d| beyond the table falls back to sincos().
__device__ __forceinline__ void sincos_tab(double d, const double2 *__restrict__ tab, double *sn,
                                           double *cs)
{
    const double shift = 6755399441055744.0;  // 1.5 * 2^52
    const double t = fma(d, (double)kTrigScale, shift);
    const int k = __double2loint(t);
    if (k < -kTrigK || k > kTrigK) {
        sincos(d, sn, cs);
        return;
    }
    const double kd = t - shift;
    const double e = fma(kd, -1.0 / kTrigScale, d);
    const double e2 = e * e;
    const double se = fma(e * e2, fma(e2, 1.0 / 120.0, -1.0 / 6.0), e);
    const double ce = fma(e2, fma(e2, 1.0 / 24.0, -0.5), 1.0);
    const double2 tk = __ldg(tab + (k + kTrigK));
    *sn = fma(tk.x, ce, tk.y * se);
    *cs = fma(tk.y, ce, neg(tk.x * se));
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

// put5 for a whole warp whose lanes hold 32 consecutive rows of one group
// (J0 = the first row's entries): the 160 values pass through this warp's
// shared-memory stage and leave as five coalesced 256-byte stores
__device__ __forceinline__ void put5_warp(double *stg, double *J0, int lane, bool f_lo, double vaf, double vat,
                                          double vmf, double vmt)
{
    double *r = stg + 5 * lane;
    r[0] = f_lo ? vaf : vat;
    r[1] = f_lo ? vat : vaf;
    r[2] = f_lo ? vmf : vmt;
    r[3] = f_lo ? vmt : vmf;
    r[4] = 1.0;
    __syncwarp();
#pragma unroll
    for (int m = 0; m < 5; m++)
        J0[lane + 32 * m] = stg[lane + 32 * m];
    __syncwarp();
}

// a double4_16a of read-only data as two 16-byte loads
__device__ __forceinline__ double4_16a ldg4(const double4_16a *p)
{
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    return make_double4_16a(a.x, a.y, b.x, b.y);
}

// static (never written) data of one branch item
struct BrStatic {
    int4 br;  // f, t, slot of the from-arc, slot of the to-arc
    int2 jb;  // the arcs' entries in their buses' balance rows (one period)
    double2 yff, yft, ytf, ytt;
    double r2;
};

__device__ __forceinline__ BrStatic load_br(const DevArrays &d, int kb, bool need_r2, bool need_jb)
{
    BrStatic s;
    s.br = __ldg(d.br + kb);
    s.jb = need_jb ? __ldg(d.br_jb + kb) : make_int2(0, 0);
    s.yff = __ldg(d.y_ff + kb);
    s.yft = __ldg(d.y_ft + kb);
    s.ytf = __ldg(d.y_tf + kb);
    s.ytt = __ldg(d.y_tt + kb);
    s.r2 = need_r2 ? __ldg(d.rate2 + kb) : 0.0;
    return s;
}

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
            c[0] = pf - fma(Yff.x, vf2, vft * Aft);
            c[nlT] = qf - fma(neg(Yff.y), vf2, vft * Bft);
            c[2 * nlT] = pt - fma(Ytt.x, vt2, vft * Atf);
            c[3 * nlT] = qt - fma(neg(Ytt.y), vt2, vft * Btf);
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
// gradient zeros), the other the Hessian; both evaluate the shared
// trigonometry, so the dependent chain of each is shorter at the cost of
// that duplicated work.
template <bool CONS, bool JAC, bool HESS, bool ONE, bool RECT = false>
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
    } else if (has) {
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
            const double Ue = fma(mP, A, mQ * B);
            const double Ve = flip(fma(mQ, A, neg(mP * B)), e);
            // the far end's part: angle -d, admittance Yf, its multipliers
            const double Af = fma(Yf.x, cs_, neg(Yf.y * sn));
            const double Bf = neg(fma(Yf.x, sn, Yf.y * cs_));
            const double Uf = fma(fP, Af, fQ * Bf);
            const double Vf = flip(fma(fQ, Af, neg(fP * Bf)), !e);
            const double U = e ? Uf + Ue : Ue + Uf;  // from-end part first
            const double V = e ? Vf + Ve : Ve + Vf;
            const double We = fma(mP, Yo.x, neg(mQ * Yo.y));
            h1 = vft * U;
            h2 = flip(vx * V, !e);
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
                        if (wr & 1)
                            fused_bus_warp<false, false, true, ONE, RECT>(P, wr >> 1, false);
                        else
                            fused_bus_warp<CONS, JAC, false, ONE, RECT>(P, wr >> 1, true);
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
                        if (a >= nsl)
                            break;
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
                            if (first) {
                                acc_aa = v1[u].y;
                                acc_ma = v2[u].x;
                            } else {
                                acc_aa += v1[u].y;
                                acc_ma += v2[u].x;
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
                            if (first) {
                                acc_ma = neg(v1[u].y);
                                acc_aa = neg(v1[u].x);
                                acc_mm = v2[u].y;
                            } else {
                                acc_ma -= v1[u].y;
                                acc_aa -= v1[u].x;
                                acc_mm += v2[u].y;
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
            const int i = e, ib = I.bus0 + i;
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
            for (int q = 0; q < a.y - a.x; q++) {
                const double2 w = __ldcg(Sg + 3 * q);
                dva += w.x;
                dvm += w.y;
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
cudaError_t dispatch(const KParams &P, bool one, bool occ, bool occ2, bool rect, bool stor, bool run_branch,
                     bool run_bus, int gb, int bb, int gu, int bu, cudaStream_t s, bool splitb, bool fused)
{
    cudaError_t e = cudaSuccess;
    if (fused) {  // one kernel: generator items, then the packed warps (gu counts both)
        if (!run_bus)
            return e;
        if (rect)
            return one ? launch_pdl(bus_kernel<C, J, H, true, true, false, true, true>, gu, bu, s, P)
                       : launch_pdl(bus_kernel<C, J, H, false, true, false, true, true>, gu, bu, s, P);
        return one ? launch_pdl(bus_kernel<C, J, H, true, false, false, true, true>, gu, bu, s, P)
                   : launch_pdl(bus_kernel<C, J, H, false, false, false, true, true>, gu, bu, s, P);
    }
    if (rect) {  // the rectangular branch kernel (two register budgets) and bus variant
        if (run_branch && occ2)  // two threads per branch item (gb counts both)
            e = one ? launch_pdl(rect_branch2_kernel<C, J, H, true>, gb, bb, s, P)
                    : launch_pdl(rect_branch2_kernel<C, J, H, false>, gb, bb, s, P);
        else if (run_branch && occ)
            e = one ? launch_pdl(rect_branch_kernel<C, J, H, true, true>, gb, bb, s, P)
                    : launch_pdl(rect_branch_kernel<C, J, H, false, true>, gb, bb, s, P);
        else if (run_branch)
            e = one ? launch_pdl(rect_branch_kernel<C, J, H, true, false>, gb, bb, s, P)
                    : launch_pdl(rect_branch_kernel<C, J, H, false, false>, gb, bb, s, P);
        if (e != cudaSuccess || !run_bus)
            return e;
        if (splitb)  // light buses a thread each, heavy buses a warp each
            return one ? launch_pdl(bus_kernel<C, J, H, true, true, false, true>, gu, bu, s, P)
                       : launch_pdl(bus_kernel<C, J, H, false, true, false, true>, gu, bu, s, P);
        return one ? launch_pdl(bus_kernel<C, J, H, true, true>, gu, bu, s, P)
                   : launch_pdl(bus_kernel<C, J, H, false, true>, gu, bu, s, P);
    }
    if (run_branch && occ2) {  // two threads per branch item (gb counts both)
        e = one ? launch_pdl(branch2_kernel<C, J, H, true>, gb, bb, s, P)
                : launch_pdl(branch2_kernel<C, J, H, false>, gb, bb, s, P);
    } else if (run_branch) {
        if (occ)
            e = one ? launch_pdl(branch_kernel<C, J, H, true, true>, gb, bb, s, P)
                    : launch_pdl(branch_kernel<C, J, H, false, true>, gb, bb, s, P);
        else
            e = one ? launch_pdl(branch_kernel<C, J, H, true, false>, gb, bb, s, P)
                    : launch_pdl(branch_kernel<C, J, H, false, false>, gb, bb, s, P);
    }
    if (e != cudaSuccess || !run_bus)
        return e;
    if (stor)  // storage units (polar only)
        return one ? launch_pdl(bus_kernel<C, J, H, true, false, true>, gu, bu, s, P)
                   : launch_pdl(bus_kernel<C, J, H, false, false, true>, gu, bu, s, P);
    if (splitb)  // light buses a thread each, then heavy buses a warp each (gu counts both)
        return one ? launch_pdl(bus_kernel<C, J, H, true, false, false, true>, gu, bu, s, P)
                   : launch_pdl(bus_kernel<C, J, H, false, false, false, true>, gu, bu, s, P);
    return one ? launch_pdl(bus_kernel<C, J, H, true>, gu, bu, s, P)
               : launch_pdl(bus_kernel<C, J, H, false>, gu, bu, s, P);
}

// Launches one fused evaluation with the given scratch.
int launch_all(Model &M, const EvalArgs &a, unsigned what, cudaStream_t s, int phases,
               ArcScratch *arcs, double *obj_part, int max_part, unsigned int *ticket)
{
    KParams P;
    P.d = M.d;
    P.d.arcs = arcs;
    P.d.obj_part = obj_part;
    P.d.ticket = ticket;
    P.inst0 = M.inst[0];
    P.ninst = M.ninst;
    P.link = M.link ? 1 : 0;
    P.link_c0 = M.link_c0;
    P.nbr_items = M.nbr_items;
    P.nbus_items = M.nbus_items;
    P.ngen_items = M.ngen_items;
    P.nst_items = M.nst_items;
    P.nlight_items = M.nlight_items;
    P.nheavy_items = M.nheavy_items;
    P.x = a.x;
    P.lam = a.lam;
    P.sigma = a.sigma;
    P.obj = a.obj;
    P.grad = a.grad;
    P.c = a.c;
    P.jac = a.jac;
    P.hess = a.hess;
    const bool C = what & W_CONS, J = what & W_JAC, H = what & W_HESS;
    P.want_grad = (what & W_GRAD) ? 1 : 0;
    P.want_obj = (what & W_OBJ) ? 1 : 0;
    const opf_launch &L = M.launch;
    const int bu = L.bus_block > kBusBlockMax ? kBusBlockMax : L.bus_block;
    const int gb = grid_for(M.nbr_items, L.branch_block, L.branch_ctas_per_sm, M.num_sms, 0);
    const int cap = max_part < M.max_part ? max_part : M.max_part;
    // the bus kernel pads the generator items to whole blocks (when they fit
    // in one pass of the grid): size the grid for the padded count
    const int64_t gpad = (M.ngen_items + bu - 1) / bu * bu;
    const int gu = grid_for(M.nbus_items + gpad + M.nst_items, bu, L.bus_ctas_per_sm, M.num_sms, cap);
    // the branch phase is needed for its rows and for the scratch the bus
    // phase reads (balance sums, Hessian), and to zero the p, q gradient
    const bool run_branch = (phases & 1) && (C || J || H || P.want_grad) && M.nbr_items > 0;
    const bool run_bus = phases & 2;
    const bool one = M.ninst == 1;
    const bool occ = L.branch_occupancy == 1;
    // branch_occupancy 2: two threads per branch item
    const bool occ2 = L.branch_occupancy == 2;
    const int gb2 = occ2 ? grid_for(2 * M.nbr_items, L.branch_block, L.branch_ctas_per_sm, M.num_sms, 0) : gb;
    const int bb = L.branch_block;
    P.order = L.bus_order == 1 ? M.d.bus_order : nullptr;
    // bus_order 2: the split bus phase where it applies (models without storage):
    // light buses a thread each in the first blocks, heavy buses a warp each
    // in the blocks after them; elsewhere buses in id order
    const bool splitb = L.bus_order >= 2 && M.split_ok && (phases & 2);
    // bus_order 3: the fused evaluation where it applies (no storage,
    // at most 32 arc slots per bus), one kernel per evaluation (launched
    // with the bus phase; the branch phase alone launches nothing)
    const bool fused = L.bus_order == 3 && M.fuse_ok;
    int gu_all = gu;
    if (fused) {
        const int tb = grid_for(gpad, bu, L.bus_ctas_per_sm, M.num_sms, cap);
        P.split_tblocks = tb;
        P.npack_items = M.npack_items;
        // two roles only where there is both a Hessian and rows or Jacobian to write
        P.fuse_roles = L.branch_occupancy == 2 && H && (C || J) ? 1 : 0;
        const int64_t warps = M.npack_items * (P.fuse_roles ? 2 : 1);
        gu_all = tb + (int)((warps + bu / 32 - 1) / (bu / 32));
    } else if (splitb) {
        const int tb = grid_for(M.nlight_items + gpad, bu, L.bus_ctas_per_sm, M.num_sms, cap);
        P.split_tblocks = tb;
        gu_all = tb + (int)((M.nheavy_items + bu / 32 - 1) / (bu / 32));
    }
    cudaError_t e;
    switch ((C ? 1 : 0) | (J ? 2 : 0) | (H ? 4 : 0)) {
    case 0: e = dispatch<false, false, false>(P, one, occ, occ2, M.rect, M.storage, run_branch, run_bus, gb2, bb, gu_all, bu, s, splitb, fused); break;
    case 1: e = dispatch<true, false, false>(P, one, occ, occ2, M.rect, M.storage, run_branch, run_bus, gb2, bb, gu_all, bu, s, splitb, fused); break;
    case 2: e = dispatch<false, true, false>(P, one, occ, occ2, M.rect, M.storage, run_branch, run_bus, gb2, bb, gu_all, bu, s, splitb, fused); break;
    case 3: e = dispatch<true, true, false>(P, one, occ, occ2, M.rect, M.storage, run_branch, run_bus, gb2, bb, gu_all, bu, s, splitb, fused); break;
    case 4: e = dispatch<false, false, true>(P, one, occ, occ2, M.rect, M.storage, run_branch, run_bus, gb2, bb, gu_all, bu, s, splitb, fused); break;
    case 5: e = dispatch<true, false, true>(P, one, occ, occ2, M.rect, M.storage, run_branch, run_bus, gb2, bb, gu_all, bu, s, splitb, fused); break;
    case 6: e = dispatch<false, true, true>(P, one, occ, occ2, M.rect, M.storage, run_branch, run_bus, gb2, bb, gu_all, bu, s, splitb, fused); break;
    default: e = dispatch<true, true, true>(P, one, occ, occ2, M.rect, M.storage, run_branch, run_bus, gb2, bb, gu_all, bu, s, splitb, fused); break;
    }
    if (e == cudaSuccess && M.reserve && (C || J) && (phases & 2)) {
        const int64_t threads = 32 * M.nres;
        reserve_kernel<<<(int)((threads + 255) / 256), 256, 0, s>>>(M.d, M.nres, M.res_c0, a.x, C ? a.c : nullptr,
                                                                    J ? a.jac : nullptr);
    }
    if (e == cudaSuccess)
        e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("kernel launch failed: %s", cudaGetErrorString(e));
        return OPF_ECUDA;
    }
    return OPF_OK;
}

}  // namespace

int launch_eval(Model &M, const EvalArgs &a, unsigned what, cudaStream_t s, int phases)
{
    return launch_all(M, a, what, s, phases, M.d.arcs, M.d.obj_part, M.max_part, M.d.ticket);
}

// The fused evaluation with caller-chosen scratch (arc slots, objective
// partials, block counter) in place of the model's own; used by
// opf_eval_all_noalloc. Same kernels and launch shape as launch_eval.
int launch_eval_scratch(Model &M, const EvalArgs &a, unsigned what, cudaStream_t s,
                        ArcScratch *arcs, double *obj_part, int max_part, unsigned int *ticket)
{
    return launch_all(M, a, what, s, 3, arcs, obj_part, max_part, ticket);
}

int launch_sincos(Model &M, const double *d, int64_t n, double *sn, double *cs, cudaStream_t s)
{
    const int grid = grid_for(n, 256, 8, M.num_sms, 0);
    sincos_tab_kernel<<<grid, 256, 0, s>>>(M.d.trig, d, n, sn, cs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("kernel launch failed: %s", cudaGetErrorString(e));
        return OPF_ECUDA;
    }
    return OPF_OK;
}

namespace {
KParams base_params(Model &M)
{
    KParams P{};
    P.d = M.d;
    P.inst0 = M.inst[0];
    P.ninst = M.ninst;
    P.link = M.link ? 1 : 0;
    P.link_c0 = M.link_c0;
    P.nbr_items = M.nbr_items;
    P.nbus_items = M.nbus_items;
    P.ngen_items = M.ngen_items;
    P.nst_items = M.nst_items;
    P.nlight_items = M.nlight_items;
    P.nheavy_items = M.nheavy_items;
    return P;
}

int launch_status()
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("kernel launch failed: %s", cudaGetErrorString(e));
        return OPF_ECUDA;
    }
    return OPF_OK;
}
}  // namespace

namespace {
template <bool AL>
int jtprod_launch(Model &M, const KParams &P, cudaStream_t s)
{
    const int gb = grid_for(M.nbr_items, 128, 0, M.num_sms, 0);
    const int gu = grid_for(M.nbus_items + M.ngen_items, 128, 0, M.num_sms, 0);
    const bool one = M.ninst == 1;
    cudaError_t e = cudaSuccess;
    if (M.launch.bus_order == 3 && M.fuse_ok) {  // the fused evaluation's layout: one kernel
        const int bu = M.launch.bus_block > kBusBlockMax ? kBusBlockMax : M.launch.bus_block;
        KParams Q = P;
        Q.split_tblocks = grid_for(M.ngen_items, bu, M.launch.bus_ctas_per_sm, M.num_sms, 0);
        Q.npack_items = M.npack_items;
        const int grid = Q.split_tblocks + (int)((M.npack_items + bu / 32 - 1) / (bu / 32));
        if (M.rect)
            e = one ? launch_pdl(jt_fused_kernel<true, true, AL>, grid, bu, s, Q)
                    : launch_pdl(jt_fused_kernel<false, true, AL>, grid, bu, s, Q);
        else
            e = one ? launch_pdl(jt_fused_kernel<true, false, AL>, grid, bu, s, Q)
                    : launch_pdl(jt_fused_kernel<false, false, AL>, grid, bu, s, Q);
    } else if (M.rect) {
        if (M.nbr_items > 0)
            e = one ? launch_pdl(jt_branch_kernel<true, true, AL>, gb, 128, s, P)
                    : launch_pdl(jt_branch_kernel<false, true, AL>, gb, 128, s, P);
        if (e == cudaSuccess)
            e = one ? launch_pdl(jt_bus_kernel<true, true, false, AL>, gu, 128, s, P)
                    : launch_pdl(jt_bus_kernel<false, true, false, AL>, gu, 128, s, P);
    } else {
        if (M.nbr_items > 0)
            e = one ? launch_pdl(jt_branch_kernel<true, false, AL>, gb, 128, s, P)
                    : launch_pdl(jt_branch_kernel<false, false, AL>, gb, 128, s, P);
        if (e == cudaSuccess && M.storage)
            e = one ? launch_pdl(jt_bus_kernel<true, false, true, AL>, gu, 128, s, P)
                    : launch_pdl(jt_bus_kernel<false, false, true, AL>, gu, 128, s, P);
        else if (e == cudaSuccess)
            e = one ? launch_pdl(jt_bus_kernel<true, false, false, AL>, gu, 128, s, P)
                    : launch_pdl(jt_bus_kernel<false, false, false, AL>, gu, 128, s, P);
    }
    if (e != cudaSuccess) {
        set_error("kernel launch failed: %s", cudaGetErrorString(e));
        return OPF_ECUDA;
    }
    return launch_status();
}
}  // namespace

int launch_jtprod(Model &M, const double *x, const double *v, double *out, cudaStream_t s)
{
    KParams P = base_params(M);
    P.x = x;
    P.lam = v;
    P.grad = out;
    return jtprod_launch<false>(M, P, s);
}

// out = J^T mu with the augmented Lagrangian's mu_i = rho (s_i - clip(s_i,
// gl_i, gu_i)), s_i = c_i + lambda_i / rho, computed where each entry is
// read from the rows c at x (no mu vector); advances the step state bp
int launch_jtprod_al(Model &M, const double *x, const double *c, const double *lam, const double *gl,
                     const double *gu, double rho, double *out, double *bp, cudaStream_t s)
{
    KParams P = base_params(M);
    P.x = x;
    P.lam = lam;
    P.c = const_cast<double *>(c);  // read only in this mode
    P.gl = gl;
    P.gu = gu;
    P.rho = rho;
    P.inv_rho = 1.0 / rho;
    P.bp = bp;
    P.grad = out;
    return jtprod_launch<true>(M, P, s);
}

bool al_grad_fused_ok(const Model &M)
{
    return M.launch.bus_order == 3 && M.fuse_ok && !M.rect && !M.link && !M.reserve;
}

// out = grad f + J^T mu of the augmented Lagrangian in one kernel (see
// al_grad_kernel); only where al_grad_fused_ok
int launch_al_grad(Model &M, const double *x, const double *lam, const double *gl, const double *gu, double rho,
                   double *out, double *bp, cudaStream_t s)
{
    KParams P = base_params(M);
    P.x = x;
    P.lam = lam;
    P.gl = gl;
    P.gu = gu;
    P.rho = rho;
    P.inv_rho = 1.0 / rho;
    P.bp = bp;
    P.grad = out;
    P.npack_items = M.npack_items;
    const int bu = M.launch.bus_block > kBusBlockMax ? kBusBlockMax : M.launch.bus_block;
    const int grid = (int)((M.npack_items + bu / 32 - 1) / (bu / 32));
    cudaError_t e = M.ninst == 1 ? launch_pdl(al_grad_kernel<true>, grid < 1 ? 1 : grid, bu, s, P)
                                 : launch_pdl(al_grad_kernel<false>, grid < 1 ? 1 : grid, bu, s, P);
    if (e != cudaSuccess) {
        set_error("kernel launch failed: %s", cudaGetErrorString(e));
        return OPF_ECUDA;
    }
    return launch_status();
}

int launch_cons_setflows(Model &M, double *x, double *obj, double *grad, double *c, cudaStream_t s)
{
    if (M.ninst != 1 || M.rect) {
        set_error("launch_cons_setflows: single-instance polar models only");
        return OPF_ESTATE;
    }
    KParams P = base_params(M);
    P.x = x;
    P.xw = x;
    P.lam = nullptr;
    P.sigma = 1.0;
    P.obj = obj;
    P.grad = grad;
    P.c = c;
    P.jac = nullptr;
    P.hess = nullptr;
    P.want_grad = grad ? 1 : 0;
    P.want_obj = obj ? 1 : 0;
    cudaError_t e = cudaSuccess;
    if (M.nbr_items > 0)
        e = launch_pdl(branch_kernel<true, false, false, true, false, true>,
                       grid_for(M.nbr_items, 128, 0, M.num_sms, 0), 128, s, P);
    if (e == cudaSuccess)
        e = launch_pdl(bus_kernel<true, false, false, true>,
                       grid_for(M.nbus_items + (M.ngen_items + 127) / 128 * 128, 128, 0, M.num_sms, M.max_part), 128,
                       s, P);
    if (e != cudaSuccess) {
        set_error("kernel launch failed: %s", cudaGetErrorString(e));
        return OPF_ECUDA;
    }
    return launch_status();
}

int launch_flows(Model &M, double *x, cudaStream_t s)
{
    if (M.nbr_items == 0)
        return OPF_OK;
    KParams P = base_params(M);
    const int grid = grid_for(M.nbr_items, 128, 0, M.num_sms, 0);
    if (M.rect && M.ninst == 1)
        flows_kernel<true, true><<<grid, 128, 0, s>>>(P, x);
    else if (M.rect)
        flows_kernel<false, true><<<grid, 128, 0, s>>>(P, x);
    else if (M.ninst == 1)
        flows_kernel<true><<<grid, 128, 0, s>>>(P, x);
    else
        flows_kernel<false><<<grid, 128, 0, s>>>(P, x);
    return launch_status();
}

int launch_set_loads(Model &M, const double *pd, const double *qd, cudaStream_t s)
{
    KParams P = base_params(M);
    const int grid = grid_for(M.nbus_items, 128, 0, M.num_sms, 0);
    if (M.ninst == 1)
        set_loads_kernel<true><<<grid, 128, 0, s>>>(P, pd, qd);
    else
        set_loads_kernel<false><<<grid, 128, 0, s>>>(P, pd, qd);
    return launch_status();
}

int launch_flat_start(Model &M, double *x, cudaStream_t s)
{
    const int64_t total = M.nbr_items + M.nbus_items + M.ngen_items;
    const int block = 256;
    const int grid = grid_for(total, block, 8, M.num_sms, 0);
    flat_kernel<<<grid, block, 0, s>>>(M.d, M.ninst, M.nbr_items, M.nbus_items, M.ngen_items, M.rect ? 1 : 0, x);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("kernel launch failed: %s", cudaGetErrorString(e));
        return OPF_ECUDA;
    }
    return OPF_OK;
}

}  // namespace opf

// k_common.cuh: kernel parameters and the helpers every evaluation kernel uses
//
// Part of the translation unit of kernels.cu, which includes it inside
// namespace opf::(anonymous) after model.h; not a standalone header.

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

#include "bits.cuh"  // twice (and the other integer-pipe helpers)

// ---- FP32 <-> FP64 on the integer pipe (the conversion instructions run at
// the FP64 rate, the scarce unit here)

// v > 0 (or 0) truncated to FP32 (relative error below 2^-23); values below
// the FP32 normal range give 0
__device__ __forceinline__ float f32_of_pos(double v)
{
    const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
    if (hi < (897u << 20))
        return 0.0f;
    return __uint_as_float(((hi - (896u << 20)) << 3) | (lo >> 29));
}

// exact widening of a normal FP32 value (zero and subnormals give 0)
__device__ __forceinline__ double f64_of(float f)
{
    const unsigned b = __float_as_uint(f);
    const unsigned ex = (b >> 23) & 0xffu;
    const unsigned hi = (b & 0x80000000u) | ((ex + 896u) << 20) | ((b & 0x7fffffu) >> 3);
    const unsigned lo = b << 29;
    return ex == 0u ? 0.0 : __hiloint2double((int)hi, (int)lo);
}

// k / kTrigScale exactly, for |k| < 2048
__device__ __forceinline__ double k_over_scale(int k)
{
    const unsigned a = (unsigned)(k < 0 ? -k : k);
    const int nbit = 31 - __clz((int)(a | 1u));  // position of the leading bit
    const unsigned mant = (a << (20 - nbit)) & 0xfffffu;
    const unsigned hi = (k < 0 ? 0x80000000u : 0u) | ((unsigned)(1023 + nbit - 8) << 20) | mant;
    return a == 0u ? 0.0 : __hiloint2double((int)hi, 0);
}
static_assert(kTrigScale == 256, "k_over_scale divides by 2^8");

// CUDA's sincos, kept out of line: the rare path of sincos_tab (its argument
// reduction is long and would otherwise be inlined at every call site)
__device__ __noinline__ void sincos_far(double d, double *sn, double *cs)
{
    sincos(d, sn, cs);
}

// Table-driven sine and cosine (the table-lookup method of Tang, 1989, and
// of Gal and Bachelis, 1991): d = k h + e with h = 1/256, k = rint(d / h)
// (by adding 1.5 * 2^52 to 256 d), e = d - k h (exact, Sterbenz), |e| <= 1/512;
//   sin e = e + e^3 c,  c = -1/6 + e^2/120,
//   cos e = 1 + q,      q = -e^2/2 + e^4/24,
// with c and e^4/24 in FP32 (absolute errors below 1e-8 in c, so below 4e-17
// in e^3 c, and below 1e-19 in e^4/24), e^2, e^3 and the rest in FP64; the
// series' truncation is below 1e-21; then
//   sin d = S + S q + C sin e,  cos d = C + C q - S sin e
// with (S, C) = (sin kh, cos kh) from the table. Ten FP64 operations.
// |d| >= 3.140625 (or NaN) falls back to CUDA's sincos.
__device__ __forceinline__ void sincos_tab(double d, const double2 *__restrict__ tab, double *sn,
                                           double *cs)
{
    if (((unsigned)__double2hiint(d) & 0x7fffffffu) >= 0x40092000u) {  // |d| >= 3.140625
        sincos_far(d, sn, cs);
        return;
    }
    const double t = fma(d, (double)kTrigScale, 6755399441055744.0);  // + 1.5 * 2^52
    const int k = __double2loint(t);
    const double2 tk = __ldg(tab + (k + kTrigK));
    const double e = d - k_over_scale(k);
    const double e2 = e * e;
    const float z = f32_of_pos(e2);
    const float cf = fmaf(z, 1.0f / 120.0f, -1.0f / 6.0f);
    const float rf = (z * z) * (1.0f / 24.0f);
    const double se = fma(e * e2, f64_of(cf), e);
    const double q = fma(e2, -0.5, f64_of(rf));
    *sn = fma(tk.y, se, fma(tk.x, q, tk.x));
    *cs = fma(neg(tk.x), se, fma(tk.y, q, tk.y));
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

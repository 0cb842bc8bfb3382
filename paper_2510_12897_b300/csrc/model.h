// Internal structures of libopf (host and device). Not part of the C ABI.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/opf.h"

namespace opf {

// Callback selection of one fused evaluation.
enum : unsigned { W_OBJ = 1u, W_GRAD = 2u, W_CONS = 4u, W_JAC = 8u, W_HESS = 16u };

// Per-arc scratch written by the branch phase at the arc's slot in its bus's
// arc list and read back, in that order, by the bus phase. i = the arc's bus,
// j = its far bus; L = the Lagrangian restricted to the branch's flow rows.
//   p, q    the arc's flow variables (balance sums)
//   d_aa    d2L/dva_i^2        (d2L/dva_i dva_j = -d_aa)
//   d_ma    d2L/dvm_i dva_i    (d2L/dvm_i dva_j = -d_ma)
//   d_mm    d2L/dvm_i^2
//   x_mm    d2L/dvm_i dvm_j
// In the rectangular form the last four fields hold instead
//   d_aa    d2L/dvr_i^2 (= d2L/dvi_i^2)
//   d_ma    d2L/dvr_i dvr_j (= d2L/dvi_i dvi_j)
//   d_mm    d2L/dvi_i dvr_j (d2L/dvr_i dvi_j is its negation)
//   x_mm    unused
struct __align__(16) ArcScratch {
    double p, q, d_aa, d_ma, d_mm, x_mm;
};

// Table of the table-driven sine/cosine of the branch kernel: (sin, cos) at
// k / kTrigScale for |k| <= kTrigK, which covers |d| <= pi.
constexpr int kTrigScale = 256;
constexpr int kTrigK = 804;

// split bus phase: buses with more arc slots than this (and at most 32) are
// handled by a warp each, one lane per slot (6 measured best on the 10k
// grid, among 4, 6, 8 and 10: a thread walks at most two chunks of slots)
constexpr int kLightSlots = 6;

// slot codes: the slot closes its far bus's group / the far bus is lower
enum : uint8_t { SLOT_LAST = 1u, SLOT_LOWER = 2u };

// fused evaluation (bus_order 3): whole buses packed into warps, one lane per
// arc slot (a bus without arcs takes one lane). Per lane an int4 (arc id or
// -1, local bus, flags, group index of the slot within its bus); flags:
enum : int32_t { PK_VALID = 1, PK_HEAD = 2, PK_TAIL = 4, PK_GTAIL = 8, PK_LOWER = 16 };

// One instance of a batch, as seen by the kernels. Offsets are absolute
// positions in the caller's x / g / Jacobian / Hessian arrays and in the
// model's concatenated network arrays.
struct __align__(16) InstDev {
    int32_t nb, nl, ng, T;
    int32_t ref;        // local reference bus
    int32_t ramp;       // ramp rows present
    int32_t br0;        // first branch in the concatenated branch arrays
    int32_t bus0;       // first bus in the concatenated bus arrays
    int32_t gen0;       // first generator
    int32_t gl0;        // first entry of this instance's bus->generator list
    int32_t slot0;      // first slot code of this instance (2 nl per instance)
    int32_t nload;      // loads of this instance
    int32_t lp0;        // first entry of this instance's bus->load pointers (nb + 1)
    int32_t ll0;        // first entry of this instance's bus->load list
    int32_t st_compl;   // storage complementarity rows present
    int32_t pad2;
    int64_t x0, c0, j0, h0;
    int64_t ld0;        // first entry of this instance's loads in opf_set_loads arrays [T][nload]
    int64_t scr0;       // first arc-scratch slot (2 nl T slots per instance)
    int64_t pd0;        // first entry of per-bus demand [T][nb]
    int64_t jP;         // Jacobian entries of one period of the P-balance group (nb + ng + 2 nl)
    int64_t hva, hvm;   // Hessian entries of one period of the va rows / vm rows
    int64_t link_c, link_j;  // this instance's linking rows and their Jacobian offset; -1 if none
    int64_t link_x0;    // first pg of instance 0 (linking partner)
    int64_t res_c, res_j;  // this instance's reserve rows (one per period) and their Jacobian offset; -1 if none
    int64_t st_c, st_j, st_h;  // storage: first row, Jacobian value, Hessian value, inside the instance
    int32_t ns;         // storage units
    int32_t st0;        // first unit in the concatenated storage arrays
    int32_t nlight, light0;  // split bus phase: buses one per thread (count, first list entry)
    int32_t nheavy, heavy0;  // split bus phase: buses one per warp (more than kLightSlots slots)
    int32_t npack, pack0;    // fused evaluation: packed warps of one period (count, first warp)
};
static_assert(sizeof(InstDev) % 16 == 0, "InstDev is loaded as int4 words");

struct DevArrays {
    int2 *res_st = nullptr;       // per reserve row: (instance, period)
    int32_t *bus_order = nullptr; // per instance: buses by arc count, warps dealt heavy / light
    // branches (concatenated over instances)
    int4 *br = nullptr;           // local (f, t, slot of the from-arc, slot of the to-arc)
    int2 *br_jb = nullptr;        // entries of the from-arc and to-arc in their buses' balance
                                  // rows, inside one period's balance-row group
    double2 *y_ff = nullptr, *y_ft = nullptr, *y_tf = nullptr, *y_tt = nullptr;  // (G, B)
    double *rate2 = nullptr;      // rate_a^2
    double2 *tanb = nullptr;      // (tan angmax, tan angmin), rectangular form only
    // buses
    int4 *bus_a = nullptr;        // (first slot, end slot, first gen entry, end gen entry)
    int4 *bus_b = nullptr;        // (balance-row offset, va-row offset, vm-row offset,
                                  //  distinct far buses | lower ones << 16) inside one period
    int2 *bus_c = nullptr;        // (bit j: slot j closes its group of parallel arcs, for
                                  //  buses with <= 32 slots; slots whose far bus is lower)
    double2 *gsbs = nullptr;      // (gs, bs)
    uint8_t *slot_code = nullptr; // per slot: SLOT_LAST / SLOT_LOWER (buses with > 32 slots)
    double2 *trig = nullptr;      // (sin, cos) of k / kTrigScale, k = -kTrigK..kTrigK
    int32_t *gen_list = nullptr;  // local generator ids, ascending per bus
    double *Pd = nullptr, *Qd = nullptr;  // demand per bus and period
    int32_t *load_ptr = nullptr;  // CSR bus -> loads, nb + 1 per instance
    int32_t *load_list = nullptr; // local load ids, ascending per bus
    // generators
    int32_t *gen_busid = nullptr; // local bus of each generator
    double *c2 = nullptr, *c1 = nullptr, *c0 = nullptr;
    double2 *pbnd = nullptr, *qbnd = nullptr;  // (min, max), flat start only
    double2 *vbnd = nullptr;                   // (vmin, vmax) per bus, flat start only
    // storage (multi-period model with storage)
    int2 *bus_st = nullptr;       // per bus: (first, end) entry of its units in st_list
    int32_t *st_list = nullptr;   // local unit ids, ascending per bus
    double4_16a *st_par = nullptr;    // per unit: (dt eta_c, dt / eta_d, r, e_init)
    int32_t *st_busid = nullptr;  // per unit: its local bus
    // split bus phase: light buses (one thread each) and heavy buses (one
    // warp each), local ids ascending per instance, and their item prefixes
    int32_t *light_list = nullptr, *heavy_list = nullptr;
    int64_t *light_items = nullptr, *heavy_items = nullptr;
    // fused evaluation: 32 lane words per packed warp, and the prefix of
    // packed-warp items (npack T) over instances
    int4 *pack = nullptr;
    int64_t *pack_items = nullptr;
    int64_t *st_items = nullptr;  // prefix of storage items (ns T) over instances, ninst + 1
    // instances and work lists
    InstDev *inst = nullptr;
    int64_t *br_items = nullptr;   // prefix of branch items (nl T) over instances, ninst + 1
    int64_t *bus_items = nullptr;  // prefix of bus items (nb T)
    int64_t *gen_items = nullptr;  // prefix of generator items (ng T)
    // scratch
    ArcScratch *arcs = nullptr;    // total arc slots (sum over instances of 2 nl T)
    double *obj_part = nullptr;    // per-CTA partial objective sums
    unsigned int *ticket = nullptr;
};

// Host copy of one instance's structure, kept to answer opf_sparsity and
// opf_bounds without storing the (possibly very large) patterns.
struct HostInst {
    int32_t nb = 0, nl = 0, ng = 0, T = 1, ref = 0;
    bool ramp = false;
    double ramp_ratio = 0.0;
    std::vector<int32_t> f, t;
    std::vector<int32_t> arc_ptr;   // nb + 1
    std::vector<int32_t> slot_arc;  // arc id of each bus-sorted slot
    std::vector<int32_t> slot_nbr;  // far bus of each slot
    std::vector<int32_t> gen_ptr;   // nb + 1
    std::vector<int32_t> gen_list;  // ascending per bus
    std::vector<double> vmin, vmax, rate, angmin, angmax, pmin, pmax, qmin, qmax;
    // storage units
    int32_t ns = 0;
    std::vector<int32_t> st_bus, st_ptr, st_list;  // st_ptr: nb + 1, st_list ascending per bus
    std::vector<double> st_E, st_Pc, st_Pd, st_S, st_qmin, st_qmax, st_einit, st_ploss;
};

struct Model {
    int32_t ninst = 0;
    bool on_device = false;  // false: structure only (no device arrays)
    bool rect = false;       // rectangular voltages (vr, vi) instead of polar (va, vm)
    bool storage = false;    // some instance has storage units
    bool st_compl = false;   // storage complementarity rows
    bool link = false;
    double link_ratio = 0.0;
    std::vector<double> link_ratios;   // per instance (entry 0 unused)
    bool reserve = false;
    double reserve_frac = 0.0;
    std::vector<double> res_cap;       // per reserve row: sum pmax - reserve * total Pd
    int64_t nres = 0;                  // reserve rows (one per instance and period)
    int64_t n = 0, m = 0, nnzj = 0, nnzh = 0;
    int64_t link_c0 = 0, link_j0 = 0;  // first linking row / its first Jacobian value
    int64_t res_c0 = 0, res_j0 = 0;    // first reserve row / its first Jacobian value
    int64_t nbr_items = 0, nbus_items = 0, ngen_items = 0, narc_slots = 0;
    int64_t nst_items = 0;        // storage items (units x periods, all instances)
    int64_t nlight_items = 0, nheavy_items = 0;  // split bus phase items
    bool split_ok = false;        // the split bus phase applies (no storage)
    int64_t npack_items = 0;      // fused evaluation: packed warps x periods, all instances
    bool fuse_ok = false;         // the fused evaluation applies (no storage, <= 32 slots per bus)
    int64_t nload_total = 0;      // sum over instances of nload * nperiod
    int32_t max_part = 0;         // capacity of obj_part
    int device = 0, num_sms = 148;
    opf_launch launch{};
    std::vector<InstDev> inst;
    std::vector<HostInst> host;
    DevArrays d;
    std::vector<void *> allocations;
    // staging buffers of opf_eval_all_host (allocated on first use)
    double *stage = nullptr;
    size_t stage_bytes = 0;
    // pipelined host-buffer evaluation (opf_eval_all_host_async): two staging
    // slots, copy-in / compute / copy-out streams and their events
    double *astage[2] = {nullptr, nullptr};
    cudaStream_t s_in = nullptr, s_cmp = nullptr, s_out = nullptr;
    cudaEvent_t ev_entry = nullptr, ev_in[2] = {nullptr, nullptr}, ev_cmp[2] = {nullptr, nullptr},
                ev_out[2] = {nullptr, nullptr};
    int aslot = 0;
};

struct EvalArgs {
    const double *x;
    const double *lam;
    double sigma;
    double *obj, *grad, *c, *jac, *hess;
};

// kernels.cu
int launch_eval(Model &M, const EvalArgs &a, unsigned what, cudaStream_t s, int phases = 3);
int launch_flat_start(Model &M, double *x, cudaStream_t s);
int launch_sincos(Model &M, const double *d, int64_t n, double *sn, double *cs, cudaStream_t s);
int launch_jtprod(Model &M, const double *x, const double *v, double *out, cudaStream_t s);
// J^T mu of the augmented Lagrangian, mu from the rows c, lambda and the row
// bounds where it is read; advances the step state bp (4 doubles) if not null
int launch_jtprod_al(Model &M, const double *x, const double *c, const double *lam, const double *gl,
                     const double *gu, double rho, double *out, double *bp, cudaStream_t s);
// the augmented Lagrangian's gradient grad f + J^T mu in one kernel (fused
// layout, polar, no linking or reserve rows: al_grad_fused_ok)
bool al_grad_fused_ok(const Model &M);
int launch_al_grad(Model &M, const double *x, const double *lam, const double *gl, const double *gu, double rho,
                   double *out, double *bp, cudaStream_t s);
int launch_flows(Model &M, double *x, cudaStream_t s);
// single instance: p, q := flows at x's voltages (written into x), then the
// objective, gradient and constraints at that point (flow rows zero)
int launch_cons_setflows(Model &M, double *x, double *obj, double *grad, double *c, cudaStream_t s);
int launch_set_loads(Model &M, const double *pd, const double *qd, cudaStream_t s);

// abi.cu
void set_error(const char *fmt, ...);

}  // namespace opf

// the opaque handle of the C ABI
struct opf_model {
    opf::Model *M;
};

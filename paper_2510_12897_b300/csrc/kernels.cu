// Evaluation kernels of libopf (sm_103a, FP64). The kernels themselves are
// in the k_*.cuh files this translation unit includes (common helpers, branch
// phase, bus phase and fused evaluation, J^T v, auxiliary kernels); this file
// holds the launch code.
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
#include <cuda/atomic>

#include "model.h"

namespace opf {

namespace {

#include "k_common.cuh"
#include "k_branch.cuh"
#include "k_bus.cuh"
#include "k_jt.cuh"
#include "k_aux.cuh"

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
    // bus_order 3: the fused evaluation where it applies (no storage,
    // at most 32 arc slots per bus), one kernel per evaluation (launched
    // with the bus phase; the branch phase alone launches nothing)
    const bool fused = L.bus_order == 3 && M.fuse_ok;
    // fused, branch_occupancy 2: two roles (a rows warp and a Hessian warp
    // per packed warp) where there is both a Hessian and rows or Jacobian to
    // write; for the Jacobian and Hessian alone only while the packed warps
    // fit one per SM sub-partition (beyond that the operands both warps form
    // cost more FP64 issue than the shorter chains save)
    const bool fill = M.npack_items <= 4 * (int64_t)M.num_sms;
    const bool roles = fused && L.branch_occupancy == 2 && H && (C || (J && fill));
    int bu = L.bus_block > kBusBlockMax ? kBusBlockMax : L.bus_block;
    // the other calls of a two-role shape with arc work (rows, Jacobian or
    // Hessian) run one warp per packed warp in blocks of half the size: as
    // many packed warps per block (the objective and gradient alone keep
    // the block: its packed warps only write gradient zeros)
    if (fused && L.branch_occupancy == 2 && !roles && (C || J || H) && bu >= 64)
        bu /= 2;
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
    int gu_all = gu;
    if (fused) {
        const int tb = grid_for(gpad, bu, L.bus_ctas_per_sm, M.num_sms, cap);
        P.split_tblocks = tb;
        P.npack_items = M.npack_items;
        P.fuse_roles = roles ? 1 : 0;
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

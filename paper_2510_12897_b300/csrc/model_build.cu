// Host side of libopf: validation of the networks, the branch admittances of
// the pi-model, the layout of x / g / Jacobian / Hessian (Listing 3 order,
// 2-D index rule of Listing 10), the per-bus tables the bus kernel walks, and
// the patterns and bounds generated on demand from that layout.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "model.h"

namespace opf {

namespace {

bool finite_all(const double *p, int64_t n)
{
    for (int64_t i = 0; i < n; i++)
        if (!std::isfinite(p[i]))
            return false;
    return true;
}

int validate(const opf_network &n, int s)
{
    if (n.nbus < 1 || n.nbranch < 0 || n.ngen < 0 || n.nload < 0 || n.nperiod < 1) {
        set_error("instance %d: bad sizes (nbus %d, nbranch %d, ngen %d, nload %d, nperiod %d)", s,
                  n.nbus, n.nbranch, n.ngen, n.nload, n.nperiod);
        return OPF_EINVAL;
    }
    if (n.ref_bus < 0 || n.ref_bus >= n.nbus) {
        set_error("instance %d: ref_bus %d out of range", s, n.ref_bus);
        return OPF_EINVAL;
    }
    if (!n.bus_vmin || !n.bus_vmax || (n.nbranch && (!n.br_f || !n.br_t || !n.br_r || !n.br_x ||
        !n.br_b || !n.br_rate_a || !n.br_angmin || !n.br_angmax)) ||
        (n.ngen && (!n.gen_bus || !n.gen_pmin || !n.gen_pmax || !n.gen_qmin || !n.gen_qmax ||
        !n.gen_c2 || !n.gen_c1)) || (n.nload && (!n.load_bus || !n.load_pd || !n.load_qd))) {
        set_error("instance %d: a required array is NULL", s);
        return OPF_EINVAL;
    }
    int64_t nb = n.nbus, nl = n.nbranch, ng = n.ngen;
    // every in-instance offset (variables, rows, Jacobian and Hessian values,
    // scratch slots) must fit in 32 bits; the Jacobian is the largest (the
    // rectangular form's bound covers both forms)
    if ((int64_t)n.nperiod * (1 + 36 * nl + 6 * nb + 4 * ng) > INT32_MAX / 2 ||
        (int64_t)n.nperiod * (2 * nb + 2 * ng + 4 * nl + 10 * nl + 2 * nb) > INT32_MAX / 2) {
        set_error("instance %d: too large for 32-bit in-instance offsets", s);
        return OPF_EINVAL;
    }
    for (int k = 0; k < n.nbranch; k++) {
        if (n.br_f[k] < 0 || n.br_f[k] >= n.nbus || n.br_t[k] < 0 || n.br_t[k] >= n.nbus) {
            set_error("instance %d: branch %d endpoint out of range", s, k);
            return OPF_EINVAL;
        }
        if (n.br_f[k] == n.br_t[k]) {
            set_error("instance %d: branch %d is a self-loop", s, k);
            return OPF_EINVAL;
        }
        if (n.br_r[k] == 0.0 && n.br_x[k] == 0.0) {
            set_error("instance %d: branch %d has r = x = 0", s, k);
            return OPF_EINVAL;
        }
        if (n.br_tap && n.br_tap[k] < 0.0) {
            set_error("instance %d: branch %d has a negative tap", s, k);
            return OPF_EINVAL;
        }
    }
    for (int g = 0; g < n.ngen; g++)
        if (n.gen_bus[g] < 0 || n.gen_bus[g] >= n.nbus) {
            set_error("instance %d: generator %d bus out of range", s, g);
            return OPF_EINVAL;
        }
    for (int l = 0; l < n.nload; l++)
        if (n.load_bus[l] < 0 || n.load_bus[l] >= n.nbus) {
            set_error("instance %d: load %d bus out of range", s, l);
            return OPF_EINVAL;
        }
    bool ok = finite_all(n.bus_vmin, nb) && finite_all(n.bus_vmax, nb) &&
              (!n.bus_gs || finite_all(n.bus_gs, nb)) && (!n.bus_bs || finite_all(n.bus_bs, nb));
    if (nl)
        ok = ok && finite_all(n.br_r, nl) && finite_all(n.br_x, nl) && finite_all(n.br_b, nl) &&
             (!n.br_tap || finite_all(n.br_tap, nl)) && (!n.br_shift || finite_all(n.br_shift, nl)) &&
             finite_all(n.br_rate_a, nl);
    if (ng)
        ok = ok && finite_all(n.gen_c2, ng) && finite_all(n.gen_c1, ng) &&
             (!n.gen_c0 || finite_all(n.gen_c0, ng));
    if (n.nload)
        ok = ok && finite_all(n.load_pd, (int64_t)n.nload * n.nperiod) &&
             finite_all(n.load_qd, (int64_t)n.nload * n.nperiod);
    if (!ok) {
        set_error("instance %d: a network parameter is not finite", s);
        return OPF_EINVAL;
    }
    return OPF_OK;
}

template <class T>
int upload(Model &M, T **dst, const std::vector<T> &src)
{
    size_t bytes = sizeof(T) * (src.empty() ? 1 : src.size());
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc of %zu bytes failed", bytes);
        return OPF_ENOMEM;
    }
    M.allocations.push_back(p);
    if (!src.empty() && cudaMemcpy(p, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice) !=
                            cudaSuccess) {
        set_error("cudaMemcpy failed: %s", cudaGetErrorString(cudaGetLastError()));
        return OPF_ECUDA;
    }
    *dst = static_cast<T *>(p);
    return OPF_OK;
}

template <class T>
int alloc(Model &M, T **dst, size_t count)
{
    size_t bytes = sizeof(T) * (count ? count : 1);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc of %zu bytes failed", bytes);
        return OPF_ENOMEM;
    }
    M.allocations.push_back(p);
    *dst = static_cast<T *>(p);
    return OPF_OK;
}

}  // namespace

void free_model(Model *M)
{
    if (!M)
        return;
    for (void *p : M->allocations)
        cudaFree(p);
    if (M->stage)
        cudaFree(M->stage);
    if (M->s_cmp) {  // the pipelined host-buffer path was used
        cudaStreamSynchronize(M->s_in);
        cudaStreamSynchronize(M->s_cmp);
        cudaStreamSynchronize(M->s_out);
        for (int k = 0; k < 2; k++) {
            cudaFree(M->astage[k]);
            cudaEventDestroy(M->ev_in[k]);
            cudaEventDestroy(M->ev_cmp[k]);
            cudaEventDestroy(M->ev_out[k]);
        }
        cudaEventDestroy(M->ev_entry);
        cudaStreamDestroy(M->s_in);
        cudaStreamDestroy(M->s_cmp);
        cudaStreamDestroy(M->s_out);
    }
    delete M;
}

// Builds one model over `ninst` networks. On error returns a code and frees
// everything it allocated.
int build_model(const opf_network *nets, int32_t ninst, const opf_batch_opts *opts, bool device, Model **out)
{
    *out = nullptr;
    if (!nets || ninst < 1) {
        set_error("need at least one network");
        return OPF_EINVAL;
    }
    for (int s = 0; s < ninst; s++) {
        int rc = validate(nets[s], s);
        if (rc)
            return rc;
    }
    const double link_ratio = opts ? opts->link_ratio : 0.0;
    const double reserve = opts ? opts->reserve : 0.0;
    const int32_t form = opts ? opts->form : OPF_FORM_POLAR;
    if (form != OPF_FORM_POLAR && form != OPF_FORM_RECT) {
        set_error("form must be OPF_FORM_POLAR or OPF_FORM_RECT");
        return OPF_EINVAL;
    }
    const bool rect = form == OPF_FORM_RECT;
    if (rect)  // the tangent form of the angle rows needs limits inside (-pi/2, pi/2)
        for (int s = 0; s < ninst; s++)
            for (int k = 0; k < nets[s].nbranch; k++)
                if (!(std::fabs(nets[s].br_angmin[k]) < M_PI / 2) || !(std::fabs(nets[s].br_angmax[k]) < M_PI / 2)) {
                    set_error("instance %d: branch %d angle limits outside (-pi/2, pi/2) (rectangular form)", s, k);
                    return OPF_EINVAL;
                }
    if (!(link_ratio >= 0.0) || !std::isfinite(link_ratio) || !(reserve >= 0.0) || !std::isfinite(reserve)) {
        set_error("link_ratio and reserve must be finite and >= 0");
        return OPF_EINVAL;
    }
    if (opts && opts->link_ratios)
        for (int s = 1; s < ninst; s++)
            if (!(opts->link_ratios[s] >= 0.0) || !std::isfinite(opts->link_ratios[s])) {
                set_error("link_ratios[%d] must be finite and >= 0", s);
                return OPF_EINVAL;
            }
    const opf_storage *stor = opts ? opts->storage : nullptr;
    if (stor) {
        if (rect) {
            set_error("storage needs the polar form");
            return OPF_EINVAL;
        }
        for (int s = 0; s < ninst; s++) {
            const opf_storage &u = stor[s];
            if (u.nstor < 0 || (u.nstor > 0 && (!u.bus || !u.energy_rating || !u.charge_rating ||
                !u.discharge_rating || !u.thermal_rating || !u.eta_c || !u.eta_d || !u.r || !u.p_loss ||
                !u.qmin || !u.qmax || !u.e_init))) {
                set_error("instance %d: bad storage description (negative count or NULL array)", s);
                return OPF_EINVAL;
            }
            if (u.nstor > 0 && !(u.dt > 0.0 && std::isfinite(u.dt))) {
                set_error("instance %d: storage dt must be finite and > 0", s);
                return OPF_EINVAL;
            }
            for (int k = 0; k < u.nstor; k++) {
                if (u.bus[k] < 0 || u.bus[k] >= nets[s].nbus) {
                    set_error("instance %d: storage %d bus out of range", s, k);
                    return OPF_EINVAL;
                }
                const double v[] = {u.energy_rating[k], u.charge_rating[k], u.discharge_rating[k],
                                    u.thermal_rating[k], u.r[k]};
                bool ok = u.eta_c[k] > 0.0 && u.eta_d[k] > 0.0 && std::isfinite(u.eta_c[k]) &&
                          std::isfinite(u.eta_d[k]) && std::isfinite(u.p_loss[k]) && std::isfinite(u.qmin[k]) &&
                          std::isfinite(u.qmax[k]) && std::isfinite(u.e_init[k]);
                for (double w : v)
                    ok = ok && w >= 0.0 && std::isfinite(w);
                if (!ok) {
                    set_error("instance %d: storage %d: efficiencies must be > 0, ratings and r >= 0, "
                              "all finite", s, k);
                    return OPF_EINVAL;
                }
            }
            if ((int64_t)nets[s].nperiod * u.nstor * 22 > INT32_MAX / 2) {
                set_error("instance %d: storage too large for 32-bit in-instance offsets", s);
                return OPF_EINVAL;
            }
        }
    }
    bool link = (link_ratio > 0.0 || (opts && opts->link_ratios)) && ninst > 1;
    if (link)
        for (int s = 0; s < ninst; s++)
            if (nets[s].ngen != nets[0].ngen || nets[s].nperiod != 1) {
                set_error("linking rows need equal ngen and nperiod 1 in every instance");
                return OPF_ESTATE;
            }

    Model *M = new Model();
    M->ninst = ninst;
    M->rect = rect;
    for (int s = 0; stor && s < ninst; s++)
        M->storage = M->storage || stor[s].nstor > 0;
    M->st_compl = M->storage && opts->storage_complementarity != 0;
    M->link = link;
    M->link_ratio = link_ratio;
    M->link_ratios.assign(ninst, link_ratio);
    if (opts && opts->link_ratios)
        for (int s = 1; s < ninst; s++)
            M->link_ratios[s] = opts->link_ratios[s];
    M->reserve = reserve > 0.0;
    M->reserve_frac = reserve;
    M->on_device = device;
    if (device) {
        if (cudaGetDevice(&M->device) != cudaSuccess ||
            cudaDeviceGetAttribute(&M->num_sms, cudaDevAttrMultiProcessorCount, M->device) !=
                cudaSuccess) {
            cudaGetLastError();
            set_error("no usable CUDA device");
            delete M;
            return OPF_ECUDA;
        }
        if (M->num_sms <= 0)
            M->num_sms = 148;
    }

    // concatenated host arrays
    std::vector<int4> br, bus_a, bus_b;
    std::vector<int2> bus_c, br_jb;
    std::vector<int32_t> bus_order, light_list, heavy_list;
    std::vector<int64_t> light_items(1, 0), heavy_items(1, 0), pack_items(1, 0);
    std::vector<int4> pack;
    bool fits32 = true;  // every bus has at most 32 arc slots
    std::vector<double2> y_ff, y_ft, y_tf, y_tt, gsbs, pbnd, qbnd, vbnd;
    std::vector<double> rate2, Pd, Qd, c2, c1, c0;
    std::vector<double2> tanb;
    std::vector<int2> bus_st;
    std::vector<int32_t> st_list;
    std::vector<double4_16a> st_par;
    std::vector<int32_t> gen_list, load_ptr, load_list, gen_busid;
    std::vector<uint8_t> slot_code;
    std::vector<int64_t> br_items(1, 0), bus_items(1, 0), gen_items(1, 0), st_items(1, 0);
    std::vector<int32_t> st_busid;

    int64_t xo = 0, co = 0, jo = 0, ho = 0, so = 0, po = 0;
    M->inst.resize(ninst);
    M->host.resize(ninst);
    for (int s = 0; s < ninst; s++) {
        const opf_network &n = nets[s];
        HostInst &H = M->host[s];
        InstDev &I = M->inst[s];
        const int nb = n.nbus, nl = n.nbranch, ng = n.ngen, T = n.nperiod, na = 2 * nl;
        H.nb = nb; H.nl = nl; H.ng = ng; H.T = T; H.ref = n.ref_bus;
        H.ramp = T > 1 && n.ramp_ratio > 0.0;
        H.ramp_ratio = n.ramp_ratio;
        H.f.assign(n.br_f, n.br_f + nl);
        H.t.assign(n.br_t, n.br_t + nl);
        H.vmin.assign(n.bus_vmin, n.bus_vmin + nb);
        H.vmax.assign(n.bus_vmax, n.bus_vmax + nb);
        H.rate.assign(n.br_rate_a, n.br_rate_a + nl);
        H.angmin.assign(n.br_angmin, n.br_angmin + nl);
        H.angmax.assign(n.br_angmax, n.br_angmax + nl);
        H.pmin.assign(n.gen_pmin, n.gen_pmin + ng);
        H.pmax.assign(n.gen_pmax, n.gen_pmax + ng);
        H.qmin.assign(n.gen_qmin, n.gen_qmin + ng);
        H.qmax.assign(n.gen_qmax, n.gen_qmax + ng);

        I.nb = nb; I.nl = nl; I.ng = ng; I.T = T; I.ref = n.ref_bus; I.ramp = H.ramp;
        I.br0 = (int32_t)y_ff.size();
        I.bus0 = (int32_t)gsbs.size();
        I.gen0 = (int32_t)c2.size();
        I.gl0 = (int32_t)gen_list.size();
        I.slot0 = (int32_t)slot_code.size();
        I.nload = n.nload;
        I.lp0 = (int32_t)load_ptr.size();
        I.ll0 = (int32_t)load_list.size();
        I.ld0 = M->nload_total;
        M->nload_total += (int64_t)n.nload * T;

        // ---- branches: pi-model admittances (G, B) of Yff, Yft, Ytf, Ytt
        for (int k = 0; k < nl; k++) {
            double r = n.br_r[k], x = n.br_x[k], b = n.br_b[k];
            double tau = (n.br_tap && n.br_tap[k] != 0.0) ? n.br_tap[k] : 1.0;
            double th = n.br_shift ? n.br_shift[k] : 0.0;
            double den = r * r + x * x;
            double gs_ = r / den, bs_ = -x / den;  // ys = 1 / (r + j x)
            double ct = std::cos(th), st = std::sin(th);
            double2 tt = make_double2(gs_, bs_ + 0.5 * b);
            double2 ff = make_double2(tt.x / (tau * tau), tt.y / (tau * tau));
            // Yft = -ys e^{j th} / tau,  Ytf = -ys e^{-j th} / tau
            double2 ft = make_double2(-(gs_ * ct - bs_ * st) / tau, -(gs_ * st + bs_ * ct) / tau);
            double2 tf = make_double2(-(gs_ * ct + bs_ * st) / tau, (gs_ * st - bs_ * ct) / tau);
            y_ff.push_back(ff);
            y_ft.push_back(ft);
            y_tf.push_back(tf);
            y_tt.push_back(tt);
            rate2.push_back(n.br_rate_a[k] * n.br_rate_a[k]);
            if (rect)
                tanb.push_back(make_double2(std::tan(n.br_angmax[k]), std::tan(n.br_angmin[k])));
        }

        // ---- arcs sorted per bus by (far bus, arc id)
        std::vector<int32_t> deg(nb + 1, 0);
        for (int a = 0; a < na; a++)
            deg[a < nl ? n.br_f[a] : n.br_t[a - nl]]++;
        H.arc_ptr.assign(nb + 1, 0);
        for (int i = 0; i < nb; i++)
            H.arc_ptr[i + 1] = H.arc_ptr[i] + deg[i];
        std::vector<std::pair<int64_t, int32_t>> keyed(na);
        for (int a = 0; a < na; a++) {
            int bus = a < nl ? n.br_f[a] : n.br_t[a - nl];
            int far = a < nl ? n.br_t[a] : n.br_f[a - nl];
            keyed[a] = {((int64_t)bus * nb + far) * na + a, a};
        }
        std::sort(keyed.begin(), keyed.end());
        H.slot_arc.resize(na);
        H.slot_nbr.resize(na);
        std::vector<int32_t> pos_of(na);
        for (int p = 0; p < na; p++) {
            int a = keyed[p].second;
            H.slot_arc[p] = a;
            H.slot_nbr[p] = a < nl ? n.br_t[a] : n.br_f[a - nl];
            pos_of[a] = p;
        }
        for (int k = 0; k < nl; k++)
            br.push_back(make_int4(n.br_f[k], n.br_t[k], pos_of[k], pos_of[nl + k]));

        // ---- generators per bus (ascending id)
        std::vector<int32_t> gcnt(nb + 1, 0);
        for (int g = 0; g < ng; g++)
            gcnt[n.gen_bus[g]]++;
        H.gen_ptr.assign(nb + 1, 0);
        for (int i = 0; i < nb; i++)
            H.gen_ptr[i + 1] = H.gen_ptr[i] + gcnt[i];
        H.gen_list.assign(ng, 0);
        {
            std::vector<int32_t> fill(H.gen_ptr.begin(), H.gen_ptr.end() - 1);
            for (int g = 0; g < ng; g++)
                H.gen_list[fill[n.gen_bus[g]]++] = g;
        }
        for (int g = 0; g < ng; g++)
            gen_list.push_back(H.gen_list[g]);

        // ---- storage units per bus (ascending id)
        const int ns = stor ? stor[s].nstor : 0;
        H.ns = ns;
        H.st_ptr.assign(nb + 1, 0);
        H.st_list.assign(ns, 0);
        if (ns) {
            const opf_storage &u = stor[s];
            H.st_bus.assign(u.bus, u.bus + ns);
            H.st_E.assign(u.energy_rating, u.energy_rating + ns);
            H.st_Pc.assign(u.charge_rating, u.charge_rating + ns);
            H.st_Pd.assign(u.discharge_rating, u.discharge_rating + ns);
            H.st_S.assign(u.thermal_rating, u.thermal_rating + ns);
            H.st_qmin.assign(u.qmin, u.qmin + ns);
            H.st_qmax.assign(u.qmax, u.qmax + ns);
            H.st_einit.assign(u.e_init, u.e_init + ns);
            H.st_ploss.assign(u.p_loss, u.p_loss + ns);
            for (int k = 0; k < ns; k++)
                H.st_ptr[u.bus[k] + 1]++;
            for (int i = 0; i < nb; i++)
                H.st_ptr[i + 1] += H.st_ptr[i];
            std::vector<int32_t> fill(H.st_ptr.begin(), H.st_ptr.end() - 1);
            for (int k = 0; k < ns; k++)
                H.st_list[fill[u.bus[k]]++] = k;
        }
        I.ns = ns;
        I.st0 = (int32_t)st_par.size();
        I.st_compl = M->st_compl && ns > 0;
        for (int k = 0; k < ns; k++) {
            const opf_storage &u = stor[s];
            st_par.push_back(make_double4_16a(u.dt * u.eta_c[k], u.dt / u.eta_d[k], u.r[k], u.e_init[k]));
        }

        // ---- per-bus row offsets inside one period, slot codes
        int64_t jsum = 0, hva = 0, hvm = 0;
        std::vector<int32_t> jp_local(nb);
        for (int i = 0; i < nb; i++) {
            jp_local[i] = (int32_t)jsum;
            int p0 = H.arc_ptr[i], p1 = H.arc_ptr[i + 1];
            int nd = 0, nlt = 0, nlow = 0;
            uint32_t lastmask = 0;
            for (int p = p0; p < p1; p++) {
                bool first = p == p0 || H.slot_nbr[p] != H.slot_nbr[p - 1];
                bool last = p + 1 == p1 || H.slot_nbr[p + 1] != H.slot_nbr[p];
                if (first) {
                    nd++;
                    if (H.slot_nbr[p] < i)
                        nlt++;
                }
                slot_code.push_back((uint8_t)((last ? SLOT_LAST : 0) | (H.slot_nbr[p] < i ? SLOT_LOWER : 0)));
                if (last && p - p0 < 32)
                    lastmask |= 1u << (p - p0);
                if (H.slot_nbr[p] < i)
                    nlow++;
            }
            if (nd > 0x7fff) {
                set_error("instance %d: bus %d has more than 32767 distinct neighbours", s, i);
                delete M;
                return OPF_EINVAL;
            }
            bus_a.push_back(make_int4(p0, p1, H.gen_ptr[i], H.gen_ptr[i + 1]));
            bus_b.push_back(make_int4((int32_t)jsum, (int32_t)hva, (int32_t)hvm, nd | (nlt << 16)));
            bus_c.push_back(make_int2((int32_t)lastmask, nlow));
            // balance rows: the voltage entries (vm; or vr, vi), generators, arcs
            jsum += (rect ? 2 : 1) + (H.gen_ptr[i + 1] - H.gen_ptr[i]) + (p1 - p0) +
                    (H.st_ptr[i + 1] - H.st_ptr[i]);  // storage units after the arcs
            if (rect) {  // rows vr_i: lower vr_j, diagonal; rows vi_i: every vr_j, lower vi_j, diagonal
                hva += nlt + 1;
                hvm += nd + nlt + 1;
            } else if (p1 > p0) {
                hva += nlt + 1;
                hvm += (nd + 1) + nlt + 1;
            } else {
                hvm += 1;
            }
            double gsv = n.bus_gs ? n.bus_gs[i] : 0.0, bsv = n.bus_bs ? n.bus_bs[i] : 0.0;
            gsbs.push_back(make_double2(gsv, bsv));
            vbnd.push_back(make_double2(n.bus_vmin[i], n.bus_vmax[i]));
            bus_st.push_back(make_int2((int32_t)st_list.size() + H.st_ptr[i], (int32_t)st_list.size() + H.st_ptr[i + 1]));
        }

        // ---- split bus phase lists: heavy buses (kLightSlots < slots <= 32)
        // get a warp each, the others a thread each; both in id order
        I.light0 = (int32_t)light_list.size();
        I.heavy0 = (int32_t)heavy_list.size();
        for (int i = 0; i < nb; i++) {
            const int ns_i = H.arc_ptr[i + 1] - H.arc_ptr[i];
            if (ns_i > kLightSlots && ns_i <= 32)
                heavy_list.push_back(i);
            else
                light_list.push_back(i);
        }
        I.nlight = (int32_t)light_list.size() - I.light0;
        I.nheavy = (int32_t)heavy_list.size() - I.heavy0;

        // ---- fused evaluation: buses packed whole into warps of 32 lanes,
        // one lane per arc slot (one for a bus without arcs), in order of
        // arc count (descending, then id): the buses of a warp have similar
        // slot counts, so most warps' segmented scans take fewer steps (a
        // warp scans as many steps as its largest bus needs); the rest of a
        // warp that cannot take the next bus is padding
        I.pack0 = (int32_t)(pack.size() / 32);
        {
            const size_t lo = (size_t)I.slot0;
            auto close_warp = [&]() {
                while (pack.size() % 32)
                    pack.push_back(make_int4(-1, -1, 0, 0));
            };
            std::vector<int32_t> by_deg(nb);
            std::iota(by_deg.begin(), by_deg.end(), 0);
            std::stable_sort(by_deg.begin(), by_deg.end(), [&](int x, int y) {
                return H.arc_ptr[x + 1] - H.arc_ptr[x] > H.arc_ptr[y + 1] - H.arc_ptr[y];
            });
            for (int i : by_deg) {
                const int p0 = H.arc_ptr[i], p1 = H.arc_ptr[i + 1];
                const int lanes = p1 > p0 ? p1 - p0 : 1;
                if (lanes > 32) {
                    fits32 = false;
                    continue;
                }
                if (pack.size() % 32 + lanes > 32)
                    close_warp();
                if (p1 == p0) {
                    pack.push_back(make_int4(-1, i, PK_VALID | PK_HEAD | PK_TAIL | PK_GTAIL, 0));
                    continue;
                }
                int grp = 0;
                for (int p = p0; p < p1; p++) {
                    const uint8_t code = slot_code[lo + p];
                    int fl = PK_VALID | (p == p0 ? PK_HEAD : 0) | (p + 1 == p1 ? PK_TAIL : 0) |
                             ((code & SLOT_LAST) ? PK_GTAIL : 0) | ((code & SLOT_LOWER) ? PK_LOWER : 0);
                    pack.push_back(make_int4(H.slot_arc[p], i, fl, grp));
                    if (code & SLOT_LAST)
                        grp++;
                }
            }
            close_warp();
        }
        I.npack = (int32_t)(pack.size() / 32) - I.pack0;

        // ---- each arc's +1 entry in its bus's balance row: after the voltage
        // entries and the bus's generators, arcs in ascending id
        {
            std::vector<int32_t> jb(na);
            std::vector<int32_t> ids;
            for (int i = 0; i < nb; i++) {
                ids.assign(H.slot_arc.begin() + H.arc_ptr[i], H.slot_arc.begin() + H.arc_ptr[i + 1]);
                std::sort(ids.begin(), ids.end());
                const int base = jp_local[i] + (rect ? 2 : 1) + (H.gen_ptr[i + 1] - H.gen_ptr[i]);
                for (size_t r = 0; r < ids.size(); r++)
                    jb[ids[r]] = base + (int32_t)r;
            }
            for (int k = 0; k < nl; k++)
                br_jb.push_back(make_int2(jb[k], jb[nl + k]));
        }
        // ---- alternative bus-phase order: buses sorted by arc count (stable),
        // cut into warps of 32, the warps dealt heaviest, lightest, next
        // heaviest, ... so that lanes of a warp walk similar slot counts and
        // the heavy warps spread over the grid
        {
            std::vector<int32_t> ord(nb);
            std::iota(ord.begin(), ord.end(), 0);
            std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
                return H.arc_ptr[a + 1] - H.arc_ptr[a] < H.arc_ptr[b + 1] - H.arc_ptr[b];
            });
            const int nw = (nb + 31) / 32;
            int lo = 0, hi = nw - 1;
            bool heavy = true;
            while (lo <= hi) {
                const int w = heavy ? hi-- : lo++;
                heavy = !heavy;
                for (int q = w * 32; q < std::min(nb, w * 32 + 32); q++)
                    bus_order.push_back(ord[q]);
            }
        }
        // ---- loads per bus (ascending id), the order the demand sums use
        {
            std::vector<int32_t> cnt(nb + 1, 0);
            for (int l = 0; l < n.nload; l++)
                cnt[n.load_bus[l] + 1]++;
            for (int i = 0; i < nb; i++)
                cnt[i + 1] += cnt[i];
            std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1), lst(n.nload);
            for (int l = 0; l < n.nload; l++)
                lst[fill[n.load_bus[l]]++] = l;
            load_ptr.insert(load_ptr.end(), cnt.begin(), cnt.end());
            load_list.insert(load_list.end(), lst.begin(), lst.end());
        }
        // ---- demand per bus and period
        size_t pd_base = Pd.size();
        Pd.resize(pd_base + (size_t)nb * T, 0.0);
        Qd.resize(pd_base + (size_t)nb * T, 0.0);
        for (int t = 0; t < T; t++)
            for (int l = 0; l < n.nload; l++) {
                Pd[pd_base + (size_t)t * nb + n.load_bus[l]] += n.load_pd[(size_t)t * n.nload + l];
                Qd[pd_base + (size_t)t * nb + n.load_bus[l]] += n.load_qd[(size_t)t * n.nload + l];
            }

        st_list.insert(st_list.end(), H.st_list.begin(), H.st_list.end());
        for (int g = 0; g < ng; g++) {
            gen_busid.push_back(n.gen_bus[g]);
            c2.push_back(n.gen_c2[g]);
            c1.push_back(n.gen_c1[g]);
            c0.push_back(n.gen_c0 ? n.gen_c0[g] : 0.0);
            pbnd.push_back(make_double2(n.gen_pmin[g], n.gen_pmax[g]));
            qbnd.push_back(make_double2(n.gen_qmin[g], n.gen_qmax[g]));
        }

        // ---- offsets
        I.jP = (int64_t)(rect ? 2 * nb : nb) + ng + na + ns;
        I.hva = hva;
        I.hvm = hvm;
        I.x0 = xo;
        I.c0 = co;
        I.j0 = jo;
        I.h0 = ho;
        I.scr0 = so;
        I.pd0 = po;
        I.link_c = I.link_j = -1;
        I.link_x0 = 0;
        I.res_c = I.res_j = -1;
        xo += (int64_t)T * (2 * nb + 2 * ng + 2 * na + 5 * (int64_t)ns);
        // rectangular: one more angle row per branch and a magnitude row per bus
        const int64_t rows0 = (int64_t)T * (1 + (rect ? 8 : 7) * (int64_t)nl + (rect ? 3 : 2) * nb) +
                              (H.ramp ? (int64_t)ng * (T - 1) : 0);
        const int64_t jac0 = (int64_t)T * (1 + (rect ? 36 : 30) * (int64_t)nl + (rect ? 6 : 2) * nb + 2 * ng) +
                             (H.ramp ? 2 * (int64_t)ng * (T - 1) : 0) + 2 * (int64_t)T * ns;  // + balance entries
        const int64_t hes0 = (int64_t)T * (hva + hvm + ng + 2 * (int64_t)na);
        // storage rows: state of charge (3 entries in the first period, 4
        // after), losses (5), thermal (2), complementarity (2); Hessian
        // (ps, vm), (ps, ps), (qs, vm), (qs, qs), complementarity (sd, sc)
        I.st_c = rows0;
        I.st_j = jac0;
        I.st_h = hes0;
        co += rows0 + (int64_t)(3 + I.st_compl) * ns * T;
        jo += jac0 + (int64_t)ns * (4 * T - 1) + 7 * (int64_t)ns * T + (I.st_compl ? 2 * (int64_t)ns * T : 0);
        ho += hes0 + (int64_t)(4 + I.st_compl) * ns * T;
        so += (int64_t)na * T;
        po += (int64_t)nb * T;
        br_items.push_back(br_items.back() + (int64_t)nl * T);
        bus_items.push_back(bus_items.back() + (int64_t)nb * T);
        gen_items.push_back(gen_items.back() + (int64_t)ng * T);
        st_items.push_back(st_items.back() + (int64_t)ns * T);
        light_items.push_back(light_items.back() + (int64_t)I.nlight * T);
        heavy_items.push_back(heavy_items.back() + (int64_t)I.nheavy * T);
        pack_items.push_back(pack_items.back() + (int64_t)I.npack * T);
        for (int k = 0; k < ns; k++)
            st_busid.push_back(stor[s].bus[k]);
    }
    M->link_c0 = co;
    M->link_j0 = jo;
    if (link) {
        int64_t ng = nets[0].ngen;
        for (int s = 1; s < ninst; s++) {
            M->inst[s].link_c = co + ng * (s - 1);
            M->inst[s].link_j = jo + 2 * ng * (s - 1);
            M->inst[s].link_x0 = M->inst[0].x0 + 2 * (int64_t)nets[0].nbus;  // pg of instance 0
        }
        co += ng * (ninst - 1);
        jo += 2 * ng * (ninst - 1);
    }
    // reserve rows: per instance, one per period, after the linking rows
    M->res_c0 = co;
    M->res_j0 = jo;
    std::vector<int2> res_st;
    if (M->reserve) {
        for (int s = 0; s < ninst; s++) {
            const opf_network &n = nets[s];
            M->inst[s].res_c = co;
            M->inst[s].res_j = jo;
            double cap = 0.0;
            for (int g = 0; g < n.ngen; g++)
                cap += n.gen_pmax[g];
            for (int t = 0; t < n.nperiod; t++) {
                double pd = 0.0;
                for (int l = 0; l < n.nload; l++)
                    pd += n.load_pd[(int64_t)t * n.nload + l];
                M->res_cap.push_back(cap - reserve * pd);
                res_st.push_back(make_int2(s, t));
            }
            co += n.nperiod;
            jo += (int64_t)n.nperiod * n.ngen;
        }
        M->nres = (int64_t)res_st.size();
    }
    M->n = xo;
    M->m = co;
    M->nnzj = jo;
    M->nnzh = ho;
    M->nbr_items = br_items.back();
    M->nbus_items = bus_items.back();
    M->ngen_items = gen_items.back();
    M->nst_items = st_items.back();
    M->nlight_items = light_items.back();
    M->nheavy_items = heavy_items.back();
    M->split_ok = !stor;
    M->npack_items = pack_items.back();
    M->fuse_ok = !stor && fits32;
    M->narc_slots = so;
    M->max_part = 16 * M->num_sms;
    M->launch = opf_launch{128, 128, 0, 0, 0, 0};

    if (!device) {
        *out = M;
        return OPF_OK;
    }
    int rc = OPF_OK;
    DevArrays &d = M->d;
#define UP(field, vec)                           \
    if (!rc)                                     \
        rc = upload(*M, &d.field, vec);
    UP(br, br) UP(y_ff, y_ff) UP(y_ft, y_ft) UP(y_tf, y_tf) UP(y_tt, y_tt) UP(rate2, rate2) UP(tanb, tanb)
    std::vector<double2> trig;
    for (int k = -kTrigK; k <= kTrigK; k++)
        trig.push_back(make_double2(std::sin((double)k / kTrigScale), std::cos((double)k / kTrigScale)));
    UP(trig, trig)
    UP(br_jb, br_jb) UP(bus_order, bus_order) UP(res_st, res_st) UP(load_ptr, load_ptr) UP(load_list, load_list)
    UP(gen_busid, gen_busid)
    UP(bus_a, bus_a) UP(bus_b, bus_b) UP(bus_c, bus_c) UP(gsbs, gsbs) UP(slot_code, slot_code) UP(gen_list, gen_list)
    UP(Pd, Pd) UP(Qd, Qd) UP(c2, c2) UP(c1, c1) UP(c0, c0) UP(pbnd, pbnd) UP(qbnd, qbnd)
    if (M->split_ok) {
        UP(light_list, light_list) UP(heavy_list, heavy_list) UP(light_items, light_items)
        UP(heavy_items, heavy_items)
    }
    if (M->fuse_ok) {
        UP(pack, pack) UP(pack_items, pack_items)
    }
    if (M->storage) {
        UP(bus_st, bus_st) UP(st_list, st_list) UP(st_par, st_par) UP(st_busid, st_busid) UP(st_items, st_items)
    }
    UP(vbnd, vbnd) UP(inst, M->inst) UP(br_items, br_items) UP(bus_items, bus_items)
    UP(gen_items, gen_items)
#undef UP
    if (!rc)
        rc = alloc(*M, &d.arcs, (size_t)M->narc_slots);
    if (!rc)
        rc = alloc(*M, &d.obj_part, (size_t)M->max_part);
    if (!rc)
        rc = alloc(*M, &d.ticket, 1);
    if (!rc && cudaMemset(d.ticket, 0, sizeof(unsigned int)) != cudaSuccess) {
        set_error("cudaMemset failed");
        rc = OPF_ECUDA;
    }
    if (rc) {
        free_model(M);
        return rc;
    }
    *out = M;
    return OPF_OK;
}

// ------------------------------------------------------------ patterns --

namespace {

struct Offs {  // group bases of one instance
    int64_t va, vm, pg, qg, p, q;
};

Offs xoffs(const HostInst &H, const InstDev &I)
{
    int64_t T = H.T, nbT = (int64_t)H.nb * T, ngT = (int64_t)H.ng * T, naT = 2 * (int64_t)H.nl * T;
    return Offs{I.x0, I.x0 + nbT, I.x0 + 2 * nbT, I.x0 + 2 * nbT + ngT, I.x0 + 2 * nbT + 2 * ngT,
                I.x0 + 2 * nbT + 2 * ngT + naT};
}

// distinct far buses of bus i, ascending
void neighbours(const HostInst &H, int i, std::vector<int32_t> &out)
{
    out.clear();
    for (int p = H.arc_ptr[i]; p < H.arc_ptr[i + 1]; p++)
        if (out.empty() || out.back() != H.slot_nbr[p])
            out.push_back(H.slot_nbr[p]);
}

}  // namespace

void jac_pattern(const Model &M, int64_t *rows, int64_t *cols)
{
    int64_t e = 0;
    auto put = [&](int64_t r, int64_t c) {
        rows[e] = r;
        cols[e] = c;
        e++;
    };
    std::vector<int32_t> arcs;
    for (int s = 0; s < M.ninst; s++) {
        const HostInst &H = M.host[s];
        const InstDev &I = M.inst[s];
        const Offs X = xoffs(H, I);
        const int64_t nb = H.nb, nl = H.nl, ng = H.ng, T = H.T, na = 2 * nl;
        int64_t r = I.c0;
        for (int64_t t = 0; t < T; t++)  // va_ref, or vi_ref (rectangular)
            put(r++, (M.rect ? X.vm : X.va) + H.ref + nb * t);
        for (int grp = 0; grp < 4; grp++)
            for (int64_t t = 0; t < T; t++)
                for (int64_t k = 0; k < nl; k++) {
                    int64_t f = H.f[k], b = H.t[k], lo = std::min(f, b), hi = std::max(f, b);
                    int64_t own = (grp == 0 ? X.p + k : grp == 1 ? X.q + k : grp == 2 ? X.p + nl + k
                                                                                     : X.q + nl + k) + na * t;
                    put(r, X.va + lo + nb * t);
                    put(r, X.va + hi + nb * t);
                    put(r, X.vm + lo + nb * t);
                    put(r, X.vm + hi + nb * t);
                    put(r, own);
                    r++;
                }
        // angle rows: (va_lo, va_hi); rectangular: (vr_lo, vr_hi, vi_lo, vi_hi)
        auto angle_rows = [&]() {
            for (int64_t t = 0; t < T; t++)
                for (int64_t k = 0; k < nl; k++) {
                    int64_t f = H.f[k], b = H.t[k];
                    put(r, X.va + std::min(f, b) + nb * t);
                    put(r, X.va + std::max(f, b) + nb * t);
                    if (M.rect) {
                        put(r, X.vm + std::min(f, b) + nb * t);
                        put(r, X.vm + std::max(f, b) + nb * t);
                    }
                    r++;
                }
        };
        angle_rows();
        for (int pq = 0; pq < 2; pq++)
            for (int64_t t = 0; t < T; t++)
                for (int i = 0; i < H.nb; i++) {
                    if (M.rect)
                        put(r, X.va + i + nb * t);
                    put(r, X.vm + i + nb * t);
                    for (int p = H.gen_ptr[i]; p < H.gen_ptr[i + 1]; p++)
                        put(r, (pq ? X.qg : X.pg) + H.gen_list[p] + ng * t);
                    arcs.assign(H.slot_arc.begin() + H.arc_ptr[i], H.slot_arc.begin() + H.arc_ptr[i + 1]);
                    std::sort(arcs.begin(), arcs.end());
                    for (int a : arcs)
                        put(r, (pq ? X.q : X.p) + a + na * t);
                    for (int u = H.st_ptr[i]; u < H.st_ptr[i + 1]; u++)  // storage: ps or qs
                        put(r, X.q + na * T + (pq ? (int64_t)H.ns * T : 0) + H.st_list[u] + (int64_t)H.ns * t);
                    r++;
                }
        for (int side = 0; side < 2; side++)
            for (int64_t t = 0; t < T; t++)
                for (int64_t k = 0; k < nl; k++) {
                    int64_t a = side ? nl + k : k;
                    put(r, X.p + a + na * t);
                    put(r, X.q + a + na * t);
                    r++;
                }
        if (M.rect) {  // lower angle rows, then the magnitude rows (vr_i, vi_i)
            angle_rows();
            for (int64_t t = 0; t < T; t++)
                for (int64_t i = 0; i < nb; i++) {
                    put(r, X.va + i + nb * t);
                    put(r, X.vm + i + nb * t);
                    r++;
                }
        }
        if (H.ramp)
            for (int64_t t = 1; t < T; t++)
                for (int64_t g = 0; g < ng; g++) {
                    put(r, X.pg + g + ng * (t - 1));
                    put(r, X.pg + g + ng * t);
                    r++;
                }
        if (H.ns) {  // storage rows: state of charge, losses, thermal, complementarity
            const int64_t ns = H.ns, st = X.q + na * T;
            auto v = [&](int w, int64_t k, int64_t t) { return st + w * ns * T + k + ns * t; };
            for (int64_t t = 0; t < T; t++)
                for (int64_t k = 0; k < ns; k++, r++) {
                    put(r, v(2, k, t));
                    put(r, v(3, k, t));
                    if (t >= 1)
                        put(r, v(4, k, t - 1));
                    put(r, v(4, k, t));
                }
            for (int64_t t = 0; t < T; t++)
                for (int64_t k = 0; k < ns; k++, r++) {
                    put(r, X.vm + H.st_bus[k] + nb * t);
                    for (int w = 0; w < 4; w++)
                        put(r, v(w, k, t));
                }
            for (int64_t t = 0; t < T; t++)
                for (int64_t k = 0; k < ns; k++, r++) {
                    put(r, v(0, k, t));
                    put(r, v(1, k, t));
                }
            for (int64_t t = 0; t < T && I.st_compl; t++)
                for (int64_t k = 0; k < ns; k++, r++) {
                    put(r, v(2, k, t));
                    put(r, v(3, k, t));
                }
        }
    }
    if (M.link) {
        int64_t r = M.link_c0, ng = M.host[0].ng;
        Offs X0 = xoffs(M.host[0], M.inst[0]);
        for (int s = 1; s < M.ninst; s++) {
            Offs Xs = xoffs(M.host[s], M.inst[s]);
            for (int64_t g = 0; g < ng; g++) {
                put(r, X0.pg + g);
                put(r, Xs.pg + g);
                r++;
            }
        }
    }
    if (M.reserve) {
        int64_t r = M.res_c0;
        for (int s = 0; s < M.ninst; s++) {
            Offs Xs = xoffs(M.host[s], M.inst[s]);
            const int64_t ng = M.host[s].ng, T = M.host[s].T;
            for (int64_t t = 0; t < T; t++, r++)
                for (int64_t g = 0; g < ng; g++)
                    put(r, Xs.pg + g + ng * t);
        }
    }
}

void hess_pattern(const Model &M, int64_t *rows, int64_t *cols)
{
    int64_t e = 0;
    auto put = [&](int64_t r, int64_t c) {
        rows[e] = r;
        cols[e] = c;
        e++;
    };
    std::vector<int32_t> nbr;
    for (int s = 0; s < M.ninst; s++) {
        const HostInst &H = M.host[s];
        const InstDev &I = M.inst[s];
        const Offs X = xoffs(H, I);
        const int64_t nb = H.nb, ng = H.ng, T = H.T, na = 2 * (int64_t)H.nl;
        if (M.rect) {
            for (int64_t t = 0; t < T; t++)  // rows vr_i: lower vr_j, diagonal
                for (int i = 0; i < H.nb; i++) {
                    neighbours(H, i, nbr);
                    for (int j : nbr)
                        if (j < i)
                            put(X.va + i + nb * t, X.va + j + nb * t);
                    put(X.va + i + nb * t, X.va + i + nb * t);
                }
            for (int64_t t = 0; t < T; t++)  // rows vi_i: every vr_j, lower vi_j, diagonal
                for (int i = 0; i < H.nb; i++) {
                    neighbours(H, i, nbr);
                    const int64_t r = X.vm + i + nb * t;
                    for (int j : nbr)
                        put(r, X.va + j + nb * t);
                    for (int j : nbr)
                        if (j < i)
                            put(r, X.vm + j + nb * t);
                    put(r, r);
                }
        }
        for (int64_t t = 0; t < T && !M.rect; t++)  // rows va_i
            for (int i = 0; i < H.nb; i++) {
                neighbours(H, i, nbr);
                if (nbr.empty())
                    continue;
                for (int j : nbr)
                    if (j < i)
                        put(X.va + i + nb * t, X.va + j + nb * t);
                put(X.va + i + nb * t, X.va + i + nb * t);
            }
        for (int64_t t = 0; t < T && !M.rect; t++)  // rows vm_i
            for (int i = 0; i < H.nb; i++) {
                neighbours(H, i, nbr);
                int64_t r = X.vm + i + nb * t;
                if (!nbr.empty()) {
                    bool self = false;
                    for (int j : nbr) {
                        if (!self && j > i) {
                            put(r, X.va + i + nb * t);
                            self = true;
                        }
                        put(r, X.va + j + nb * t);
                    }
                    if (!self)
                        put(r, X.va + i + nb * t);
                    for (int j : nbr)
                        if (j < i)
                            put(r, X.vm + j + nb * t);
                }
                put(r, r);
            }
        for (int64_t t = 0; t < T; t++)
            for (int64_t g = 0; g < ng; g++)
                put(X.pg + g + ng * t, X.pg + g + ng * t);
        for (int64_t t = 0; t < T; t++)
            for (int64_t a = 0; a < na; a++)
                put(X.p + a + na * t, X.p + a + na * t);
        for (int64_t t = 0; t < T; t++)
            for (int64_t a = 0; a < na; a++)
                put(X.q + a + na * t, X.q + a + na * t);
        if (H.ns) {  // rows ps, qs: (vm of the unit's bus, own diagonal); rows sd: (sd, sc)
            const int64_t ns = H.ns, st = X.q + na * T;
            for (int w = 0; w < 2; w++)
                for (int64_t t = 0; t < T; t++)
                    for (int64_t k = 0; k < ns; k++) {
                        const int64_t r = st + w * ns * T + k + ns * t;
                        put(r, X.vm + H.st_bus[k] + nb * t);
                        put(r, r);
                    }
            for (int64_t t = 0; t < T && I.st_compl; t++)
                for (int64_t k = 0; k < ns; k++)
                    put(st + 3 * ns * T + k + ns * t, st + 2 * ns * T + k + ns * t);
        }
    }
}

void bounds(const Model &M, double *xl, double *xu, double *gl, double *gu)
{
    const double inf = INFINITY;
    for (int s = 0; s < M.ninst; s++) {
        const HostInst &H = M.host[s];
        const InstDev &I = M.inst[s];
        const Offs X = xoffs(H, I);
        const int64_t nb = H.nb, nl = H.nl, ng = H.ng, T = H.T, na = 2 * nl;
        for (int64_t t = 0; t < T; t++) {
            for (int64_t i = 0; i < nb; i++) {
                if (xl && M.rect) {  // -vmax <= vr, vi <= vmax
                    xl[X.va + i + nb * t] = xl[X.vm + i + nb * t] = -H.vmax[i];
                    xu[X.va + i + nb * t] = xu[X.vm + i + nb * t] = H.vmax[i];
                } else if (xl) {
                    xl[X.va + i + nb * t] = -inf;
                    xu[X.va + i + nb * t] = inf;
                    xl[X.vm + i + nb * t] = H.vmin[i];
                    xu[X.vm + i + nb * t] = H.vmax[i];
                }
            }
            for (int64_t g = 0; g < ng; g++)
                if (xl) {
                    xl[X.pg + g + ng * t] = H.pmin[g];
                    xu[X.pg + g + ng * t] = H.pmax[g];
                    xl[X.qg + g + ng * t] = H.qmin[g];
                    xu[X.qg + g + ng * t] = H.qmax[g];
                }
            for (int64_t a = 0; a < na; a++)
                if (xl) {
                    double rate = H.rate[a % nl];
                    xl[X.p + a + na * t] = -rate;
                    xu[X.p + a + na * t] = rate;
                    xl[X.q + a + na * t] = -rate;
                    xu[X.q + a + na * t] = rate;
                }
            for (int64_t k = 0; xl && k < H.ns; k++) {  // ps, qs, sc, sd, se
                const int64_t ns = H.ns, v = X.q + na * T + k + ns * t;
                xl[v] = -H.st_S[k];
                xu[v] = H.st_S[k];
                xl[v + ns * T] = H.st_qmin[k];
                xu[v + ns * T] = H.st_qmax[k];
                xl[v + 2 * ns * T] = 0.0;
                xu[v + 2 * ns * T] = H.st_Pc[k];
                xl[v + 3 * ns * T] = 0.0;
                xu[v + 3 * ns * T] = H.st_Pd[k];
                xl[v + 4 * ns * T] = 0.0;
                xu[v + 4 * ns * T] = H.st_E[k];
            }
        }
        if (!gl)
            continue;
        // groups: ref, 4 flows, angle, P, Q balance: all [0, 0] except angle
        int64_t c = I.c0;
        for (int64_t t = 0; t < T; t++, c++)
            gl[c] = gu[c] = 0.0;
        for (int64_t r = 0; r < 4 * nl * T; r++, c++)
            gl[c] = gu[c] = 0.0;
        for (int64_t t = 0; t < T; t++)
            for (int64_t k = 0; k < nl; k++, c++) {
                gl[c] = M.rect ? -inf : H.angmin[k];
                gu[c] = M.rect ? 0.0 : H.angmax[k];
            }
        for (int64_t r = 0; r < 2 * nb * T; r++, c++)
            gl[c] = gu[c] = 0.0;
        for (int64_t r = 0; r < 2 * nl * T; r++, c++) {
            gl[c] = -inf;
            gu[c] = 0.0;
        }
        if (M.rect) {  // lower angle rows [0, inf], magnitude rows [vmin^2, vmax^2]
            for (int64_t r = 0; r < nl * T; r++, c++) {
                gl[c] = 0.0;
                gu[c] = inf;
            }
            for (int64_t t = 0; t < T; t++)
                for (int64_t i = 0; i < nb; i++, c++) {
                    gl[c] = H.vmin[i] * H.vmin[i];
                    gu[c] = H.vmax[i] * H.vmax[i];
                }
        }
        if (H.ramp)
            for (int64_t t = 1; t < T; t++)
                for (int64_t g = 0; g < ng; g++, c++) {
                    gl[c] = -H.ramp_ratio * H.pmax[g];
                    gu[c] = H.ramp_ratio * H.pmax[g];
                }
        const int64_t ns = H.ns;
        for (int64_t t = 0; t < T; t++)  // state of charge
            for (int64_t k = 0; k < ns; k++, c++)
                gl[c] = gu[c] = t == 0 ? H.st_einit[k] : 0.0;
        for (int64_t t = 0; t < T; t++)  // losses
            for (int64_t k = 0; k < ns; k++, c++)
                gl[c] = gu[c] = H.st_ploss[k];
        for (int64_t t = 0; t < T; t++)  // thermal
            for (int64_t k = 0; k < ns; k++, c++) {
                gl[c] = -inf;
                gu[c] = H.st_S[k] * H.st_S[k];
            }
        for (int64_t t = 0; t < T && I.st_compl; t++)  // complementarity
            for (int64_t k = 0; k < ns; k++, c++) {
                gl[c] = -inf;
                gu[c] = 0.0;
            }
    }
    if (M.link && gl) {
        int64_t c = M.link_c0, ng = M.host[0].ng;
        for (int s = 1; s < M.ninst; s++)
            for (int64_t g = 0; g < ng; g++, c++) {
                gl[c] = -M.link_ratios[s] * M.host[0].pmax[g];
                gu[c] = M.link_ratios[s] * M.host[0].pmax[g];
            }
    }
    if (M.reserve && gl)
        for (int64_t r = 0; r < M.nres; r++) {
            gl[M.res_c0 + r] = -INFINITY;
            gu[M.res_c0 + r] = M.res_cap[r];
        }
}

}  // namespace opf

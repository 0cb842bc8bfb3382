// opf_eval_all_noalloc: the fused evaluation with its scratch in a static
// device array instead of memory allocated by the library.
//
// Who needs it: code that must not allocate device memory while it runs,
// for example a solver embedded in a process whose device memory is owned
// and partitioned by another runtime (a fixed arena handed out at start-up,
// a memory pool that may not grow), or a caller that has to keep
// cudaMalloc/cudaFree (which can synchronise the device) out of its
// iteration loop. The model itself is still created beforehand; this entry
// point then touches no allocator at all.
//
// The scratch is one file-scope __device__ array of OPF_NOALLOC_SCRATCH_BYTES
// bytes (8 MiB), present on every device that loads this library until the
// process exits. Host code cannot use the array's name as a device address:
// on the host that name is only a stand-in, so the device address is fetched
// once per device with cudaGetSymbolAddress, with that device current, on
// the first call made on that device, and cached.
#include <mutex>

#include "model.h"

namespace opf {
int launch_eval_scratch(Model &M, const EvalArgs &a, unsigned what, cudaStream_t s,
                        ArcScratch *arcs, double *obj_part, int max_part, unsigned int *ticket);
}

namespace {

constexpr size_t kScratchBytes = (size_t)8 << 20;  // OPF_NOALLOC_SCRATCH_BYTES
constexpr size_t kTicketBytes = 256;               // ticket word, padded to the alignment
constexpr int kMaxPart = 4096;                     // per-block objective partials
constexpr size_t kPartBytes = sizeof(double) * kMaxPart;
constexpr size_t kArcBytes = kScratchBytes - kTicketBytes - kPartBytes;
constexpr int64_t kMaxSlots = (int64_t)(kArcBytes / sizeof(opf::ArcScratch));

// layout: [ticket | objective partials | arc scratch]
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_addr[kMaxDevices] = {};

// device address of g_noalloc_scratch on the current device (set up once);
// the current device must be the model's (its arrays live there)
int scratch_address(int model_device, unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        opf::set_error("noalloc: cudaGetDevice failed: %s", cudaGetErrorString(e));
        return OPF_ECUDA;
    }
    if (dev != model_device) {
        opf::set_error("noalloc: the current device is %d but the model lives on device %d; "
                       "make the model's device current before the call", dev, model_device);
        return OPF_EINVAL;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        opf::set_error("noalloc: device %d beyond the %d supported", dev, kMaxDevices);
        return OPF_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            opf::set_error("noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return OPF_ECUDA;
        }
        g_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_addr[dev];
    return OPF_OK;
}

}  // namespace

extern "C" int opf_eval_all_noalloc(opf_model *m, const double *d_x, const double *d_lambda,
                                    double obj_weight, double *d_obj, double *d_grad, double *d_c,
                                    double *d_jvals, double *d_hvals, void *stream)
{
    using namespace opf;
    if (!m || !m->M) {
        set_error("NULL model");
        return OPF_EINVAL;
    }
    Model &M = *m->M;
    if (!M.on_device) {
        set_error("structure-only model: create it with opf_model_create / opf_batch_create to evaluate");
        return OPF_ESTATE;
    }
    if (!d_x || (d_hvals && !d_lambda)) {
        set_error("d_x is NULL, or d_lambda is NULL with d_hvals requested");
        return OPF_EINVAL;
    }
    // the fused one-kernel evaluation (bus_order 3 where the model allows
    // it) keeps its per-arc parts in registers and writes no arc scratch
    const bool fused = M.launch.bus_order == 3 && M.fuse_ok;
    if (!fused && M.narc_slots > kMaxSlots) {
        set_error("noalloc: model needs %lld arc scratch slots (%lld bytes); the static scratch "
                  "holds %lld slots (OPF_NOALLOC_SCRATCH_BYTES = %zu)",
                  (long long)M.narc_slots, (long long)(M.narc_slots * (int64_t)sizeof(ArcScratch)),
                  (long long)kMaxSlots, kScratchBytes);
        return OPF_EINVAL;
    }
    unsigned char *base = nullptr;
    int rc = scratch_address(M.device, &base);
    if (rc)
        return rc;
    unsigned int *ticket = reinterpret_cast<unsigned int *>(base);
    double *part = reinterpret_cast<double *>(base + kTicketBytes);
    ArcScratch *arcs = reinterpret_cast<ArcScratch *>(base + kTicketBytes + kPartBytes);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the objective's block counter must start at zero
    cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) {
        set_error("noalloc: cudaMemsetAsync failed: %s", cudaGetErrorString(e));
        return OPF_ECUDA;
    }
    EvalArgs a{d_x, d_lambda, obj_weight, d_obj, d_grad, d_c, d_jvals, d_hvals};
    const unsigned what = (d_obj ? W_OBJ : 0u) | (d_grad ? W_GRAD : 0u) | (d_c ? W_CONS : 0u) |
                          (d_jvals ? W_JAC : 0u) | (d_hvals ? W_HESS : 0u);
    if (!what)
        return OPF_OK;
    return launch_eval_scratch(M, a, what, s, arcs, part, kMaxPart, ticket);
}

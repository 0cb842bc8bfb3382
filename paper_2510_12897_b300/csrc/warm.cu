// Learned warm start (include/opf_warm.h): a three-layer BF16 MLP trained on
// the GPU with hand-written tensor-core GEMMs, penalty gradients from the
// library's own callback kernels (cons, grad, J^T v) and Adam.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cmath>
#include <random>
#include <vector>

#include "../../include/opf_warm.h"
#include "model.h"

namespace opf {
int build_model(const opf_network *nets, int32_t ninst, const opf_batch_opts *opts, bool device, Model **out);
void free_model(Model *M);
void bounds(const Model &M, double *xl, double *xu, double *gl, double *gu);
}  // namespace opf

using bf16 = __nv_bfloat16;
using namespace opf;

namespace {

#include "bits.cuh"

// ------------------------------------------------------------------ GEMM --
//
// C[M x N] = A[M x K] B[N x K]^T with BF16 operands and FP32 accumulation on
// the 5th-generation tensor cores. Both operands are row-major with K
// contiguous (the backward pass feeds transposed copies). Persistent: one
// CTA of 320 threads per SM walks the 128 x BN tiles of C (BN 256, or 128
// where N is not a multiple of 256), M-blocks fastest:
//   warp 0, one lane   TMA producer: 128 x 64 tiles of A and BN x 64 tiles
//                      of B (128-byte swizzle) into a ring of stages across
//                      the tiles, completion counted in bytes on the
//                      stage's "full" mbarrier;
//   warp 1, one lane   MMA issuer: per stage four tcgen05.mma (M 128, N BN,
//                      K 16) from shared-memory descriptors into one of two
//                      BN-column FP32 accumulators in tensor memory, tile
//                      after tile alternating; tcgen05.commit frees the
//                      stage ("empty") and, after a tile's last stage,
//                      hands the accumulator to the epilogue ("tfull");
//   warps 2-9          epilogue: tcgen05.ld of their 32 accumulator lanes
//                      (warp w reads lanes 32 (w mod 4) and up; two warps
//                      per lane quarter, half the columns each), 32 columns
//                      at a time, staged through shared memory into row
//                      segments, bias / GELU / GELU' in FP32, stores; then
//                      the accumulator is free again ("tempty"), so one
//                      tile's epilogue runs under the next tile's MMAs.
// Every wait on an mbarrier gives up after a bounded number of polls, or
// once another role gave up, and a timeout is recorded in a device flag the
// host reads (no unbounded spin). M must be a multiple of 128, N of 128, K
// of 64.

constexpr int UBM = 128, UBK = 64;
constexpr int kEpiWarps = 8;                      // two per accumulator lane quarter
constexpr int kGemmThreads = 64 + 32 * kEpiWarps;  // producer, MMA issuer, epilogue
constexpr uint32_t kWaitPolls = 1u << 22;

// the shared-memory plan of a tile width BN: the stage ring (A then B tile
// per stage), then the mbarriers full[S], empty[S], tfull[2], tempty[2],
// quiet, the tensor-memory address slot, and the epilogue warps' staging
// blocks
template <int BN>
struct GemmCfg {
    static constexpr int ATILE = UBM * UBK * 2;  // bytes of an A stage tile
    static constexpr int BTILE = BN * UBK * 2;   // bytes of a B stage tile
    static constexpr int STAGE = ATILE + BTILE;
    static constexpr int STAGES = BN == 256 ? 4 : 6;  // 192 KB of stages
    static constexpr int NBAR = 2 * STAGES + 5;
    static constexpr int STG_LD = 20;  // staging row stride in floats (16-byte aligned rows)
    static constexpr int STG = kEpiWarps * 32 * STG_LD * 4;  // one 32 x 16 FP32 block per epilogue warp
    static constexpr int SMEM = STAGES * STAGE + 1024 + 8 * NBAR + 32 + STG;  // + alignment slack
    static constexpr uint32_t TCOLS = 2 * BN;  // two accumulators
    // instruction descriptor of kind::f16: D FP32, A and B BF16, both
    // K-major, N >> 3 at bit 17, M >> 4 at bit 24
    static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                      ((uint32_t)(UBM >> 4) << 24);
};

// a tensor map with the height of its box (128 rows for A operands; 128 or
// 256 for B operands: the tile width BN of the GEMM that reads it)
struct GMap {
    CUtensorMap map;
    int box_rows;
};

__device__ int g_umma_timeout;  // set when a bounded wait gave up

enum Epi { EPI_BIAS_GELU, EPI_BIAS, EPI_DGELU, EPI_STORE };

struct GemmArgs {
    int M, N, K, ldc;
    int epi;
    const float *bias;    // [N]
    const float *zsaved;  // [M][ldc] pre-activations (EPI_DGELU)
    float *outf;          // [M][ldc] FP32 output (pre-activation, linear output, gradient)
    bf16 *outh;           // [M][ldc] BF16 output (activation, activation gradient), or null
};

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// wait for the completion of the barrier's phase of the given parity
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    for (uint32_t i = 0; i < kWaitPolls; i++) {
        uint32_t ok;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok)
            return true;
    }
    atomicExch(&g_umma_timeout, 1);
    return false;
}

// mbar_wait that also gives up (without recording a timeout) once another
// role of the CTA has raised the abort flag
__device__ __forceinline__ bool mbar_wait_live(uint32_t bar, uint32_t parity, volatile int *abort_flag)
{
    for (uint32_t i = 0; i < kWaitPolls; i++) {
        uint32_t ok;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok)
            return true;
        if (*abort_flag)
            return false;
    }
    atomicExch(&g_umma_timeout, 1);
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// shared-memory matrix descriptor: K-major tile of 128-byte rows, 128-byte
// swizzle, 8-row groups 1024 bytes apart (start address and offsets in
// 16-byte units; version 1; swizzle mode 2 = 128 bytes)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1u << 16) | ((uint64_t)(1024u >> 4) << 32) |
           ((uint64_t)1u << 46) | ((uint64_t)2u << 61);
}

__device__ __forceinline__ void umma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc)
{
    asm volatile("{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(tmem),
                 "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 32 consecutive accumulator columns of the warp's 32 lanes, one per thread
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t r[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// GELU, tanh form: 0.5 z (1 + tanh u) = z / (1 + exp(-2u)), u = k0 (z + k1
// z^3), the logistic form (no cancellation for negative z); the fast
// exponential and division keep its relative error near 1e-6, far below the
// BF16 rounding of the activation it feeds (the argument is clamped at 80 so
// that the denominator stays finite; there the result is below 1e-34 |z|)
__device__ __forceinline__ float gelu(float z)
{
    const float k0 = 0.7978845608028654f, k1 = 0.044715f;
    const float m2u = -2.0f * k0 * fmaf(k1 * z, z * z, z);
    return __fdividef(z, 1.0f + __expf(fminf(m2u, 80.0f)));
}

// its derivative, from the tanh form (FP32 library tanh: it feeds FP32
// gradients)
__device__ __forceinline__ float gelu_grad(float z)
{
    const float k0 = 0.7978845608028654f, k1 = 0.044715f;
    const float t = tanhf(k0 * (z + k1 * z * z * z));
    return 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * k0 * (1.0f + 3.0f * k1 * z * z);
}

template <int BN>
__global__ void __launch_bounds__(kGemmThreads, 1) umma_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                                                           const __grid_constant__ CUtensorMap tmB, const GemmArgs g)
{
    using C = GemmCfg<BN>;
    extern __shared__ uint8_t smem_raw[];
    // set by a role whose bounded wait gave up: every role stops issuing,
    // and the epilogue writes nothing more
    __shared__ int s_abort;
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;  // 1024-byte aligned tiles
    const uint32_t bars = base + C::STAGES * C::STAGE;
    const uint32_t slot = bars + 8u * C::NBAR;
    uint32_t *slot_ptr = reinterpret_cast<uint32_t *>(smem_raw + (slot - raw));
    const uint32_t stg_at = (slot + 4u + 15u) & ~15u;  // after the slot, 16-byte aligned
    float *stage_f = reinterpret_cast<float *>(smem_raw + (stg_at - raw));
    auto full = [&](int st) { return bars + 8u * st; };
    auto empty = [&](int st) { return bars + 8u * (C::STAGES + st); };
    auto tfull = [&](int a) { return bars + 8u * (2 * C::STAGES + a); };
    auto tempty = [&](int a) { return bars + 8u * (2 * C::STAGES + 2 + a); };
    const uint32_t quiet = bars + 8u * (2 * C::STAGES + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mt = g.M / UBM, tiles = mt * (g.N / BN), nk = g.K / UBK;

    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int st = 0; st < C::STAGES; st++) {
            mbar_init(full(st), 1);
            mbar_init(empty(st), 1);
        }
        for (int a = 0; a < 2; a++) {
            mbar_init(tfull(a), 1);
            mbar_init(tempty(a), 32 * kEpiWarps);  // every epilogue thread arrives
        }
        mbar_init(quiet, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {  // two accumulators of BN columns
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(C::TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *slot_ptr;
    volatile int *abort_flag = &s_abort;

    int issued = 0;  // producer: stage loads issued (k steps over all its tiles)
    if (warp == 0) {
        if (lane == 0) {  // producer
            int it = 0;
            bool stop = false;
            for (int tile = blockIdx.x; tile < tiles && !stop; tile += gridDim.x) {
                const int bm = (tile % mt) * UBM, bn = (tile / mt) * BN;
                for (int kt = 0; kt < nk; kt++, it++) {
                    const int st = it % C::STAGES, round = it / C::STAGES;
                    if (*abort_flag ||
                        (round > 0 && !mbar_wait_live(empty(st), (round - 1) & 1, abort_flag))) {
                        stop = true;
                        break;
                    }
                    const uint32_t sa = base + st * C::STAGE;
                    mbar_expect_tx(full(st), C::STAGE);
                    tma_load_2d(sa, &tmA, kt * UBK, bm, full(st));
                    tma_load_2d(sa + C::ATILE, &tmB, kt * UBK, bn, full(st));
                    issued = it + 1;
                }
            }
            if (stop)
                *abort_flag = 1;
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            int it = 0, j = 0;
            bool stop = false;
            for (int tile = blockIdx.x; tile < tiles && !stop; tile += gridDim.x, j++) {
                const int acc = j & 1, use = j >> 1;
                // the accumulator's previous tile must have left tensor memory
                if (use > 0 && !mbar_wait_live(tempty(acc), (use - 1) & 1, abort_flag)) {
                    stop = true;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(acc * BN);
                for (int kt = 0; kt < nk; kt++, it++) {
                    const int st = it % C::STAGES, round = it / C::STAGES;
                    if (!mbar_wait_live(full(st), round & 1, abort_flag)) {
                        stop = true;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t sa = base + st * C::STAGE, sb = sa + C::ATILE;
#pragma unroll
                    for (int k = 0; k < UBK / 16; k++)  // 16 elements = 32 bytes along K per MMA
                        umma(d, smem_desc(sa + 32 * k), smem_desc(sb + 32 * k), C::IDESC, (kt | k) != 0);
                    umma_commit(empty(st));
                }
                if (!stop)
                    umma_commit(tfull(acc));
            }
            if (stop)
                *abort_flag = 1;
            // also after a stop: quiet then arrives once every MMA issued
            // above has completed, so tensor memory is idle before dealloc
            umma_commit(quiet);
        }
        __syncwarp();
    } else {  // epilogue: warp w reads accumulator lanes 32 (w mod 4) .. + 31,
              // warps 2-5 the first half of the columns, warps 6-9 the second
        const int e = warp - 2, q = warp & 3;
        const int c0 = (e >> 2) * (BN / 64), c1 = c0 + BN / 64;  // its 32-column chunks
        float *stg = stage_f + e * (32 * C::STG_LD);
        const int cg = lane & 3, rs = lane >> 2;
        int j = 0;
        for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x, j++) {
            const int acc = j & 1, use = j >> 1;
            if (!mbar_wait_live(tfull(acc), use & 1, abort_flag)) {
                *abort_flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int bm = (tile % mt) * UBM, bn = (tile / mt) * BN;
            const uint32_t tb = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * BN);
            // each 32 x 16 half of a chunk: thread = row out of tensor
            // memory, into the warp's staging block, back out as 4 threads
            // per 64-byte row segment (8 rows per instruction) for the
            // epilogue and coalesced stores
#pragma unroll 1
            for (int c = c0; c < c1; c++) {
                uint32_t r[32];
                tmem_ld32(tb + 32 * c, r);
#pragma unroll
                for (int hh = 0; hh < 2; hh++) {
#pragma unroll
                    for (int qq = 0; qq < 4; qq++)
                        *reinterpret_cast<float4 *>(stg + lane * C::STG_LD + 4 * qq) =
                            make_float4(__uint_as_float(r[16 * hh + 4 * qq]), __uint_as_float(r[16 * hh + 4 * qq + 1]),
                                        __uint_as_float(r[16 * hh + 4 * qq + 2]),
                                        __uint_as_float(r[16 * hh + 4 * qq + 3]));
                    __syncwarp();
                    const int n = bn + 32 * c + 16 * hh + 4 * cg;  // this thread's 4 columns
                    float4 bb = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (g.epi == EPI_BIAS_GELU || g.epi == EPI_BIAS)
                        bb = __ldg(reinterpret_cast<const float4 *>(g.bias + n));
#pragma unroll 2
                    for (int rr = 0; rr < 4; rr++) {
                        const int rl = 8 * rr + rs;  // row within the warp's 32
                        float4 v = *reinterpret_cast<const float4 *>(stg + rl * C::STG_LD + 4 * cg);
                        const size_t at = (size_t)(bm + 32 * q + rl) * g.ldc + n;
                        if (g.epi == EPI_BIAS_GELU || g.epi == EPI_BIAS) {
                            v.x += bb.x;
                            v.y += bb.y;
                            v.z += bb.z;
                            v.w += bb.w;
                        } else if (g.epi == EPI_DGELU) {
                            const float4 z = *reinterpret_cast<const float4 *>(g.zsaved + at);
                            v.x *= gelu_grad(z.x);
                            v.y *= gelu_grad(z.y);
                            v.z *= gelu_grad(z.z);
                            v.w *= gelu_grad(z.w);
                        }
                        *reinterpret_cast<float4 *>(g.outf + at) = v;
                        if (g.outh) {
                            const bool act = g.epi == EPI_BIAS_GELU;
                            __nv_bfloat162 h[2];
                            h[0] = act ? __floats2bfloat162_rn(gelu(v.x), gelu(v.y)) : __floats2bfloat162_rn(v.x, v.y);
                            h[1] = act ? __floats2bfloat162_rn(gelu(v.z), gelu(v.w)) : __floats2bfloat162_rn(v.z, v.w);
                            *reinterpret_cast<uint2 *>(g.outh + at) = *reinterpret_cast<const uint2 *>(h);
                        }
                    }
                    __syncwarp();  // the block is read before the next one is staged
                }
            }
            // this thread's reads of the accumulator are complete (the
            // loads waited): the MMA issuer may overwrite it
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(tempty(acc));
        }
    }

    // every MMA issued has completed once quiet's first phase has
    mbar_wait(quiet, 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0 && lane == 0 && *abort_flag) {
        // the producer's own copies in flight: wait (bounded) for the last
        // load phase of each stage it used, so that no TMA write lands in
        // shared memory after the block exits (phases of one barrier
        // complete in order, so the last one implies the earlier ones)
        for (int kt = issued > C::STAGES ? issued - C::STAGES : 0; kt < issued; kt++)
            mbar_wait(full(kt % C::STAGES), (kt / C::STAGES) & 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1)  // always freed, also after a stop
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TCOLS));
}

// out [C][R] = in [R][C]^T (BF16; R and C multiples of 32), 32 x 32 tiles
__global__ void transpose_bf16_kernel(const bf16 *in, int R, int C, bf16 *out)
{
    __shared__ unsigned short t[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    const unsigned short *src = reinterpret_cast<const unsigned short *>(in);
    unsigned short *dst = reinterpret_cast<unsigned short *>(out);
    for (int y = threadIdx.y; y < 32; y += blockDim.y)
        t[y][threadIdx.x] = src[(size_t)(r0 + y) * C + c0 + threadIdx.x];
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y)
        dst[(size_t)(c0 + y) * R + r0 + threadIdx.x] = t[threadIdx.x][y];
}

cudaError_t transpose(const bf16 *in, int R, int C, bf16 *out, cudaStream_t s)
{
    transpose_bf16_kernel<<<dim3(C / 32, R / 32), dim3(32, 8), 0, s>>>(in, R, C, out);
    return cudaGetLastError();
}

// the tile width of a GEMM whose C has N columns
int tile_n(int N)
{
    return N % 256 == 0 ? 256 : 128;
}

// one persistent launch: min(tiles, SMs) CTAs; the shapes, the maps' box
// heights and the alignment of the epilogue's vector accesses are checked
// here, before anything runs
cudaError_t gemm(const GMap &A, const GMap &B, const GemmArgs &g, cudaStream_t s)
{
    const int bn = B.box_rows;
    auto misaligned = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) != 0; };
    if (A.box_rows != UBM || bn != tile_n(g.N) || g.M <= 0 || g.N <= 0 || g.K <= 0 || g.M % UBM ||
        g.N % bn || g.K % UBK || g.ldc % 8 || misaligned(g.bias) || misaligned(g.zsaved) ||
        misaligned(g.outf) || misaligned(g.outh))
        return cudaErrorInvalidValue;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
        return e;
    const int tiles = (g.M / UBM) * (g.N / bn);
    const int grid = tiles < sms ? tiles : sms;
    if (bn == 256)
        umma_gemm_kernel<256><<<grid, kGemmThreads, GemmCfg<256>::SMEM, s>>>(A.map, B.map, g);
    else
        umma_gemm_kernel<128><<<grid, kGemmThreads, GemmCfg<128>::SMEM, s>>>(A.map, B.map, g);
    return cudaGetLastError();
}

// tensor map of a row-major [rows][k] BF16 matrix, boxes of box_rows rows x
// 64 (128 bytes, the swizzle span)
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

bool make_map(GMap *m, const bf16 *ptr, int rows, int k, int box_rows)
{
    static EncodeTiled encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = reinterpret_cast<EncodeTiled>(fn);
    }
    if (rows % box_rows)
        return false;
    m->box_rows = box_rows;
    const cuuint64_t dims[2] = {(cuuint64_t)k, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)k * 2};
    const cuuint32_t box[2] = {UBK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return encode(&m->map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16 *>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// A operand [M][K]: boxes of 128 rows; B operand [N][K]: boxes of the
// GEMM's tile width
bool map_a(GMap *m, const bf16 *ptr, int rows, int k)
{
    return make_map(m, ptr, rows, k, UBM);
}

bool map_b(GMap *m, const bf16 *ptr, int rows, int k)
{
    return make_map(m, ptr, rows, k, tile_n(rows));
}

// ------------------------------------------------------------- elementwise --

// The element-wise kernels below take kBatch elements per thread and loop
// step, their loads issued before any of their arithmetic, so that each
// thread keeps kBatch loads in flight (one at a time left these kernels at
// a fraction of the memory bandwidth); every thread still visits its
// elements in the same order.
constexpr int kBatch = 4;

// The FP64 work of these kernels is rare (a violated bound, a nonzero
// residual), so it sits behind a warp vote: a warp in which no lane needs it
// skips the instructions, which would otherwise issue for the whole warp
// (predicated, or computed on every lane and selected). Each lane's result
// does not depend on the vote.

// x - clip(x, lo, hi), the subtraction only in warps with a lane outside
__device__ __forceinline__ double excess_w(double x, double lo, double hi)
{
    const long long kx = order_key(x);
    const bool below = kx < order_key(lo), above = kx > order_key(hi);
    double r = 0.0;
    if (__any_sync(__activemask(), below || above))
        r = below ? x - lo : above ? x - hi : 0.0;
    return r;
}

// x - clip(x, -h, h), h >= 0, likewise
__device__ __forceinline__ double excess_sym_w(double x, double h)
{
    const bool out = (__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFll) > __double_as_longlong(h);
    double r = 0.0;
    if (__any_sync(__activemask(), out))
        r = excess_sym(x, h);
    return r;
}

// acc + r^2, the FMA only in warps with a nonzero r
__device__ __forceinline__ double add_square_w(double acc, double r)
{
    return __any_sync(__activemask(), !is_zero(r)) ? fma(r, r, acc) : acc;
}

struct WarmDev {
    int B, nb, ng, nl, nload, Kin, Nout, nbp, ngp, ref;
    double va_scale, penalty;
    const float *pk, *qk;                    // 5 / base load (0 where the base is 0)
    const double *vmin, *vmax;               // per bus
    const double *pmin, *pmax, *qmin, *qmax; // per generator
    const double *angmin, *angmax, *rate;    // per branch
    // (lo + hi) / 2 and (hi - lo) / 2 of vm, pg, qg (the output map's terms)
    const double *vmid, *pmid, *phalf, *qmid, *qhalf;
    double inv_b;  // 1 / B
};

// u = normalised loads (BF16, zero padding): (load / base - 1) / 0.2 as one
// FP32 FMA with the precomputed 5 / base (0 where the base load is 0); the
// result is rounded to BF16 anyway
// one load's input entry j of a profile whose loads start at ps, qs
__device__ __forceinline__ float input_of(const WarmDev &w, const double *ps, const double *qs, int j, double v)
{
    if (j < w.nload) {
        const float k = w.pk[j];
        return k != 0.f ? fmaf(f32_rn(v), k, -5.f) : 0.f;
    }
    if (j < 2 * w.nload) {
        const float k = w.qk[j - w.nload];
        return k != 0.f ? fmaf(f32_rn(v), k, -5.f) : 0.f;
    }
    return 0.f;
}

// grid (column blocks, profile blocks); each warp takes 256 consecutive
// entries of a row as 8 rounds of 32 (coalesced loads, eight in flight per
// thread; 64-byte stores); rows y, y + gridDim.y, ... per block row
__global__ void prep_kernel(const WarmDev w, const double *pd, const double *qd, bf16 *U)
{
    const int jb = blockIdx.x * (blockDim.x * 8) + (threadIdx.x >> 5) * 256 + (threadIdx.x & 31);
    if (jb >= w.Kin)
        return;
    for (int s = blockIdx.y; s < w.B; s += gridDim.y) {
        const double *ps = pd + (int64_t)s * w.nload, *qs = qd + (int64_t)s * w.nload;
        bf16 *us = U + (int64_t)s * w.Kin;
        double v[8];
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const int j = jb + 32 * q;
            v[q] = j < w.nload ? __ldg(ps + j) : j < 2 * w.nload ? __ldg(qs + j - w.nload) : 0.0;
        }
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const int j = jb + 32 * q;
            if (j < w.Kin)
                us[j] = __float2bfloat16_rn(input_of(w, ps, qs, j, v[q]));
        }
    }
}

// network output y = [ya | yv | yp | yq] (block widths nbp, nbp, ngp, ngp)
// -> va, vm, pg, qg of the batch model (period t = profile t): va = va_scale
// ya (0 at the reference bus), vm = mid + yv, pg = mid + half-range yp, qg
// likewise; y = 0 is the flat start
// block b takes the periods b, b + gridDim.x, ...; its threads walk a
// period's outputs (no division); the FP32 outputs are widened exactly on
// the integer pipe
__global__ void map_kernel(const WarmDev w, const float *__restrict__ Y, double *__restrict__ x)
{
    const int per = 2 * w.nb + 2 * w.ng;
    const int64_t nbT = (int64_t)w.nb * w.B, ngT = (int64_t)w.ng * w.B;
    for (int t = blockIdx.x; t < w.B; t += gridDim.x) {
        const float *y = Y + (int64_t)t * w.Nout;
        for (int j0 = threadIdx.x; j0 < per; j0 += kBatch * blockDim.x) {
            float yv[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; u++) {  // output column of entry j
                const int j = j0 + u * blockDim.x;
                const int col = j < w.nb ? j : j < 2 * w.nb ? w.nbp + j - w.nb
                                : j < 2 * w.nb + w.ng ? 2 * w.nbp + j - 2 * w.nb
                                                      : 2 * w.nbp + w.ngp + j - 2 * w.nb - w.ng;
                yv[u] = __ldg(y + (j < per ? col : 0));
            }
#pragma unroll
            for (int u = 0; u < kBatch; u++) {
                const int j = j0 + u * blockDim.x;
                if (j >= per)
                    break;
                if (j < w.nb) {
                    x[(int64_t)w.nb * t + j] = j == w.ref ? 0.0 : w.va_scale * widen(yv[u]);
                } else if (j < 2 * w.nb) {
                    const int i = j - w.nb;
                    x[nbT + (int64_t)w.nb * t + i] = w.vmid[i] + widen(yv[u]);
                } else if (j < 2 * w.nb + w.ng) {
                    const int g = j - 2 * w.nb;
                    x[2 * nbT + (int64_t)w.ng * t + g] = fma(w.phalf[g], widen(yv[u]), w.pmid[g]);
                } else {
                    const int g = j - 2 * w.nb - w.ng;
                    x[2 * nbT + ngT + (int64_t)w.ng * t + g] = fma(w.qhalf[g], widen(yv[u]), w.qmid[g]);
                }
            }
        }
    }
}

__device__ __forceinline__ double block_sum(double acc, double *red)
{
    for (int off = 16; off; off >>= 1)
        acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0)
        red[threadIdx.x >> 5] = acc;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < (int)(blockDim.x >> 5); q++)
            s += red[q];
    return s;
}

// Bounds of the batch model's rows and variables from their structure (no
// bound arrays read): rows [ref | 4 flow groups | angle | P, Q balance |
// thermal from, to], each group [period][element]; only the angle rows
// ([angmin, angmax] of the branch) and the thermal rows ((-inf, 0]) are not
// equalities. Variables [va | vm | pg | qg | p | q]: va free, vm in
// [vmin, vmax], pg, qg in their limits, p, q in [-rate_a, rate_a].
__device__ __forceinline__ void row_bounds(const WarmDev &w, int64_t r, double &lo, double &hi)
{
    const int64_t T = w.B, nlT = (int64_t)w.nl * T, nbT = (int64_t)w.nb * T;
    lo = 0.0;
    hi = 0.0;
    if (r >= T + 4 * nlT && r < T + 5 * nlT) {
        const unsigned k = (unsigned)(r - T - 4 * nlT) % (unsigned)w.nl;  // 32-bit: the batch model has < 2^31 rows
        lo = w.angmin[k];
        hi = w.angmax[k];
    } else if (r >= T + 5 * nlT + 2 * nbT) {
        lo = -INFINITY;
    }
}

__device__ __forceinline__ bool var_bounds(const WarmDev &w, int64_t j, double &lo, double &hi)
{
    const int64_t T = w.B, nbT = (int64_t)w.nb * T, ngT = (int64_t)w.ng * T, naT = 2 * (int64_t)w.nl * T;
    if (j < nbT)
        return false;  // va
    // 32-bit remainders: the batch model has fewer than 2^31 variables
    if (j < 2 * nbT) {
        const unsigned i = (unsigned)(j - nbT) % (unsigned)w.nb;
        lo = w.vmin[i];
        hi = w.vmax[i];
    } else if (j < 2 * nbT + ngT) {
        const unsigned g = (unsigned)(j - 2 * nbT) % (unsigned)w.ng;
        lo = w.pmin[g];
        hi = w.pmax[g];
    } else if (j < 2 * nbT + 2 * ngT) {
        const unsigned g = (unsigned)(j - 2 * nbT - ngT) % (unsigned)w.ng;
        lo = w.qmin[g];
        hi = w.qmax[g];
    } else {
        int64_t off = j - 2 * nbT - 2 * ngT;  // p block, then q block, each [period][arc]
        if (off >= naT)
            off -= naT;
        const unsigned k = (unsigned)off % (unsigned)w.nl;  // arc k and nl + k share branch k's rating
        hi = w.rate[k];
        lo = -hi;
    }
    return true;
}

// one-time check at creation: the structured bounds equal the model's
__global__ void bounds_check_kernel(const WarmDev w, const double *xl, const double *xu, int64_t n,
                                    const double *gl, const double *gu, int64_t m, unsigned *bad)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m + n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double lo = -INFINITY, hi = INFINITY;
        bool ok;
        if (i < m) {
            row_bounds(w, i, lo, hi);
            ok = lo == gl[i] && hi == gu[i];
        } else {
            var_bounds(w, i - m, lo, hi);
            ok = lo == xl[i - m] && hi == xu[i - m];
        }
        if (!ok)
            atomicAdd(bad, 1u);
    }
}

// constraint rows: rho = c - clip(c, gl, gu); v1 = (2 penalty / B) rho;
// per-block sums of rho^2 into part. The rows with bounds [0, 0] (flow,
// balance and reference rows) have rho = c: only the angle and thermal rows
// clip
__global__ void resid_kernel(const WarmDev w, const double *__restrict__ c, int64_t m, double *__restrict__ v1,
                             double *part)
{
    __shared__ double red[32];
    double acc = 0.0;
    const double k = 2.0 * w.penalty / w.B;
    const int64_t T = w.B, nlT = (int64_t)w.nl * T, nbT = (int64_t)w.nb * T;
    const int64_t a0 = T + 4 * nlT, a1 = T + 5 * nlT, th = T + 5 * nlT + 2 * nbT;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < m; i0 += kBatch * stride) {
        double cv[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; u++) {
            const int64_t i = i0 + u * stride;
            cv[u] = i < m ? __ldg(c + i) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kBatch; u++) {
            const int64_t i = i0 + u * stride;
            if (i >= m)
                break;
            const double ci = cv[u];
            double rho = ci;
            if (i >= a0 && i < a1) {  // angle rows
                const unsigned kk = (unsigned)(i - a0) % (unsigned)w.nl;  // 32-bit: the batch model has < 2^31 rows
                rho = excess_w(ci, w.angmin[kk], w.angmax[kk]);
            } else if (i >= th) {  // thermal rows: (-inf, 0]
                rho = order_key(ci) > 0 ? ci : 0.0;
            }
            // two FP64 instructions per row: the floor of this kernel on this
            // GPU (a vote to skip the zero rows measured slower: the balance
            // rows are nonzero in every warp)
            v1[i] = k * rho;
            acc = fma(rho, rho, acc);
        }
    }
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0)
        part[blockIdx.x] = s;
}

// variable e of a period's bounded entries (vm, pg, qg, p, q; va has no
// bounds): its index in period t and its bounds ([-hi, hi] where sym)
struct BoundRef {
    int64_t j;
    double lo, hi;
    bool sym;
};

__device__ __forceinline__ BoundRef bound_ref(const WarmDev &w, int t, int e)
{
    const int nb = w.nb, ng = w.ng, nl = w.nl, na = 2 * nl;
    const int64_t T = w.B, nbT = (int64_t)nb * T, ngT = (int64_t)ng * T, naT = (int64_t)na * T;
    BoundRef r;
    r.sym = false;
    if (e < nb) {
        r.j = nbT + (int64_t)nb * t + e;
        r.lo = w.vmin[e];
        r.hi = w.vmax[e];
    } else if (e < nb + ng) {
        const int g = e - nb;
        r.j = 2 * nbT + (int64_t)ng * t + g;
        r.lo = w.pmin[g];
        r.hi = w.pmax[g];
    } else if (e < nb + 2 * ng) {
        const int g = e - nb - ng;
        r.j = 2 * nbT + ngT + (int64_t)ng * t + g;
        r.lo = w.qmin[g];
        r.hi = w.qmax[g];
    } else {  // p block, then q block, each [period][arc]; arcs k and nl + k share branch k's rating
        int a = e - nb - 2 * ng;
        r.j = 2 * nbT + 2 * ngT + (int64_t)na * t;
        if (a >= na) {
            a -= na;
            r.j += naT;
        }
        r.j += a;
        r.hi = w.rate[a < nl ? a : a - nl];
        r.lo = 0.0;
        r.sym = true;
    }
    return r;
}

// variable bounds: per-block sums of r^2, r = x - clip(x, xl, xu) (their
// gradient enters through the flow multipliers for p, q and through the
// output map for vm, pg, qg); only violated bounds add. Block b takes the
// periods b, b + gridDim.x, ...; its threads walk a period's bounded
// entries, so every bound is indexed directly, with no division
__global__ void bound_kernel(const WarmDev w, const double *__restrict__ x, double *part)
{
    __shared__ double red[32];
    double acc = 0.0;
    const int per = w.nb + 2 * w.ng + 4 * w.nl;
    for (int t = blockIdx.x; t < w.B; t += gridDim.x) {
        for (int e0 = threadIdx.x; e0 < per; e0 += kBatch * blockDim.x) {
            BoundRef br[kBatch];
            double xv[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; u++) {
                const int e = e0 + u * blockDim.x;
                br[u] = bound_ref(w, t, e < per ? e : 0);
                xv[u] = __ldg(x + br[u].j);
            }
#pragma unroll
            for (int u = 0; u < kBatch; u++) {
                if (e0 + u * (int)blockDim.x >= per)
                    break;
                const double r = br[u].sym ? excess_sym_w(xv[u], br[u].hi) : excess_w(xv[u], br[u].lo, br[u].hi);
                acc = add_square_w(acc, r);
            }
        }
    }
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0)
        part[blockIdx.x] = s;
}

// The flow variables are functions of the voltages (p, q = F(va, vm)), so
// the gradient of the penalised loss with respect to the voltages is
// J_v^T v1 + J_v(F)^T g_pq, g_pq the loss's gradient in the arc variables:
// the thermal and balance rows where each arc variable appears, plus its
// bound term. Since a flow row is (own arc variable) - F, J_v(F) = -J_v(flow
// row), and the whole gradient is J_v^T v2 with v2 = v1 except on the flow
// rows, where v2 = -g_own = -(2 x_own v_thermal + v_balance + k r_own),
// k = 2 penalty / B. This kernel overwrites the flow rows of v1 with v2 (one
// thread per branch and period, its four arc variables).
// Block b takes the periods b, b + gridDim.x, ...; its threads the
// branches, two per loop step with every load issued first. The clip, the
// doubling and the signs are exact integer work or free FMA operand
// negations: one FMA per arc variable, a second where its bound is violated.
__global__ void flowmult_kernel(const WarmDev w, const int4 *__restrict__ br, const double *__restrict__ x,
                                double *v)
{
    constexpr int NB = 2;  // branches per thread and loop step
    const int64_t T = w.B, nl = w.nl, nb = w.nb, ng = w.ng, na = 2 * nl;
    const int64_t nlT = nl * T, nbT = nb * T, ngT = ng * T;
    const double kpen = 2.0 * w.penalty / w.B;
    for (int t = blockIdx.x; t < w.B; t += gridDim.x) {
        const int64_t ip = 2 * nbT + 2 * ngT + na * t, iq = ip + na * T;
        const int64_t bal = T + 5 * nlT + nb * t;  // P balance of bus 0 in period t; + nbT: Q
        for (int k0 = threadIdx.x; k0 < w.nl; k0 += NB * blockDim.x) {
            int4 bb[NB];
            double xo[NB][4], vt[NB][2], vbv[NB][4], rate[NB];
#pragma unroll
            for (int u = 0; u < NB; u++) {
                const int k = min(k0 + u * (int)blockDim.x, w.nl - 1);  // past the end: a valid branch, not stored
                bb[u] = __ldg(br + k);
                rate[u] = w.rate[k];
                xo[u][0] = __ldg(x + ip + k);
                xo[u][1] = __ldg(x + iq + k);
                xo[u][2] = __ldg(x + ip + nl + k);
                xo[u][3] = __ldg(x + iq + nl + k);
                const int64_t th = T + 5 * nlT + 2 * nbT + nl * t + k;  // thermal row (from); + nlT: to
                vt[u][0] = v[th];
                vt[u][1] = v[th + nlT];
            }
#pragma unroll
            for (int u = 0; u < NB; u++) {
                vbv[u][0] = v[bal + bb[u].x];
                vbv[u][1] = v[bal + nbT + bb[u].x];
                vbv[u][2] = v[bal + bb[u].y];
                vbv[u][3] = v[bal + nbT + bb[u].y];
            }
#pragma unroll
            for (int u = 0; u < NB; u++) {
                const int k = k0 + u * blockDim.x;
                if (k >= w.nl)
                    break;
                const int64_t it = nl * t + k;
#pragma unroll
                for (int g = 0; g < 4; g++) {
                    const double r = excess_sym_w(xo[u][g], rate[u]);
                    double out = fma(-twice(xo[u][g]), vt[u][g < 2 ? 0 : 1], -vbv[u][g]);
                    if (__any_sync(__activemask(), !is_zero(r)))
                        out = fma(-kpen, r, out);
                    v[T + it + g * nlT] = out;
                }
            }
        }
    }
}

// batch means: loss, cost, sum of squared residuals (constraints and bounds);
// one warp, lane-strided partial sums then a fixed shuffle tree
__global__ void stats_kernel(const WarmDev w, const double *part, int nparts, const double *obj,
                             double *stats)
{
    double r = 0.0;
    for (int q = threadIdx.x; q < nparts; q += 32)
        r += part[q];
    for (int off = 16; off; off >>= 1)
        r += __shfl_down_sync(0xffffffffu, r, off);
    if (threadIdx.x == 0) {
        const double cost = obj[0] / w.B, res = r / w.B;
        stats[0] = cost + w.penalty * res;
        stats[1] = cost;
        stats[2] = res;
    }
}

// dL/dy from dL/dx = u (J^T v2) + the bound term + grad f / B (on pg),
// through the output map: FP32 for the checks and the bias gradient, BF16
// copies for the GEMMs; padding entries and the reference angle get 0
// block b takes the periods b, b + gridDim.x, ...; its threads walk a
// period's outputs (no division); clips and conversions on the integer pipe
__global__ void dmap_kernel(const WarmDev w, const double *__restrict__ x, const double *__restrict__ u2,
                            const double *__restrict__ gradf, float *__restrict__ dYf, bf16 *__restrict__ dYh)
{
    const int64_t nbT = (int64_t)w.nb * w.B, ngT = (int64_t)w.ng * w.B;
    const double k = 2.0 * w.penalty / w.B;
    for (int t = blockIdx.x; t < w.B; t += gridDim.x) {
        for (int j0 = threadIdx.x; j0 < w.Nout; j0 += kBatch * blockDim.x) {
            // the entry's block (0 va, 1 vm, 2 pg, 3 qg; -1 padding or the
            // reference angle), element, variable index, and its loads
            int blk[kBatch], el[kBatch];
            double uv[kBatch], xv[kBatch], gv[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; u++) {
                const int j = j0 + u * blockDim.x;
                int b = -1, e = 0;
                int64_t i = 0;
                if (j < w.nbp) {
                    if (j < w.nb && j != w.ref) {
                        b = 0;
                        e = j;
                        i = (int64_t)w.nb * t + j;
                    }
                } else if (j < 2 * w.nbp) {
                    e = j - w.nbp;
                    if (e < w.nb) {
                        b = 1;
                        i = nbT + (int64_t)w.nb * t + e;
                    }
                } else if (j < 2 * w.nbp + w.ngp) {
                    e = j - 2 * w.nbp;
                    if (e < w.ng) {
                        b = 2;
                        i = 2 * nbT + (int64_t)w.ng * t + e;
                    }
                } else if (j < w.Nout) {
                    e = j - 2 * w.nbp - w.ngp;
                    if (e < w.ng) {
                        b = 3;
                        i = 2 * nbT + ngT + (int64_t)w.ng * t + e;
                    }
                }
                blk[u] = b;
                el[u] = e;
                uv[u] = b >= 0 ? __ldg(u2 + i) : 0.0;
                xv[u] = b >= 1 ? __ldg(x + i) : 0.0;
                gv[u] = b == 2 ? __ldg(gradf + i) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < kBatch; u++) {
                const int j = j0 + u * blockDim.x;
                if (j >= w.Nout)
                    break;
                const int e = el[u];
                double d = 0.0;
                if (blk[u] == 0) {
                    d = w.va_scale * uv[u];
                } else if (blk[u] == 1) {
                    d = uv[u];
                    const double r = excess_w(xv[u], w.vmin[e], w.vmax[e]);
                    if (__any_sync(__activemask(), !is_zero(r)))
                        d = fma(k, r, d);
                } else if (blk[u] == 2) {
                    double a = fma(gv[u], w.inv_b, uv[u]);
                    const double r = excess_w(xv[u], w.pmin[e], w.pmax[e]);
                    if (__any_sync(__activemask(), !is_zero(r)))
                        a = fma(k, r, a);
                    d = w.phalf[e] * a;
                } else if (blk[u] == 3) {
                    double a = uv[u];
                    const double r = excess_w(xv[u], w.qmin[e], w.qmax[e]);
                    if (__any_sync(__activemask(), !is_zero(r)))
                        a = fma(k, r, a);
                    d = w.qhalf[e] * a;
                }
                const int64_t at = (int64_t)w.Nout * t + j;
                const float df = f32_rn(d);
                dYf[at] = df;
                dYh[at] = __float2bfloat16_rn(df);
            }
        }
    }
}

// column sums of a [rows][cols] FP32 matrix (bias gradients): a block of
// 32 x 32 threads per 32 columns; thread (c, r) sums rows r, r + 32, ... of
// column c, then row 0 of the block adds the 32 partials in order
__global__ void colsum_kernel(const float *X, int rows, int cols, float *out)
{
    __shared__ float part[32][33];
    const int c = blockIdx.x * 32 + threadIdx.x;
    float acc = 0.f;
    if (c < cols)
        for (int i = threadIdx.y; i < rows; i += 32)
            acc += X[(int64_t)i * cols + c];
    part[threadIdx.y][threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.y == 0 && c < cols) {
        float s = 0.f;
        for (int r = 0; r < 32; r++)
            s += part[r][threadIdx.x];
        out[c] = s;
    }
}

__global__ void to_bf16_kernel(const float *x, bf16 *y, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

// Adam (Kingma and Ba) on a range of the flat FP32 parameters
__global__ void adam_kernel(float *p, const float *g, float *m1, float *m2, int64_t n, float lr,
                            float bc1, float bc2)
{
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float a = b1 * m1[i] + (1.f - b1) * gi;
        const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
        m1[i] = a;
        m2[i] = b;
        p[i] -= lr * (a / bc1) / (sqrtf(b / bc2) + eps);
    }
}

int grid1(int64_t n, int block = 256)
{
    int64_t g = (n + block - 1) / block;
    if (g > 148 * 16)
        g = 148 * 16;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

struct opf_warm {
    Model *M = nullptr;  // callback model: B periods of the network
    int B = 0, H = 0, Kin = 0, Nout = 0, nb = 0, ng = 0, nl = 0, nload = 0, ref = 0;
    int nbp = 0, ngp = 0;
    int64_t n = 0, m = 0, n1 = 0;
    double penalty = 1e3, lr = 1e-4, lr_out = 1e-2, va_scale = 1.0;
    int64_t nparams = 0, oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0;
    int64_t step = 0;
    std::vector<void *> allocs;
    float *params = nullptr, *grads = nullptr, *am = nullptr, *av = nullptr;
    bf16 *W1h = nullptr, *W2h = nullptr, *W3h = nullptr;
    float *pk = nullptr, *qk = nullptr;
    double *vmid = nullptr, *pmid = nullptr, *phalf = nullptr, *qmid = nullptr, *qhalf = nullptr;
    double *vmin = nullptr, *vmax = nullptr, *pmin = nullptr,
           *pmax = nullptr, *qmin = nullptr, *qmax = nullptr, *gl = nullptr, *gu = nullptr,
           *xl = nullptr, *xu = nullptr, *angmin = nullptr, *angmax = nullptr, *rate = nullptr;
    bf16 *U = nullptr, *H1 = nullptr, *H2 = nullptr, *dYh = nullptr, *dZ2h = nullptr, *dZ1h = nullptr;
    // transposed BF16 copies (the backward GEMMs take K-contiguous operands)
    bf16 *UT = nullptr, *H1T = nullptr, *H2T = nullptr, *W2T = nullptr, *W3T = nullptr, *dYT = nullptr,
         *dZ2T = nullptr, *dZ1T = nullptr;
    // TMA tensor maps of every GEMM operand (buffers fixed for the model's life)
    GMap mU, mW1, mH1, mW2, mH2, mW3, mdYT, mH2T, mdY, mW3T, mdZ2T, mH1T, mdZ2, mW2T, mdZ1T, mUT;
    float *Z1 = nullptr, *Z2 = nullptr, *Y = nullptr, *dYf = nullptr, *dZ2f = nullptr, *dZ1f = nullptr;
    double *x = nullptr, *c = nullptr, *gradf = nullptr, *obj = nullptr, *v1 = nullptr, *u2 = nullptr,
           *part = nullptr;
    int nparts = 0;
};

namespace {

template <class T>
int walloc(opf_warm *w, T **p, size_t count)
{
    void *q = nullptr;
    if (cudaMalloc(&q, sizeof(T) * (count ? count : 1)) != cudaSuccess) {
        cudaGetLastError();
        set_error("opf_warm: cudaMalloc of %zu bytes failed", sizeof(T) * count);
        return OPF_ENOMEM;
    }
    w->allocs.push_back(q);
    *p = static_cast<T *>(q);
    return OPF_OK;
}

template <class T>
int wupload(opf_warm *w, T **p, const std::vector<T> &v)
{
    int rc = walloc(w, p, v.size());
    if (!rc && !v.empty() && cudaMemcpy(*p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        set_error("opf_warm: cudaMemcpy failed");
        return OPF_ECUDA;
    }
    return rc;
}

void destroy(opf_warm *w)
{
    if (!w)
        return;
    for (void *p : w->allocs)
        cudaFree(p);
    if (w->M)
        free_model(w->M);
    delete w;
}

WarmDev dev_of(const opf_warm *w)
{
    WarmDev d;
    d.B = w->B;
    d.nb = w->nb;
    d.ng = w->ng;
    d.nl = w->nl;
    d.nload = w->nload;
    d.Kin = w->Kin;
    d.Nout = w->Nout;
    d.nbp = w->nbp;
    d.ngp = w->ngp;
    d.ref = w->ref;
    d.va_scale = w->va_scale;
    d.penalty = w->penalty;
    d.pk = w->pk;
    d.qk = w->qk;
    d.vmin = w->vmin;
    d.vmax = w->vmax;
    d.pmin = w->pmin;
    d.pmax = w->pmax;
    d.qmin = w->qmin;
    d.qmax = w->qmax;
    d.angmin = w->angmin;
    d.angmax = w->angmax;
    d.rate = w->rate;
    d.vmid = w->vmid;
    d.pmid = w->pmid;
    d.phalf = w->phalf;
    d.qmid = w->qmid;
    d.qhalf = w->qhalf;
    d.inv_b = 1.0 / w->B;
    return d;
}

int check_cuda(cudaError_t e, const char *what)
{
    if (e != cudaSuccess) {
        set_error("opf_warm: %s: %s", what, cudaGetErrorString(e));
        return OPF_ECUDA;
    }
    return OPF_OK;
}

int refresh_bf16(opf_warm *w, cudaStream_t s)
{
    to_bf16_kernel<<<grid1((int64_t)w->H * w->Kin), 256, 0, s>>>(w->params + w->oW1, w->W1h, (int64_t)w->H * w->Kin);
    to_bf16_kernel<<<grid1((int64_t)w->H * w->H), 256, 0, s>>>(w->params + w->oW2, w->W2h, (int64_t)w->H * w->H);
    to_bf16_kernel<<<grid1((int64_t)w->Nout * w->H), 256, 0, s>>>(w->params + w->oW3, w->W3h, (int64_t)w->Nout * w->H);
    cudaError_t e = transpose(w->W2h, w->H, w->H, w->W2T, s);
    if (e == cudaSuccess)
        e = transpose(w->W3h, w->Nout, w->H, w->W3T, s);
    return check_cuda(e == cudaSuccess ? cudaGetLastError() : e, "bf16 copies");
}

// a GEMM wait that gave up since the last check (the flag is cleared)
int check_timeout()
{
    int v = 0, zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_umma_timeout, sizeof(int));
    if (e == cudaSuccess && v)
        e = cudaMemcpyToSymbol(g_umma_timeout, &zero, sizeof(int));
    if (e != cudaSuccess)
        return check_cuda(e, "GEMM status");
    if (v) {
        set_error("opf_warm: a tensor-core GEMM wait timed out; results are invalid");
        return OPF_ECUDA;
    }
    return OPF_OK;
}

GemmArgs gargs(int M, int N, int K, int ldc, int epi, const float *bias, const float *zsaved, float *outf,
               bf16 *outh)
{
    GemmArgs g;
    g.M = M; g.N = N; g.K = K; g.ldc = ldc; g.epi = epi;
    g.bias = bias; g.zsaved = zsaved; g.outf = outf; g.outh = outh;
    return g;
}

// forward pass: U (already prepared) -> Z1, H1, Z2, H2, and Y into y
// (w->Y unless given)
int forward(opf_warm *w, cudaStream_t s, float *y = nullptr)
{
    const int B = w->B, H = w->H;
    cudaError_t e =
        gemm(w->mU, w->mW1, gargs(B, H, w->Kin, H, EPI_BIAS_GELU, w->params + w->ob1, nullptr, w->Z1, w->H1), s);
    if (e == cudaSuccess)
        e = gemm(w->mH1, w->mW2, gargs(B, H, H, H, EPI_BIAS_GELU, w->params + w->ob2, nullptr, w->Z2, w->H2), s);
    if (e == cudaSuccess)
        e = gemm(w->mH2, w->mW3, gargs(B, w->Nout, H, w->Nout, EPI_BIAS, w->params + w->ob3, nullptr, y ? y : w->Y, nullptr), s);
    return check_cuda(e, "forward GEMMs");
}

// backward pass of dY (dYf, dYh set) into grads, after a forward pass of
// the same batch (U, H1, H2 are read through transposed copies)
int backward(opf_warm *w, cudaStream_t s)
{
    const int B = w->B, H = w->H;
    float *gr = w->grads;
    cudaError_t e = transpose(w->U, B, w->Kin, w->UT, s);
    if (e == cudaSuccess)
        e = transpose(w->H1, B, H, w->H1T, s);
    if (e == cudaSuccess)
        e = transpose(w->H2, B, H, w->H2T, s);
    // dW3 = dY^T H2 [Nout][H], db3 = colsum dY
    if (e == cudaSuccess)
        e = transpose(w->dYh, B, w->Nout, w->dYT, s);
    if (e == cudaSuccess)
        e = gemm(w->mdYT, w->mH2T, gargs(w->Nout, H, B, H, EPI_STORE, nullptr, nullptr, gr + w->oW3, nullptr), s);
    colsum_kernel<<<(w->Nout + 31) / 32, dim3(32, 32), 0, s>>>(w->dYf, B, w->Nout, gr + w->ob3);
    // dZ2 = (dY W3) * gelu'(Z2)
    if (e == cudaSuccess)
        e = gemm(w->mdY, w->mW3T, gargs(B, H, w->Nout, H, EPI_DGELU, nullptr, w->Z2, w->dZ2f, w->dZ2h), s);
    // dW2 = dZ2^T H1, db2
    if (e == cudaSuccess)
        e = transpose(w->dZ2h, B, H, w->dZ2T, s);
    if (e == cudaSuccess)
        e = gemm(w->mdZ2T, w->mH1T, gargs(H, H, B, H, EPI_STORE, nullptr, nullptr, gr + w->oW2, nullptr), s);
    colsum_kernel<<<(H + 31) / 32, dim3(32, 32), 0, s>>>(w->dZ2f, B, H, gr + w->ob2);
    // dZ1 = (dZ2 W2) * gelu'(Z1)
    if (e == cudaSuccess)
        e = gemm(w->mdZ2, w->mW2T, gargs(B, H, H, H, EPI_DGELU, nullptr, w->Z1, w->dZ1f, w->dZ1h), s);
    // dW1 = dZ1^T U, db1
    if (e == cudaSuccess)
        e = transpose(w->dZ1h, B, H, w->dZ1T, s);
    if (e == cudaSuccess)
        e = gemm(w->mdZ1T, w->mUT, gargs(H, w->Kin, B, w->Kin, EPI_STORE, nullptr, nullptr, gr + w->oW1, nullptr), s);
    colsum_kernel<<<(H + 31) / 32, dim3(32, 32), 0, s>>>(w->dZ1f, B, H, gr + w->ob1);
    if (e == cudaSuccess)
        e = cudaGetLastError();
    return check_cuda(e, "backward GEMMs");
}

// The loss of the batch at the network output w->Y and its gradient dL/dY
// (into dYf, dYh): the point from the output map, flows from the voltages,
// the library's callbacks, the penalty gradient through one J^T product of
// the reduced multipliers (flowmult_kernel).
int loss_grad(opf_warm *w, const double *d_pd, const double *d_qd, double *d_stats, cudaStream_t s)
{
    const WarmDev d = dev_of(w);
    map_kernel<<<w->B < w->nparts ? w->B : w->nparts, 256, 0, s>>>(d, w->Y, w->x);
    int rc = launch_set_loads(*w->M, d_pd, d_qd, s);
    if (!rc)  // p, q := flows at the voltages; objective, gradient, constraints there
        rc = launch_cons_setflows(*w->M, w->x, w->obj, w->gradf, w->c, s);
    if (!rc) {  // v1 = 2 penalty rho / B; residual sums; flow rows of v1 := v2
        resid_kernel<<<w->nparts, 256, 0, s>>>(d, w->c, w->m, w->v1, w->part);
        bound_kernel<<<w->nparts, 256, 0, s>>>(d, w->x, w->part + w->nparts);
        if (d_stats)
            stats_kernel<<<1, 32, 0, s>>>(d, w->part, 2 * w->nparts, w->obj, d_stats);
        flowmult_kernel<<<w->B < w->nparts ? w->B : w->nparts, 256, 0, s>>>(d, w->M->d.br, w->x, w->v1);
        rc = launch_jtprod(*w->M, w->x, w->v1, w->u2, s);
    }
    if (!rc)
        dmap_kernel<<<w->B < w->nparts ? w->B : w->nparts, 256, 0, s>>>(d, w->x, w->u2, w->gradf, w->dYf, w->dYh);
    if (!rc)
        rc = check_cuda(cudaGetLastError(), "loss gradient");
    return rc;
}

int round_up(int v, int q)
{
    return (v + q - 1) / q * q;
}

}  // namespace

extern "C" {

int opf_warm_create(const opf_network *net, const opf_warm_opts *opts, opf_warm **out)
{
    if (!out) {
        set_error("out is NULL");
        return OPF_EINVAL;
    }
    *out = nullptr;
    if (!net || !opts) {
        set_error("opf_warm_create: net and opts are required");
        return OPF_EINVAL;
    }
    if (net->nperiod != 1 || opts->batch < 128 || opts->batch % 128 || opts->hidden < 128 ||
        opts->hidden % 128 || !(opts->penalty >= 0.0) || !(opts->lr > 0.0) || !(opts->lr_out > 0.0) ||
        !std::isfinite(opts->va_scale)) {
        set_error("opf_warm_create: need nperiod 1, batch and hidden multiples of 128, penalty >= 0, "
                  "lr > 0, lr_out > 0, finite va_scale");
        return OPF_EINVAL;
    }
    opf_warm *w = new opf_warm();
    w->B = opts->batch;
    w->H = opts->hidden;
    w->nb = net->nbus;
    w->ng = net->ngen;
    w->nl = net->nbranch;
    w->nload = net->nload;
    w->ref = net->ref_bus;
    w->penalty = opts->penalty;
    w->lr = opts->lr;
    w->lr_out = opts->lr_out;
    w->va_scale = opts->va_scale;
    w->Kin = round_up(2 * w->nload, 128);
    w->nbp = round_up(w->nb, 128);
    w->ngp = round_up(w->ng, 128);
    w->Nout = 2 * w->nbp + 2 * w->ngp;
    // the callback model: batch periods, no ramp rows, loads replaced per call
    opf_network n2 = *net;
    n2.nperiod = w->B;
    n2.ramp_ratio = 0.0;
    std::vector<double> lp((size_t)w->B * w->nload), lq((size_t)w->B * w->nload);
    for (int t = 0; t < w->B; t++)
        for (int l = 0; l < w->nload; l++) {
            lp[(size_t)t * w->nload + l] = net->load_pd[l];
            lq[(size_t)t * w->nload + l] = net->load_qd[l];
        }
    n2.load_pd = lp.data();
    n2.load_qd = lq.data();
    int rc = build_model(&n2, 1, nullptr, true, &w->M);
    if (rc) {
        delete w;
        return rc;
    }
    w->n = w->M->n;
    w->m = w->M->m;
    if (w->n >= (int64_t)1 << 31 || w->m >= (int64_t)1 << 31) {
        set_error("opf_warm_create: batch x network too large (%lld variables, %lld rows; the warm start's "
                  "kernels index them in 32 bits)", (long long)w->n, (long long)w->m);
        destroy(w);
        return OPF_EINVAL;
    }
    w->n1 = w->n / w->B;
    // parameters: W1 [H][Kin], b1 [H], W2 [H][H], b2 [H], W3 [Nout][H], b3 [Nout]
    w->oW1 = 0;
    w->ob1 = w->oW1 + (int64_t)w->H * w->Kin;
    w->oW2 = w->ob1 + w->H;
    w->ob2 = w->oW2 + (int64_t)w->H * w->H;
    w->oW3 = w->ob2 + w->H;
    w->ob3 = w->oW3 + (int64_t)w->Nout * w->H;
    w->nparams = w->ob3 + w->Nout;
    std::vector<float> p(w->nparams, 0.f);
    std::mt19937_64 rng(opts->seed);
    auto init_rows = [&](int64_t off, int cols, int r0, int r1, int used_cols) {
        std::normal_distribution<double> nd(0.0, 1.0 / std::sqrt((double)used_cols));
        for (int r = r0; r < r1; r++)
            for (int c = 0; c < used_cols; c++)
                p[off + (int64_t)r * cols + c] = (float)nd(rng);
    };
    init_rows(w->oW1, w->Kin, 0, w->H, 2 * w->nload);
    init_rows(w->oW2, w->H, 0, w->H, w->H);
    // W3 and b3 start at zero: the untrained network proposes the flat start
    std::vector<float> pk(w->nload), qk(w->nload);
    for (int l = 0; l < w->nload; l++) {
        pk[l] = net->load_pd[l] > 0.0 ? (float)(5.0 / net->load_pd[l]) : 0.f;
        qk[l] = net->load_qd[l] > 0.0 ? (float)(5.0 / net->load_qd[l]) : 0.f;
    }
    std::vector<double> vmin(net->bus_vmin, net->bus_vmin + w->nb), vmax(net->bus_vmax, net->bus_vmax + w->nb);
    std::vector<double> pmin(net->gen_pmin, net->gen_pmin + w->ng), pmax(net->gen_pmax, net->gen_pmax + w->ng);
    std::vector<double> qmin(net->gen_qmin, net->gen_qmin + w->ng), qmax(net->gen_qmax, net->gen_qmax + w->ng);
    std::vector<double> xl(w->n), xu(w->n), gl(w->m), gu(w->m);
    bounds(*w->M, xl.data(), xu.data(), gl.data(), gu.data());
    w->nparts = 148 * 8;
    const int64_t act = (int64_t)w->B * w->H;
    const int64_t outsz = (int64_t)w->B * w->Nout;
    if (!rc) rc = wupload(w, &w->params, p);
    if (!rc) rc = walloc(w, &w->grads, w->nparams);
    if (!rc) rc = walloc(w, &w->am, w->nparams);
    if (!rc) rc = walloc(w, &w->av, w->nparams);
    if (!rc) rc = walloc(w, &w->W1h, (size_t)w->H * w->Kin);
    if (!rc) rc = walloc(w, &w->W2h, (size_t)w->H * w->H);
    if (!rc) rc = walloc(w, &w->W3h, (size_t)w->Nout * w->H);
    if (!rc) rc = wupload(w, &w->pk, pk);
    if (!rc) rc = wupload(w, &w->qk, qk);
    if (!rc) rc = wupload(w, &w->vmin, vmin);
    if (!rc) rc = wupload(w, &w->vmax, vmax);
    if (!rc) rc = wupload(w, &w->pmin, pmin);
    if (!rc) rc = wupload(w, &w->pmax, pmax);
    if (!rc) rc = wupload(w, &w->qmin, qmin);
    if (!rc) rc = wupload(w, &w->qmax, qmax);
    if (!rc) rc = wupload(w, &w->angmin, std::vector<double>(net->br_angmin, net->br_angmin + w->nl));
    if (!rc) rc = wupload(w, &w->angmax, std::vector<double>(net->br_angmax, net->br_angmax + w->nl));
    if (!rc) rc = wupload(w, &w->rate, std::vector<double>(net->br_rate_a, net->br_rate_a + w->nl));
    {
        std::vector<double> vmid(w->nb), pmid(w->ng), phalf(w->ng), qmid(w->ng), qhalf(w->ng);
        for (int i = 0; i < w->nb; i++)
            vmid[i] = 0.5 * (vmin[i] + vmax[i]);
        for (int g = 0; g < w->ng; g++) {
            pmid[g] = 0.5 * (pmin[g] + pmax[g]);
            phalf[g] = 0.5 * (pmax[g] - pmin[g]);
            qmid[g] = 0.5 * (qmin[g] + qmax[g]);
            qhalf[g] = 0.5 * (qmax[g] - qmin[g]);
        }
        if (!rc) rc = wupload(w, &w->vmid, vmid);
        if (!rc) rc = wupload(w, &w->pmid, pmid);
        if (!rc) rc = wupload(w, &w->phalf, phalf);
        if (!rc) rc = wupload(w, &w->qmid, qmid);
        if (!rc) rc = wupload(w, &w->qhalf, qhalf);
    }
    if (!rc) rc = walloc(w, &w->U, (size_t)w->B * w->Kin);
    if (!rc) rc = walloc(w, &w->H1, act);
    if (!rc) rc = walloc(w, &w->H2, act);
    if (!rc) rc = walloc(w, &w->dZ2h, act);
    if (!rc) rc = walloc(w, &w->dZ1h, act);
    if (!rc) rc = walloc(w, &w->Z1, act);
    if (!rc) rc = walloc(w, &w->Z2, act);
    if (!rc) rc = walloc(w, &w->dZ2f, act);
    if (!rc) rc = walloc(w, &w->dZ1f, act);
    if (!rc) rc = walloc(w, &w->UT, (size_t)w->Kin * w->B);
    if (!rc) rc = walloc(w, &w->H1T, act);
    if (!rc) rc = walloc(w, &w->H2T, act);
    if (!rc) rc = walloc(w, &w->W2T, (size_t)w->H * w->H);
    if (!rc) rc = walloc(w, &w->W3T, (size_t)w->H * w->Nout);
    if (!rc) rc = walloc(w, &w->dYT, outsz);
    if (!rc) rc = walloc(w, &w->dZ2T, act);
    if (!rc) rc = walloc(w, &w->dZ1T, act);
    if (!rc) rc = walloc(w, &w->Y, outsz);
    if (!rc) rc = walloc(w, &w->dYf, outsz);
    if (!rc) rc = walloc(w, &w->dYh, outsz);
    if (!rc) rc = walloc(w, &w->x, w->n);
    if (!rc) rc = walloc(w, &w->c, w->m);
    if (!rc) rc = walloc(w, &w->gradf, w->n);
    if (!rc) rc = walloc(w, &w->obj, 1);
    if (!rc) rc = walloc(w, &w->v1, w->m);
    if (!rc) rc = walloc(w, &w->u2, w->n);
    if (!rc) rc = walloc(w, &w->part, 2 * (size_t)w->nparts);
    if (!rc) {  // tensor maps: A operands [M][K], B operands [N][K]
        const int B = w->B, H = w->H, Kin = w->Kin, No = w->Nout;
        const bool ok = map_a(&w->mU, w->U, B, Kin) && map_b(&w->mW1, w->W1h, H, Kin) &&
                        map_a(&w->mH1, w->H1, B, H) && map_b(&w->mW2, w->W2h, H, H) &&
                        map_a(&w->mH2, w->H2, B, H) && map_b(&w->mW3, w->W3h, No, H) &&
                        map_a(&w->mdYT, w->dYT, No, B) && map_b(&w->mH2T, w->H2T, H, B) &&
                        map_a(&w->mdY, w->dYh, B, No) && map_b(&w->mW3T, w->W3T, H, No) &&
                        map_a(&w->mdZ2T, w->dZ2T, H, B) && map_b(&w->mH1T, w->H1T, H, B) &&
                        map_a(&w->mdZ2, w->dZ2h, B, H) && map_b(&w->mW2T, w->W2T, H, H) &&
                        map_a(&w->mdZ1T, w->dZ1T, H, B) && map_b(&w->mUT, w->UT, Kin, B);
        if (!ok) {
            set_error("opf_warm_create: cuTensorMapEncodeTiled failed");
            rc = OPF_ECUDA;
        }
    }
    if (!rc)
        rc = check_cuda(cudaFuncSetAttribute(umma_gemm_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             GemmCfg<256>::SMEM),
                        "GEMM shared memory");
    if (!rc)
        rc = check_cuda(cudaFuncSetAttribute(umma_gemm_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             GemmCfg<128>::SMEM),
                        "GEMM shared memory");
    if (!rc) {  // the structured bounds of the kernels against the model's own
        double *b = nullptr;
        unsigned *bad = nullptr, nbad = 0;
        const size_t bytes = sizeof(double) * 2 * (size_t)(w->n + w->m);
        if (cudaMalloc(&b, bytes) != cudaSuccess || cudaMalloc(&bad, sizeof(unsigned)) != cudaSuccess) {
            cudaGetLastError();
            set_error("opf_warm_create: cudaMalloc of %zu bytes failed", bytes);
            rc = OPF_ENOMEM;
        } else {
            double *bxl = b, *bxu = b + w->n, *bgl = b + 2 * w->n, *bgu = b + 2 * w->n + w->m;
            cudaMemcpy(bxl, xl.data(), sizeof(double) * w->n, cudaMemcpyHostToDevice);
            cudaMemcpy(bxu, xu.data(), sizeof(double) * w->n, cudaMemcpyHostToDevice);
            cudaMemcpy(bgl, gl.data(), sizeof(double) * w->m, cudaMemcpyHostToDevice);
            cudaMemcpy(bgu, gu.data(), sizeof(double) * w->m, cudaMemcpyHostToDevice);
            cudaMemset(bad, 0, sizeof(unsigned));
            bounds_check_kernel<<<grid1(w->n + w->m), 256>>>(dev_of(w), bxl, bxu, w->n, bgl, bgu, w->m, bad);
            rc = check_cuda(cudaMemcpy(&nbad, bad, sizeof(unsigned), cudaMemcpyDeviceToHost), "bounds check");
            if (!rc && nbad) {
                set_error("opf_warm_create: %u structured bounds differ from the model's", nbad);
                rc = OPF_ESTATE;
            }
        }
        cudaFree(b);
        cudaFree(bad);
    }
    if (!rc && (cudaMemset(w->am, 0, sizeof(float) * w->nparams) != cudaSuccess ||
                cudaMemset(w->av, 0, sizeof(float) * w->nparams) != cudaSuccess ||
                cudaMemset(w->grads, 0, sizeof(float) * w->nparams) != cudaSuccess ||
                cudaMemset(w->Y, 0, sizeof(float) * outsz) != cudaSuccess))
        rc = check_cuda(cudaGetLastError(), "memset");
    if (!rc)
        rc = refresh_bf16(w, nullptr);
    if (!rc)
        rc = check_cuda(cudaDeviceSynchronize(), "create");
    if (rc) {
        destroy(w);
        return rc;
    }
    *out = w;
    return OPF_OK;
}

int opf_warm_destroy(opf_warm *w)
{
    destroy(w);
    return OPF_OK;
}

int opf_warm_dims(const opf_warm *w, int32_t *n_in, int32_t *n_out, int32_t *n_x, int64_t *n_params)
{
    if (!w) {
        set_error("opf_warm_dims: w is NULL");
        return OPF_EINVAL;
    }
    if (n_in) *n_in = w->Kin;
    if (n_out) *n_out = w->Nout;
    if (n_x) *n_x = (int32_t)w->n1;
    if (n_params) *n_params = w->nparams;
    return OPF_OK;
}

int opf_warm_forward(opf_warm *w, const double *d_pd, const double *d_qd, float *d_y, void *stream)
{
    if (!w || !d_pd || !d_qd) {
        set_error("opf_warm_forward: bad arguments");
        return OPF_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    prep_kernel<<<dim3((w->Kin + 1023) / 1024, w->B < 65535 ? w->B : 65535), 128, 0, s>>>(dev_of(w), d_pd, d_qd, w->U);
    // the output layer writes the caller's buffer directly where its
    // vector stores may (16-byte aligned), else w->Y and a copy
    const bool direct = d_y && (reinterpret_cast<uintptr_t>(d_y) & 15u) == 0;
    int rc = forward(w, s, direct ? d_y : nullptr);
    if (!rc && d_y && !direct)
        rc = check_cuda(cudaMemcpyAsync(d_y, w->Y, sizeof(float) * w->B * w->Nout, cudaMemcpyDeviceToDevice, s), "copy output");
    return rc;
}

int opf_warm_backward(opf_warm *w, const float *d_dy, float *d_grad, void *stream)
{
    if (!w || !d_dy) {
        set_error("opf_warm_backward: bad arguments");
        return OPF_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = check_cuda(cudaMemcpyAsync(w->dYf, d_dy, sizeof(float) * w->B * w->Nout, cudaMemcpyDeviceToDevice, s), "copy dy");
    if (!rc)
        to_bf16_kernel<<<grid1((int64_t)w->B * w->Nout), 256, 0, s>>>(w->dYf, w->dYh, (int64_t)w->B * w->Nout);
    if (!rc)
        rc = backward(w, s);
    if (!rc && d_grad)
        rc = check_cuda(cudaMemcpyAsync(d_grad, w->grads, sizeof(float) * w->nparams, cudaMemcpyDeviceToDevice, s), "copy grads");
    return rc;
}

int opf_warm_loss_grad(opf_warm *w, const double *d_pd, const double *d_qd, const float *d_y,
                       float *d_dy, double *d_stats, void *stream)
{
    if (!w || !d_pd || !d_qd || !d_y) {
        set_error("opf_warm_loss_grad: bad arguments");
        return OPF_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = check_cuda(cudaMemcpyAsync(w->Y, d_y, sizeof(float) * w->B * w->Nout, cudaMemcpyDeviceToDevice, s), "copy output");
    if (!rc)
        rc = loss_grad(w, d_pd, d_qd, d_stats, s);
    if (!rc && d_dy)
        rc = check_cuda(cudaMemcpyAsync(d_dy, w->dYf, sizeof(float) * w->B * w->Nout, cudaMemcpyDeviceToDevice, s), "copy dy");
    return rc;
}

int opf_warm_train_step(opf_warm *w, const double *d_pd, const double *d_qd, double *d_stats, void *stream)
{
    if (!w || !d_pd || !d_qd) {
        set_error("opf_warm_train_step: bad arguments");
        return OPF_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    prep_kernel<<<dim3((w->Kin + 1023) / 1024, w->B < 65535 ? w->B : 65535), 128, 0, s>>>(dev_of(w), d_pd, d_qd, w->U);
    int rc = forward(w, s);
    if (!rc)
        rc = loss_grad(w, d_pd, d_qd, d_stats, s);
    if (!rc)
        rc = backward(w, s);
    if (!rc) {
        w->step++;
        const float bc1 = 1.f - (float)std::pow(0.9, (double)w->step);
        const float bc2 = 1.f - (float)std::pow(0.999, (double)w->step);
        // weights and hidden biases at lr, the output bias at lr_out
        adam_kernel<<<grid1(w->ob3), 256, 0, s>>>(w->params, w->grads, w->am, w->av, w->ob3, (float)w->lr,
                                                  bc1, bc2);
        adam_kernel<<<grid1(w->Nout), 256, 0, s>>>(w->params + w->ob3, w->grads + w->ob3, w->am + w->ob3,
                                                   w->av + w->ob3, w->Nout, (float)w->lr_out, bc1, bc2);
        rc = refresh_bf16(w, s);
    }
    return rc;
}

int opf_warm_predict(opf_warm *w, const double *d_pd, const double *d_qd, double *d_x, void *stream)
{
    if (!w || !d_pd || !d_qd || !d_x) {
        set_error("opf_warm_predict: bad arguments");
        return OPF_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const WarmDev d = dev_of(w);
    prep_kernel<<<dim3((w->Kin + 1023) / 1024, w->B < 65535 ? w->B : 65535), 128, 0, s>>>(d, d_pd, d_qd, w->U);
    int rc = forward(w, s);
    if (!rc) {
        rc = check_cuda(cudaMemsetAsync(d_x, 0, sizeof(double) * w->n, s), "clear x");
        map_kernel<<<w->B < w->nparts ? w->B : w->nparts, 256, 0, s>>>(d, w->Y, d_x);
        if (!rc)
            rc = launch_flows(*w->M, d_x, s);
    }
    return rc;
}

int opf_warm_set_lr(opf_warm *w, double lr, double lr_out)
{
    if (!w || !(lr > 0.0) || !(lr_out > 0.0)) {
        set_error("opf_warm_set_lr: bad arguments");
        return OPF_EINVAL;
    }
    w->lr = lr;
    w->lr_out = lr_out;
    return OPF_OK;
}

int opf_warm_get_activations(const opf_warm *w, uint16_t *h_u, float *h_z1, uint16_t *h_h1, float *h_z2,
                             uint16_t *h_h2, float *h_dz2, float *h_dz1)
{
    if (!w) {
        set_error("opf_warm_get_activations: NULL handle");
        return OPF_EINVAL;
    }
    const size_t bh = (size_t)w->B * w->H, bk = (size_t)w->B * w->Kin;
    struct Part {
        void *dst;
        const void *src;
        size_t bytes;
    } parts[] = {{h_u, w->U, 2 * bk},      {h_z1, w->Z1, 4 * bh},   {h_h1, w->H1, 2 * bh}, {h_z2, w->Z2, 4 * bh},
                 {h_h2, w->H2, 2 * bh},    {h_dz2, w->dZ2f, 4 * bh}, {h_dz1, w->dZ1f, 4 * bh}};
    int rc = OPF_OK;
    for (const Part &q : parts)
        if (!rc && q.dst)
            rc = check_cuda(cudaMemcpy(q.dst, q.src, q.bytes, cudaMemcpyDeviceToHost), "get activations");
    if (!rc)
        rc = check_timeout();
    return rc;
}

int opf_warm_get_params(const opf_warm *w, float *h)
{
    if (!w || !h) {
        set_error("opf_warm_get_params: bad arguments");
        return OPF_EINVAL;
    }
    int rc = check_cuda(cudaMemcpy(h, w->params, sizeof(float) * w->nparams, cudaMemcpyDeviceToHost), "get params");
    if (!rc)
        rc = check_timeout();
    return rc;
}

int opf_warm_set_params(opf_warm *w, const float *h)
{
    if (!w || !h) {
        set_error("opf_warm_set_params: bad arguments");
        return OPF_EINVAL;
    }
    int rc = check_cuda(cudaMemcpy(w->params, h, sizeof(float) * w->nparams, cudaMemcpyHostToDevice), "set params");
    if (!rc && (cudaMemset(w->am, 0, sizeof(float) * w->nparams) != cudaSuccess ||
                cudaMemset(w->av, 0, sizeof(float) * w->nparams) != cudaSuccess))
        rc = check_cuda(cudaGetLastError(), "clear adam");
    w->step = 0;
    if (!rc)
        rc = refresh_bf16(w, nullptr);
    if (!rc)
        rc = check_cuda(cudaDeviceSynchronize(), "set params");
    return rc;
}

}  // extern "C"

// Peak-rate probes: the measured denominators of the roofline fractions.
//
// Each probe is one kernel that performs a known number of operations of one kind with
// enough independent chains per thread and enough warps per SM that only the throughput of
// that unit limits it:
//   * FFMA: 8 independent fmaf chains per thread, 64 warps per SM (FP32 pipe; 2 flops each);
//   * EX2, RSQRT: 8 independent ex2.approx / rsqrt.approx chains (MUFU; 1 op per lane);
//   * DFMA: 8 independent FP64 fma chains (2 flops each);
//   * MMA_TF32, MMA_BF16: one CTA per SM, one thread issuing back-to-back tcgen05.mma with
//     M = 128, N = 256 and one 32-byte K slice (K = 8 TF32 / 16 BF16) from shared memory into a
//     TMEM accumulator (2 M N K flops each), completion tracked by tcgen05.commit on an mbarrier.
// The caller times the launch with CUDA events on its stream.  Results feed a conditional
// store that never fires, so the arithmetic is not removed; shared-memory operands are zero.
// The one wait (the MMA completion) is bounded: on give-up the kernel sets ERRBIT_TIMEOUT,
// waits once more (bounded) for the MMAs it issued, frees TMEM and returns.
#include "common.cuh"
#include "vfmm_internal.h"

namespace vfmm {
namespace {

__device__ float g_probe_sink[8];

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_UNROLL = 16;
constexpr long long PROBE_WAIT_LIMIT = 1LL << 28;

__device__ __forceinline__ float mufu_ex2(float x)
{
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float mufu_rsqrt(float x)
{
    float y;
    asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int KIND> __global__ void __launch_bounds__(PROBE_THREADS) k_probe_alu(long long reps, float seed)
{
    float a[PROBE_CHAINS];
    const float b = 0.9999f + 1e-9f * seed, c = 1e-4f * seed;
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) a[i] = seed + 1e-3f * (float)(threadIdx.x + i);
    for (long long r = 0; r < reps; ++r) {
#pragma unroll
        for (int k = 0; k < PROBE_UNROLL; ++k)
#pragma unroll
            for (int i = 0; i < PROBE_CHAINS; ++i) {
                if (KIND == VFMM_PROBE_FFMA) a[i] = fmaf(a[i], b, c);
                else if (KIND == VFMM_PROBE_EX2) a[i] = mufu_ex2(-a[i]);   // stays in (0, 1]
                else a[i] = mufu_rsqrt(a[i]);                             // tends to 1
            }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) s += a[i];
    if (s == 1.2345e-30f) g_probe_sink[threadIdx.x & 7] = s;
}

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_dfma(long long reps, double seed)
{
    double a[PROBE_CHAINS];
    const double b = 0.9999 + 1e-12 * seed, c = 1e-4 * seed;
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) a[i] = seed + 1e-3 * (double)(threadIdx.x + i);
    for (long long r = 0; r < reps; ++r) {
#pragma unroll
        for (int k = 0; k < PROBE_UNROLL; ++k)
#pragma unroll
            for (int i = 0; i < PROBE_CHAINS; ++i) a[i] = fma(a[i], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) s += a[i];
    if (s == 1.2345e-300) g_probe_sink[threadIdx.x & 7] = (float)s;
}

// ---- tcgen05 MMA probe -------------------------------------------------------------------
constexpr int PM = 128, PN = 256;
constexpr int PA_BYTES = PM * 32, PB_BYTES = PN * 32;  // one 32-byte K slice per row
constexpr int P_TMEM_COLS = 256;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: canonical K-major layout without swizzle, 8-row x 16-byte
// core matrices, lbo = bytes to the next core matrix along K, sbo = bytes to the next 8 rows
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ bool probe_wait(uint32_t bar, uint32_t parity)
{
    for (long long it = 0; it < PROBE_WAIT_LIMIT; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

template <bool BF16> __global__ void __launch_bounds__(128, 1) k_probe_mma(long long reps, int *err)
{
    __shared__ __align__(1024) unsigned char tiles[PA_BYTES + PB_BYTES];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int i = tid; i < (PA_BYTES + PB_BYTES) / 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(tiles)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                     "r"(P_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;
    bool ok = true;
    if (tid == 0) {
        const uint32_t fmt = BF16 ? 1u : 2u;
        const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(PN >> 3) << 17) |
                               ((uint32_t)(PM >> 4) << 24);
        const uint64_t da = smem_desc(smem_addr(tiles), 128, 256);
        const uint64_t db = smem_desc(smem_addr(tiles + PA_BYTES), 128, 256);
        for (long long r = 0; r < reps; ++r) {
            const uint32_t acc = r > 0 ? 1u : 0u;
            if (BF16)
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(acc));
            else
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(acc));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_addr(&bar))
                     : "memory");
        ok = probe_wait(smem_addr(&bar), 0u);
        if (!ok) {
            atomicOr(err, ERRBIT_TIMEOUT);
            probe_wait(smem_addr(&bar), 0u);  // the issued MMAs still write TMEM: wait once more
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(P_TMEM_COLS));
    }
}

}  // namespace
}  // namespace vfmm

using namespace vfmm;

extern "C" int vfmm_probe_peak(int kind, int64_t reps, void *stream, int *err_dev, double *ops)
{
    if (reps <= 0 || !ops) return VFMM_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        return VFMM_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const int alu_blocks = sms * (2048 / PROBE_THREADS);
    const double lanes = (double)alu_blocks * PROBE_THREADS * PROBE_CHAINS * PROBE_UNROLL * (double)reps;
    switch (kind) {
    case VFMM_PROBE_FFMA:
        k_probe_alu<VFMM_PROBE_FFMA><<<alu_blocks, PROBE_THREADS, 0, st>>>(reps, 0.5f);
        *ops = 2.0 * lanes;
        break;
    case VFMM_PROBE_EX2:
        k_probe_alu<VFMM_PROBE_EX2><<<alu_blocks, PROBE_THREADS, 0, st>>>(reps, 0.5f);
        *ops = lanes;
        break;
    case VFMM_PROBE_RSQRT:
        k_probe_alu<VFMM_PROBE_RSQRT><<<alu_blocks, PROBE_THREADS, 0, st>>>(reps, 0.5f);
        *ops = lanes;
        break;
    case VFMM_PROBE_DFMA:
        k_probe_dfma<<<alu_blocks, PROBE_THREADS, 0, st>>>(reps, 0.5);
        *ops = 2.0 * lanes;
        break;
    case VFMM_PROBE_MMA_TF32:
    case VFMM_PROBE_MMA_BF16: {
        if (!err_dev) return VFMM_ERR_ARG;
        const int kdim = kind == VFMM_PROBE_MMA_BF16 ? 16 : 8;
        if (kind == VFMM_PROBE_MMA_BF16)
            k_probe_mma<true><<<sms, 128, 0, st>>>(reps, err_dev);
        else
            k_probe_mma<false><<<sms, 128, 0, st>>>(reps, err_dev);
        *ops = 2.0 * PM * PN * kdim * (double)reps * sms;
        break;
    }
    default:
        return VFMM_ERR_ARG;
    }
    return cudaGetLastError() == cudaSuccess ? VFMM_OK : VFMM_ERR_CUDA;
}

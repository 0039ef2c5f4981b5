// M2L on the fifth-generation tensor cores (tcgen05, TMEM accumulators).
//
// For target cells c of one parity g at level l and each offset t of their interaction list
// (children of the parent's neighbours outside the near field; Section 3.1 uses M2L between
// well-separated cells), L_c += T_t M_{(c + t) mod 2^l}: every cell pair that shares a lattice
// offset shares the translation matrix, so the whole list is one implicit GEMM
//   D[128 out coefs][64 cells x 3 components] = sum_t sum_j A_t[k][j] B_t[n][j]
// with A_t the (pre-tiled) translation matrix and B_t the gathered multipole rows.
//
// Precision: inputs are split x = hi + lo (hi, lo both BF16, or both TF32) and three products
// hi*hi + hi*lo + lo*hi are accumulated in FP32 in TMEM; the dropped lo*lo term is ~2^-16
// (BF16) or ~2^-22 (TF32) relative.
//
// Two kernels share the operators and the pipeline mechanics:
//   * k_m2l_lines (levels with 16 to 64 cells per side and parity, i.e. the large levels):
//     128 target cells (whole z-lines) per CTA, offsets grouped by source line, one staged
//     source line serving all z shifts of its class, every operand moved by TMA (see the
//     section below);
//   * k_m2l_tc (levels 3 and 4): 64 target cells per CTA, the B tile of every offset gathered
//     row by row, the offset list split over several CTAs when the level has few cells.
//
// Mechanics (sm_103a): one elected thread of warp 0 issues tcgen05.mma (M = 128, N = 192,
// K = 16 bf16 / 8 tf32 per instruction) from shared-memory descriptors in the canonical
// no-swizzle K-major layout (8-row x 16-byte core matrices); the pre-tiled translation
// matrices arrive by TMA bulk copies (expect_tx on a per-stage transaction barrier), the
// source rows by TMA tensor copies (k_m2l_lines) or cp.async gathers of producer warps
// (k_m2l_tc); tcgen05.commit arrives on one mbarrier per stage so a stage is refilled only
// after the MMAs that read it completed.
// Every pipeline wait is bounded (TcParams.wait_limit tries).  A thread that gives up sets a
// shared abort word, which every other pipeline wait polls, so the whole CTA stops issuing;
// producer warps decide with one lane and leave their loop together.  Before TMEM is freed
// the CTA drains its own asynchronous work: producer threads wait for their cp.async copies;
// the thread that issued TMA copies waits for the phases of the stages it filled (they
// complete once the bytes land; in k_m2l_tc every producer warp first arrives on the stages it
// had not released); the MMA thread commits once more and waits for that commit (every MMA
// it issued has then completed).  The kernel then sets the timeout bit of the error word and
// returns.
#include "common.cuh"
#include "vfmm_internal.h"

#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

namespace vfmm {

constexpr int TC_THREADS = 128;
constexpr int TC_CELLS = 64;
constexpr int TC_N = 3 * TC_CELLS;          // 192 columns
constexpr int TC_M = 128;
constexpr int TC_STAGES = 5;                 // 5 x 20 KB: two CTAs (and two 256-column TMEM blocks) per SM
constexpr int TC_A_BYTES = TC_M * TC_KBYTES;     // 4 KB
constexpr int TC_B_BYTES = TC_N * TC_KBYTES;     // 6 KB
constexpr int TC_STAGE_BYTES = 2 * TC_A_BYTES + 2 * TC_B_BYTES;  // 20 KB
constexpr int TC_SBO = TC_KG * 128;              // bytes between 8-row groups
constexpr int TC_BCHUNKS = TC_N * TC_KG / 128;   // 16-byte B chunks per producer thread per stage
constexpr int TC_MAXKB = 256;                                    // k-blocks per parity (<= 189 used)
constexpr int TC_SMEM = TC_STAGES * TC_STAGE_BYTES + 1024 + 256 + TC_MAXKB * 16 + TC_CELLS * 4;
constexpr int TC_TMEM_COLS = 256;
constexpr long long TC_WAIT_LIMIT = 1LL << 26;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ float to_tf32_dev(float v)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return __uint_as_float(r);
}

__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t layout = 0)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    // base offset 0, relative LBO; layout type (bits 61-63): 0 = no swizzle
    d |= (uint64_t)(layout & 7u) << 61;
    return d;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Pipeline wait: gives up after `limit` tries, or as soon as another thread of the CTA has given
// up (the shared abort word); a thread that gives up itself sets the abort word.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit, volatile int *abort)
{
    for (long long it = 0; it < limit; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 63) == 63 && *abort) return false;  // the abort word is polled every 64 tries
    }
    *abort = 1;
    return false;
}

// Drain wait for the CTA's own asynchronous work (bulk copies, MMAs), which completes by itself:
// not cut short by the abort word, bounded by the fixed limit.
__device__ __forceinline__ bool mbar_wait_drain(uint32_t bar, uint32_t parity)
{
    for (long long it = 0; it < TC_WAIT_LIMIT; ++it)
        if (mbar_try(bar, parity)) return true;
    return false;
}

// Warp-uniform pipeline wait: every lane waits, and the warp goes on only if every lane's wait
// succeeded (so a warp leaves a loop together and no lane is left at a __syncwarp).
__device__ __forceinline__ bool mbar_wait_warp(uint32_t bar, uint32_t parity, long long limit, volatile int *abort)
{
    const bool ok = mbar_wait(bar, parity, limit, abort);
    return __all_sync(0xffffffffu, ok) != 0;
}


__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
static_assert(TC_KG % 2 == 0, "an MMA consumes two 16-byte k-groups");

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// one-dimensional TMA bulk copy global -> shared (16-byte aligned, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

template <bool BF16>
__device__ __forceinline__ void mma_issue(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    if (BF16) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
    }
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Warp-specialised pipeline: warp 0 lane 0 issues the MMAs; warps 1..4 (128 producer threads)
// gather the multipole rows with cp.async and release a stage (fence.proxy.async by every
// lane, one arrive per warp on full[s]) TC_PF stages after issuing it; producer thread 0 also
// moves the two pre-tiled translation-matrix tiles with TMA bulk copies (expect_tx on full[s],
// so a stage is full once its four warps arrived and its bytes landed).  tcgen05.commit on
// empty[s] returns the slot to the producers.  No CTA-wide barrier inside the main loop.
// Producer release lag.  A stage is released after the producer has issued TC_PF later stages,
// and issuing stage i waits for the MMAs of stage i - TC_STAGES; TC_STAGES - TC_PF >= 3 keeps an
// MMA queued behind the running one (a lag of 4 of 5 stages serialised the MMAs).
constexpr int TC_PF = 2;
constexpr int TC_WS_THREADS = 32 + TC_THREADS;  // MMA warp + 4 producer warps

template <bool BF16>
__global__ void __launch_bounds__(TC_WS_THREADS, 2) k_m2l_tc(TcParams tp)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *stages = base;
    uint64_t *full = (uint64_t *)(base + TC_STAGES * TC_STAGE_BYTES);
    uint64_t *empty = full + TC_STAGES;
    uint64_t *drain = empty + TC_STAGES;  // final tcgen05.commit
    uint32_t *tmem_slot = (uint32_t *)(drain + 1);
    volatile int *abort = (volatile int *)(tmem_slot + 1);
    volatile int *issued_sh = abort + 1;  // stages producer thread 0 filled with bulk copies
    int4 *kb_s = (int4 *)(base + TC_STAGES * TC_STAGE_BYTES + 256);
    int *cell_s = (int *)(kb_s + TC_MAXKB);

    const int tid = threadIdx.x, warp = tid >> 5;
    const int g = blockIdx.y;
    const int n = tp.n, half = n >> 1;
    const int64_t cell0 = (int64_t)blockIdx.x * TC_CELLS;
    // k-block slice of this CTA (small levels split the offsets over blockIdx.z)
    const int nkb_all = min(tp.kb_cnt[g], TC_MAXKB);
    const int per = (nkb_all + tp.ksplit - 1) / tp.ksplit;
    const int kb0 = min(nkb_all, (int)blockIdx.z * per);
    const int nkb = min(nkb_all, kb0 + per) - kb0;
    for (int q = tid; q < nkb; q += TC_WS_THREADS) kb_s[q] = tp.kb[tp.kb_off[g] + kb0 + q];
    for (int q = tid; q < TC_CELLS; q += TC_WS_THREADS) {
        int64_t P = cell0 + q;
        int px = (int)(P / ((int64_t)half * half)), py = (int)((P / half) % half), pz = (int)(P % half);
        int cx = 2 * px + ((g >> 2) & 1), cy = 2 * py + ((g >> 1) & 1), cz = 2 * pz + (g & 1);
        cell_s[q] = (cx * n + cy) * n + cz;
    }
    const int nchunk = tp.nchunk;
    const int nk = nkb * nchunk;
    const int pc = tp.pc;
    const int esz = BF16 ? 2 : 4;

    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(smem_u32(&full[s]), TC_THREADS / 32 + 1);  // one arrival per producer warp + expect_tx
            mbar_init(smem_u32(&empty[s]), 1);                  // tcgen05.commit
        }
        mbar_init(smem_u32(drain), 1);
        *abort = 0;
        *issued_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;
    bool ok = true;

    if (warp == 0) {
        // ------------------------------- MMA issuer -------------------------------
        if (tid == 0) {
            const uint32_t fmt = BF16 ? 1u : 2u;
            const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                                   ((uint32_t)(TC_M >> 4) << 24);
            for (int i = 0; i < nk; ++i) {
                const int s = i % TC_STAGES;
                const uint32_t ph = (uint32_t)((i / TC_STAGES) & 1);
                if (!mbar_wait(smem_u32(&full[s]), ph, tp.wait_limit, abort)) {
                    ok = false;
                    break;
                }
                fence_proxy_async();  // producer cp.async writes (generic proxy) before the MMA reads
                asm volatile("tcgen05.fence::after_thread_sync;");
                unsigned char *st = stages + s * TC_STAGE_BYTES;
                uint32_t sA = smem_u32(st), sAl = sA + TC_A_BYTES, sB = sAl + TC_A_BYTES, sBl = sB + TC_B_BYTES;
#pragma unroll
                for (int ks = 0; ks < TC_KG / 2; ++ks) {
                    uint32_t koff = 256u * ks;  // two 16-byte k-groups per MMA
                    uint64_t dAh = make_desc(sA + koff, 128, TC_SBO), dAl = make_desc(sAl + koff, 128, TC_SBO);
                    uint64_t dBh = make_desc(sB + koff, 128, TC_SBO), dBl = make_desc(sBl + koff, 128, TC_SBO);
                    uint32_t acc0 = (i > 0 || ks > 0) ? 1u : 0u;
                    mma_issue<BF16>(tmem, dAh, dBh, idesc, acc0);
                    mma_issue<BF16>(tmem, dAh, dBl, idesc, 1u);
                    mma_issue<BF16>(tmem, dAl, dBh, idesc, 1u);
                }
                mma_commit(smem_u32(&empty[s]));
            }
            // drain: every MMA issued above has completed once this commit arrives
            mma_commit(smem_u32(drain));
            if (!mbar_wait_drain(smem_u32(drain), 0u)) ok = false;
        }
    } else {
        // ------------------------------- producers ---------------------------------
        const int ptid = tid - 32;
        int released = 0;  // stages this warp has released on full[]
        int slot_cx[TC_BCHUNKS], slot_cy[TC_BCHUNKS], slot_cz[TC_BCHUNKS], slot_comp[TC_BCHUNKS], slot_kg[TC_BCHUNKS];
#pragma unroll
        for (int j = 0; j < TC_BCHUNKS; ++j) {
            // chunk v sits at byte 16 v: row 8 (v / (8 KG)) + v % 8, k-group (v / 8) % KG
            int v = ptid + TC_THREADS * j;
            int nrow = 8 * (v / (8 * TC_KG)) + (v & 7);
            slot_kg[j] = (v >> 3) % TC_KG;
            int q = nrow / 3;
            slot_comp[j] = nrow - 3 * q;
            int cell = cell_s[q];
            slot_cz[j] = cell % n;
            slot_cy[j] = (cell / n) % n;
            slot_cx[j] = cell / (n * n);
        }
        const unsigned char *Ahi = (const unsigned char *)tp.Ahi, *Alo = (const unsigned char *)tp.Alo;
        const unsigned char *Bhi = (const unsigned char *)tp.Bhi, *Blo = (const unsigned char *)tp.Blo;
        const size_t row_bytes = (size_t)pc * esz;
        for (int i = 0; i < nk + TC_PF; ++i) {
            if (i < nk) {
                const int s = i % TC_STAGES;
                if (i >= TC_STAGES &&
                    !mbar_wait_warp(smem_u32(&empty[s]), (uint32_t)(((i / TC_STAGES) - 1) & 1), tp.wait_limit, abort)) {
                    ok = false;
                    break;
                }
                int kbi = i / nchunk, ch = i - kbi * nchunk;
                int4 kb = kb_s[kbi];
                kb.x = checked_index(kb.x, NT, tp.err);
                unsigned char *st = stages + s * TC_STAGE_BYTES;
                uint32_t sA = smem_u32(st), sAl = sA + TC_A_BYTES, sB = sAl + TC_A_BYTES, sBl = sB + TC_B_BYTES;
                if (ptid == 0) {
                    uint32_t fb = smem_u32(&full[s]);
                    mbar_expect_tx(fb, 2 * TC_A_BYTES);
                    bulk_g2s(sA, Ahi + ((size_t)kb.x * nchunk + ch) * TC_A_BYTES, TC_A_BYTES, fb);
                    bulk_g2s(sAl, Alo + ((size_t)kb.x * nchunk + ch) * TC_A_BYTES, TC_A_BYTES, fb);
                    *issued_sh = i + 1;
                }
#pragma unroll
                for (int j = 0; j < TC_BCHUNKS; ++j) {
                    int v = ptid + TC_THREADS * j;
                    int sx = (slot_cx[j] + kb.y) & (n - 1);
                    int sy = (slot_cy[j] + kb.z) & (n - 1);
                    int sz = (slot_cz[j] + kb.w) & (n - 1);
                    const int64_t src = checked_index<int64_t>(((int64_t)sx * n + sy) * n + sz, (int64_t)n * n * n, tp.err);
                    size_t off = (size_t)(src * 3 + slot_comp[j]) * row_bytes + (size_t)ch * TC_KBYTES + 16 * slot_kg[j];
                    cp_async16(sB + 16 * v, Bhi + off);
                    cp_async16(sBl + 16 * v, Blo + off);
                }
            }
            cp_async_commit();
            if (i >= TC_PF) {
                // this thread's copies of stage i - TC_PF have landed: make them visible to the
                // async proxy, then one lane publishes the warp's share of the stage
                cp_async_wait<TC_PF>();
                fence_proxy_async();
                __syncwarp();
                if ((tid & 31) == 0) mbar_arrive(smem_u32(&full[(i - TC_PF) % TC_STAGES]));
                released = i - TC_PF + 1;
            }
        }
        // drain.  This thread's cp.async copies first.  Then the bulk copies of producer thread 0,
        // which complete on full[]: once every producer warp has left its loop (named barrier),
        // each warp arrives once on every stage thread 0 filled that it has not released (only
        // after a give-up), so each such phase completes when its bytes land, and thread 0 waits
        // for the last phase of every stage.
        cp_async_wait<0>();
        fence_proxy_async();
        asm volatile("bar.sync 1, %0;" ::"n"(TC_THREADS) : "memory");
        const int issued = *issued_sh;
        __syncwarp();
        if ((tid & 31) == 0)
            for (int j = released; j < issued; ++j) mbar_arrive(smem_u32(&full[j % TC_STAGES]));
        asm volatile("bar.sync 1, %0;" ::"n"(TC_THREADS) : "memory");
        if (ptid == 0)
            for (int j = issued > TC_STAGES ? issued - TC_STAGES : 0; j < issued; ++j)
                if (!mbar_wait_drain(smem_u32(&full[j % TC_STAGES]), (uint32_t)((j / TC_STAGES) & 1))) ok = false;
    }
    // epilogue: the MMA thread has seen its drain commit arrive (all MMAs done) before this
    // barrier; then warps 0..3 read TMEM lanes 32w..32w+31
    ok = __syncthreads_and((ok && !*abort) ? 1 : 0) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok && warp < 4) {
        const int k = 32 * warp + (tid & 31);
        float *C = tp.ksplit > 1 ? tp.partial + (int64_t)blockIdx.z * tp.n * tp.n * tp.n * 3 * pc : tp.C;
#pragma unroll 1
        for (int c0 = 0; c0 < TC_N; c0 += 16) {
            uint32_t r[16];
            uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                int col = c0 + e;
                int q = col / 3, comp = col - 3 * q;
                C[((int64_t)cell_s[q] * 3 + comp) * pc + k] = __uint_as_float(r[e]);
            }
        }
    } else if (tid == 0) {
        atomicOr(tp.err, ERRBIT_TIMEOUT);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
    }
}

// ---------------------------------------------------------------------------------------
// Source-line variant for levels with 16 to 64 cells per side and parity.
//
// The hi/lo multipoles of the level are first rearranged by K slice and parity into
//   G[slice][b][X][kg][Zp][Yp][component][16 bytes],  b = parity (bx, by, bz), kg = k-group,
//   Zp = Z + 2 and Yp = Y + 2 (two halo cells on each side, copied periodically),
// so that the rows a CTA needs from one source x-column form one box of a 5-d tensor that a
// single TMA tensor copy lands in shared memory in the MMA's operand layout.  The CTA walks the
// K slices in the outer loop: the CTAs resident at one time then share the slice's source lines
// in L2.  The grid's fastest index is the target parity, so the eight parities of one group of
// lines (which read the same source lines) run together.
// A CTA owns whole z-lines of target cells of one parity g (128 cells: N = 384 columns of TMEM):
// LINES consecutive y-lines of one x-column.  For an offset t the sources of a target line are
// one z-line of G (parity b = (g + t) mod 2, shifted by (g + t) >> 1 in x and y) read through a
// z window shifted by shz = (g_z + t_z) >> 1.  Offsets that share (b, shx, shy) form a class (up
// to three offsets, differing in shz): the class's source lines are copied into shared memory
// once per K slice, in the no-swizzle K-major layout with 16-byte rows ([k-group][row][16 B])
// and rows ordered (Zp, line, component), so the window of every offset of the class is one
// contiguous run of 384 rows starting 3 LINES (shz + 2) rows in: two MMAs (N = 192) per offset
// and split product.  Each source row copied serves all offsets of its class and each
// translation-matrix tile 384 columns.
//
// One thread of warp 1 moves everything with TMA (the translation tiles as bulk copies, the
// source lines as one tensor copy per hi/lo), all completing on the stage's transaction
// barrier; one thread of warp 0 issues the MMAs; all four warps read TMEM in the epilogue.
constexpr int TL_CELLS = 128;              // target cells per CTA (whole z-lines)
constexpr int TL_N = 3 * TL_CELLS;         // accumulator columns
constexpr int TL_HALO = 2;                 // |shx|, |shy|, |shz| <= 2 (two near rings)
constexpr int TL_MAXOFF = 3;               // offsets per class (the z parity leaves at most three)
#ifndef VFMM_TL_STAGES
#define VFMM_TL_STAGES 3
#endif
constexpr int TL_STAGES = VFMM_TL_STAGES;
constexpr int TL_MAXCLS = 96;
constexpr int TL_TMEM_COLS = 512;
constexpr int TL_THREADS = 128;            // warp 0: MMA issuer, warp 1: TMA producer; all: epilogue
// shared bytes of one stage: up to three A tile pairs (hi, lo) and the class's source lines (hi, lo)
template <int H> struct TlGeom {
    static constexpr int LINES = TL_CELLS / H;
    static constexpr int YP = H + 2 * TL_HALO;               // y extent of G (with halo)
    static constexpr int ZP = H + 2 * TL_HALO;               // z extent of G (with halo)
    static constexpr int ROWS = ZP * LINES * 3;              // staged rows (Zp, line, component)
    static constexpr int ROW_Z = LINES * 3;                  // staged rows per z step
    static constexpr int PLANE = ROWS * 16;                  // bytes of one 16-byte k-group plane
    static constexpr int A_BYTES = TL_MAXOFF * 2 * TC_A_BYTES;
    static constexpr int BOX_BYTES = TC_KG * PLANE;          // one tensor copy (hi or lo)
    static constexpr int B_BYTES = 2 * BOX_BYTES;            // hi and lo
    static constexpr int STAGE = (A_BYTES + B_BYTES + 1023) / 1024 * 1024;
    static constexpr int SMEM = TL_STAGES * STAGE + 1024 + 256 + TL_MAXCLS * 48;
    static constexpr int BOX_X = ROW_Z * 8;                  // innermost box extent in 2-byte elements
    static_assert(TL_N == 2 * 192, "two MMAs of N = 192 per offset and product");
    static_assert(TC_KG == 2, "the tensor box holds two 16-byte k-groups");
    static_assert(BOX_X <= 256 && ZP <= 256, "TMA box extents");
    static_assert((A_BYTES % 128) == 0 && (PLANE % 128) == 0, "128-byte aligned TMA destinations");
    static_assert(SMEM <= 232448, "shared memory per CTA");
};

// TMA tensor copy of a 5-d box global -> shared, completing on `bar` (transaction bytes)
__device__ __forceinline__ void tensor_g2s_5d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                              int c4, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
        "%6}], [%7];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
        : "memory");
}

#ifndef VFMM_TL_MINB
#define VFMM_TL_MINB 1
#endif
template <bool BF16, int H>
__global__ void __launch_bounds__(TL_THREADS, VFMM_TL_MINB)
    k_m2l_lines(TcParams tp, const int4 *__restrict__ cls, const __grid_constant__ CUtensorMap tm_hi,
                const __grid_constant__ CUtensorMap tm_lo)
{
    using Gm = TlGeom<H>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *stages = base;
    uint64_t *full = (uint64_t *)(base + TL_STAGES * Gm::STAGE);
    uint64_t *empty = full + TL_STAGES;
    uint64_t *drain = empty + TL_STAGES;  // final tcgen05.commit
    uint32_t *tmem_slot = (uint32_t *)(drain + 1);
    volatile int *abort = (volatile int *)(tmem_slot + 1);
    int4 *cls_s = (int4 *)(base + TL_STAGES * Gm::STAGE + 256);

    const int tid = threadIdx.x, warp = tid >> 5;
    const int g = blockIdx.x;                  // target parity (the fastest grid index)
    const int n = tp.n;
    const int line0 = blockIdx.y * Gm::LINES;  // first target line (px * H + py) of this CTA
    const int ncls = min(tp.kb_cnt[g], TL_MAXCLS);
    for (int q = tid; q < 3 * ncls; q += TL_THREADS) cls_s[q] = cls[3 * tp.kb_off[g] + q];
    const int nchunk = tp.nchunk;
    const int nk = ncls * nchunk;
    const int pc = tp.pc;

    if (tid == 0) {
        for (int s = 0; s < TL_STAGES; ++s) {
            mbar_init(smem_u32(&full[s]), 1);   // the producer's expect_tx arrival; completes when the bytes land
            mbar_init(smem_u32(&empty[s]), 1);  // tcgen05.commit
        }
        mbar_init(smem_u32(drain), 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TL_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;
    bool ok = true;

    if (tid == 0) {
        // ------------------------------- MMA issuer -------------------------------
        const uint32_t fmt = BF16 ? 1u : 2u;
        const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(192 >> 3) << 17) |
                               ((uint32_t)(TC_M >> 4) << 24);
        for (int i = 0; i < nk; ++i) {
            const int s = i % TL_STAGES;
            const uint32_t ph = (uint32_t)((i / TL_STAGES) & 1);
            if (!mbar_wait(smem_u32(&full[s]), ph, tp.wait_limit, abort)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int ci = i % ncls;
            const int4 hd = cls_s[3 * ci], e01 = cls_s[3 * ci + 1], e23 = cls_s[3 * ci + 2];
            const int cnt = min(hd.w, TL_MAXOFF);
            const uint32_t st = smem_u32(stages + s * Gm::STAGE);
            const uint32_t sB = st + Gm::A_BYTES, sBl = sB + Gm::BOX_BYTES;
            for (int e = 0; e < cnt; ++e) {
                const int shz = e == 0 ? e01.y : e == 1 ? e01.w : e23.y;
                const uint32_t sA = st + (uint32_t)(e * 2 * TC_A_BYTES), sAl = sA + TC_A_BYTES;
                const uint64_t dAh = make_desc(sA, 128, TC_SBO), dAl = make_desc(sAl, 128, TC_SBO);
                const uint32_t acc0 = (i > 0 || e > 0) ? 1u : 0u;
#pragma unroll
                for (int hfl = 0; hfl < 2; ++hfl) {
                    const uint32_t woff = (uint32_t)(((shz + TL_HALO) * Gm::ROW_Z + 192 * hfl) * 16);
                    const uint64_t dBh = make_desc(sB + woff, Gm::PLANE, 128);
                    const uint64_t dBl = make_desc(sBl + woff, Gm::PLANE, 128);
                    const uint32_t td = tmem + (uint32_t)(192 * hfl);
                    mma_issue<BF16>(td, dAh, dBh, idesc, acc0);
                    mma_issue<BF16>(td, dAh, dBl, idesc, 1u);
                    mma_issue<BF16>(td, dAl, dBh, idesc, 1u);
                }
            }
            mma_commit(smem_u32(&empty[s]));
        }
        // drain: every MMA issued above has completed once this commit arrives
        mma_commit(smem_u32(drain));
        if (!mbar_wait_drain(smem_u32(drain), 0u)) ok = false;
    } else if (tid == 32) {
        // ------------------------------- TMA producer -----------------------------
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tm_hi)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tm_lo)) : "memory");
        const unsigned char *Ahi = (const unsigned char *)tp.Ahi, *Alo = (const unsigned char *)tp.Alo;
        const int px = line0 / H, py0 = line0 - px * H;  // the CTA's lines: y = py0 .. py0 + LINES - 1
        int issued = 0;
        for (int i = 0; i < nk; ++i) {
            const int s = i % TL_STAGES;
            if (i >= TL_STAGES &&
                !mbar_wait(smem_u32(&empty[s]), (uint32_t)(((i / TL_STAGES) - 1) & 1), tp.wait_limit, abort)) {
                ok = false;
                break;
            }
            const int ch = i / ncls, ci = i - ch * ncls;
            const int4 hd = cls_s[3 * ci], e01 = cls_s[3 * ci + 1], e23 = cls_s[3 * ci + 2];
            const int cnt = min(hd.w, TL_MAXOFF);
            const uint32_t st = smem_u32(stages + s * Gm::STAGE);
            const uint32_t fb = smem_u32(&full[s]);
            mbar_expect_tx(fb, (uint32_t)(cnt * 2 * TC_A_BYTES + Gm::B_BYTES));
            for (int e = 0; e < cnt; ++e) {
                const int tile = checked_index(e == 0 ? e01.x : e == 1 ? e01.z : e23.x, NT, tp.err);
                const uint32_t sA = st + (uint32_t)(e * 2 * TC_A_BYTES);
                bulk_g2s(sA, Ahi + ((size_t)tile * nchunk + ch) * TC_A_BYTES, TC_A_BYTES, fb);
                bulk_g2s(sA + TC_A_BYTES, Alo + ((size_t)tile * nchunk + ch) * TC_A_BYTES, TC_A_BYTES, fb);
            }
            // the class's source lines: target line (px, py) reads G[bpar][(px + shx) mod H][py + shy]
            // (periodic through the y halo) over all Zp; one box per hi/lo holds the LINES lines
            const int X = checked_index((px + hd.y) & (H - 1), H, tp.err);
            const int yp0 = checked_index(py0 + hd.z + TL_HALO, Gm::YP - Gm::LINES + 1, tp.err);
            const int c4 = checked_index(ch * 8 + hd.x, nchunk * 8, tp.err);
            const uint32_t sB = st + Gm::A_BYTES;
            tensor_g2s_5d(sB, &tm_hi, yp0 * 24, 0, 0, X, c4, fb);
            tensor_g2s_5d(sB + Gm::BOX_BYTES, &tm_lo, yp0 * 24, 0, 0, X, c4, fb);
            issued = i + 1;
        }
        // drain: a stage this thread filled completes its phase once its bytes land (one arrival,
        // made with the expect_tx); wait for the last phase of every stage
        for (int j = issued > TL_STAGES ? issued - TL_STAGES : 0; j < issued; ++j)
            if (!mbar_wait_drain(smem_u32(&full[j % TL_STAGES]), (uint32_t)((j / TL_STAGES) & 1))) ok = false;
    }
    // epilogue: the MMA thread has seen its drain commit arrive (all MMAs done) and the producer
    // its copies land before this barrier; then warps 0..3 read TMEM lanes 32w..32w+31
    ok = __syncthreads_and((ok && !*abort) ? 1 : 0) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok) {
        const int k = 32 * warp + (tid & 31);
        float *C = tp.C;
        const int gx = (g >> 2) & 1, gy = (g >> 1) & 1, gz = g & 1;
#pragma unroll 1
        for (int c0 = 0; c0 < TL_N; c0 += 16) {
            uint32_t r[16];
            uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int col = c0 + e;  // (z, line, component)
                const int pz = col / (Gm::LINES * 3), w = col - pz * Gm::LINES * 3;
                const int l = w / 3, comp = w - 3 * l;
                const int L = line0 + l;
                const int px = L / H, py = L - (L / H) * H;
                const int64_t cell = ((int64_t)(2 * px + gx) * n + (2 * py + gy)) * n + (2 * pz + gz);
                C[(cell * 3 + comp) * pc + k] = __uint_as_float(r[e]);
            }
        }
    } else if (tid == 0) {
        atomicOr(tp.err, ERRBIT_TIMEOUT);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TL_TMEM_COLS));
    }
}

// FP32 multipoles [cell][3][pc] of one level -> hi/lo parity grid
// G[slice][b][X][kg][Zp][Yp][3][16 bytes] (h = n/2 cells per side and parity, Yp = Y + 2 and
// Zp = Z + 2 with two periodic halo cells per side).  One thread per 8 consecutive
// coefficients of one (cell, component) row (pc is a multiple of 8).
template <typename TS>
__global__ void k_split_grid(int n, int pc, const float *__restrict__ M, TS *__restrict__ hi, TS *__restrict__ lo)
{
    const int h = n >> 1, ext = h + 2 * TL_HALO, pv = pc >> 3;
    const int64_t count = (int64_t)8 * h * ext * ext * 3 * pv;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    int64_t r = i;
    const int kv = (int)(r % pv); r /= pv;
    const int comp = (int)(r % 3); r /= 3;
    const int Yp = (int)(r % ext); r /= ext;  // y inside z, as in the destination
    const int Zp = (int)(r % ext); r /= ext;
    const int X = (int)(r % h); r /= h;
    const int b = (int)r;
    const int Y = (Yp - TL_HALO + h) & (h - 1), Z = (Zp - TL_HALO + h) & (h - 1);
    const int64_t cell = ((int64_t)(2 * X + ((b >> 2) & 1)) * n + (2 * Y + ((b >> 1) & 1))) * n + (2 * Z + (b & 1));
    const float4 *src = (const float4 *)(M + (cell * 3 + comp) * pc + 8 * kv);
    // 16-byte destination row of k-group kg of K slice ch (32 bytes: 16 BF16 / 8 TF32 coefficients)
    constexpr int VPS = TC_KBYTES / (8 * (int)sizeof(TS));  // 8-coefficient vectors per slice
    const int ch = kv / VPS, part = kv - ch * VPS;
    auto row16 = [&](int kg) -> int64_t {
        return (((((int64_t)ch * 8 + b) * h + X) * 2 + kg) * ext + Zp) * ext * 3 + (int64_t)Yp * 3 + comp;
    };
    const float4 a = src[0], c = src[1];
    const float v[8] = {a.x, a.y, a.z, a.w, c.x, c.y, c.z, c.w};
    if constexpr (sizeof(TS) == 2) {
        __align__(16) __nv_bfloat16 hv[8], lv[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            hv[e] = __float2bfloat16_rn(v[e]);
            lv[e] = __float2bfloat16_rn(v[e] - __bfloat162float(hv[e]));
        }
        const int64_t o = row16(part);
        reinterpret_cast<uint4 *>(hi)[o] = *reinterpret_cast<const uint4 *>(hv);
        reinterpret_cast<uint4 *>(lo)[o] = *reinterpret_cast<const uint4 *>(lv);
    } else {
        float hv[8], lv[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            hv[e] = to_tf32_dev(v[e]);
            lv[e] = to_tf32_dev(v[e] - hv[e]);
        }
        float4 *H = reinterpret_cast<float4 *>(hi), *Lo = reinterpret_cast<float4 *>(lo);
        const int64_t o0 = row16(0), o1 = row16(1);
        H[o0] = make_float4(hv[0], hv[1], hv[2], hv[3]);
        H[o1] = make_float4(hv[4], hv[5], hv[6], hv[7]);
        Lo[o0] = make_float4(lv[0], lv[1], lv[2], lv[3]);
        Lo[o1] = make_float4(lv[4], lv[5], lv[6], lv[7]);
    }
}

// FP32 multipoles -> hi/lo split in BF16 or TF32 (the latter kept in FP32 containers).
__global__ void k_split_bf16(int64_t count, const float *__restrict__ M, __nv_bfloat16 *__restrict__ hi,
                             __nv_bfloat16 *__restrict__ lo)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    float v = M[i];
    __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[i] = h;
    lo[i] = __float2bfloat16_rn(v - __bfloat162float(h));
}

__device__ __forceinline__ float to_tf32(float v)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return __uint_as_float(r);
}

__global__ void k_split_tf32(int64_t count, const float *__restrict__ M, float *__restrict__ hi, float *__restrict__ lo)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    float v = M[i];
    float h = to_tf32(v);
    hi[i] = h;
    lo[i] = to_tf32(v - h);
}

void set_carveouts_m2l()
{
    prefer_max_shared(k_m2l_tc<true>);
    prefer_max_shared(k_m2l_tc<false>);
    prefer_max_shared(k_m2l_lines<true, 16>);
    prefer_max_shared(k_m2l_lines<true, 32>);
    prefer_max_shared(k_m2l_lines<true, 64>);
    prefer_max_shared(k_m2l_lines<false, 16>);
    prefer_max_shared(k_m2l_lines<false, 32>);
    prefer_max_shared(k_m2l_lines<false, 64>);
    prefer_max_shared(k_split_grid<__nv_bfloat16>);
    prefer_max_shared(k_split_grid<float>);
    prefer_max_shared(k_split_bf16);
    prefer_max_shared(k_split_tf32);
}

bool grid_level(int level)
{
    const int h = (1 << level) / 2;
    return h >= 16 && h <= 64;
}

size_t split_count(int level, int pc)
{
    const int64_t n = (int64_t)1 << level;
    if (!grid_level(level)) return (size_t)(n * n * n * 3 * pc);
    const int64_t h = n / 2;
    return (size_t)(8 * h * (h + 2 * TL_HALO) * (h + 2 * TL_HALO) * 3 * pc);
}

int launch_split(Ctx *c, int level, bool bf16)
{
    const float *M = (const float *)c->mexp.p + c->lvl_off[level];
    if (grid_level(level)) {
        int64_t count = (int64_t)split_count(level, c->pc) / 8;  // 8 coefficients per thread
        int nb = (int)((count + 255) / 256);
        if (bf16)
            k_split_grid<__nv_bfloat16><<<nb, 256, 0, c->stream>>>(1 << level, c->pc, M, (__nv_bfloat16 *)c->mhi.p,
                                                                  (__nv_bfloat16 *)c->mlo.p);
        else
            k_split_grid<float><<<nb, 256, 0, c->stream>>>(1 << level, c->pc, M, (float *)c->mhi.p, (float *)c->mlo.p);
        VFMM_CUDA_CHECK_LAUNCH(c);
        return VFMM_OK;
    }
    int64_t count = ((int64_t)1 << (3 * level)) * 3 * c->pc;
    int nb = (int)((count + 255) / 256);
    if (bf16)
        k_split_bf16<<<nb, 256, 0, c->stream>>>(count, M, (__nv_bfloat16 *)c->mhi.p, (__nv_bfloat16 *)c->mlo.p);
    else
        k_split_tf32<<<nb, 256, 0, c->stream>>>(count, M, (float *)c->mhi.p, (float *)c->mlo.p);
    VFMM_CUDA_CHECK_LAUNCH(c);
    return VFMM_OK;
}

void build_line_classes(const std::vector<int4> &kb, int off, int cnt, int g, std::vector<int4> &out)
{
    // group the offsets of one parity's list by (source parity, x shift, y shift)
    const int gx = (g >> 2) & 1, gy = (g >> 1) & 1, gz = g & 1;
    std::vector<int4> hd, e01, e23;
    for (int q = 0; q < cnt; ++q) {
        const int4 t = kb[off + q];
        const int sx = gx + t.y, sy = gy + t.z, sz = gz + t.w;
        const int bpar = ((sx & 1) << 2) | ((sy & 1) << 1) | (sz & 1);
        const int shx = sx >> 1, shy = sy >> 1, shz = sz >> 1;
        size_t k = 0;
        while (k < hd.size() && !(hd[k].x == bpar && hd[k].y == shx && hd[k].z == shy && hd[k].w < TL_MAXOFF)) ++k;
        if (k == hd.size()) {
            hd.push_back(make_int4(bpar, shx, shy, 0));
            e01.push_back(make_int4(0, 0, 0, 0));
            e23.push_back(make_int4(0, 0, 0, 0));
        }
        int e = hd[k].w++;
        int4 &d = e < 2 ? e01[k] : e23[k];
        if (e % 2 == 0) {
            d.x = t.x;
            d.y = shz;
        } else {
            d.z = t.x;
            d.w = shz;
        }
    }
    for (size_t k = 0; k < hd.size(); ++k) {
        out.push_back(hd[k]);
        out.push_back(e01[k]);
        out.push_back(e23[k]);
    }
}

namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled from the driver, through the runtime's entry-point query (no link
// against the driver library)
EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

// Tensor map of one hi or lo parity grid G[slice][b][X][kg][Zp][Yp][3][16 B] of a level with H
// cells per side and parity, as 2-byte elements (the bytes are copied, whatever the type):
// dims (innermost first) (Yp, component, 8 elements) flattened, Zp, kg, X, (slice, b).  The box
// is LINES y-lines of all Zp and both k-groups of one (slice, b, X): in shared memory
// [kg][Zp][line][component][16 B], the operand layout of the MMA.
template <int H> bool encode_grid_map(CUtensorMap *map, const void *G, int nchunk)
{
    using Gm = TlGeom<H>;
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return false;
    const cuuint64_t row = (cuuint64_t)Gm::YP * 3 * 16;  // bytes of one (kg, Zp) run of Yp rows
    const cuuint64_t dims[5] = {(cuuint64_t)Gm::YP * 3 * 8, (cuuint64_t)Gm::ZP, 2, (cuuint64_t)H, (cuuint64_t)nchunk * 8};
    const cuuint64_t strides[4] = {row, row * Gm::ZP, row * Gm::ZP * 2, row * Gm::ZP * 2 * H};
    const cuuint32_t box[5] = {(cuuint32_t)Gm::BOX_X, (cuuint32_t)Gm::ZP, 2, 1, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 5, const_cast<void *>(G), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <bool BF16, int H> int launch_lines(Ctx *c, int level, int R, const TcParams &tp0)
{
    using Gm = TlGeom<H>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_m2l_lines<BF16, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, Gm::SMEM);
        if (e != cudaSuccess) {
            c->last_error = std::string("tensor-core M2L shared memory: ") + cudaGetErrorString(e);
            return VFMM_ERR_CUDA;
        }
        attr = true;
    }
    TcParams tp = tp0;
    for (int g = 0; g < 8; ++g) {
        tp.kb_off[g] = c->cls_off[R][g];
        tp.kb_cnt[g] = c->cls_cnt[R][g];
    }
    CUtensorMap mh, ml;
    if (!encode_grid_map<H>(&mh, tp.Bhi, tp.nchunk) || !encode_grid_map<H>(&ml, tp.Blo, tp.nchunk)) {
        c->last_error = "tensor-core M2L: cuTensorMapEncodeTiled failed";
        return VFMM_ERR_CUDA;
    }
    const int lines = H * H;  // target z-lines per parity
    dim3 grid(8, (unsigned)(lines / Gm::LINES));
    k_m2l_lines<BF16, H><<<grid, TL_THREADS, Gm::SMEM, c->stream>>>(tp, (const int4 *)c->cls.p, mh, ml);
    VFMM_CUDA_CHECK_LAUNCH(c);
    return VFMM_OK;
}
}  // namespace

int launch_tc_m2l(Ctx *c, int level, int R, bool bf16)
{
    const int n = 1 << level;
    const int64_t ncg = (int64_t)(n / 2) * (n / 2) * (n / 2);
    if (ncg % TC_CELLS != 0 || c->pc != TC_M) {
        c->last_error = "tensor-core M2L needs 64 | (n/2)^3 and 128 padded coefficients";
        return VFMM_ERR_UNSUPPORTED;
    }
    TcParams tp;
    tp.ksplit = 1;
    tp.partial = nullptr;
    tp.Ahi = c->tc_hi.p;
    tp.Alo = c->tc_lo.p;
    tp.Bhi = c->mhi.p;
    tp.Blo = c->mlo.p;
    tp.C = (float *)c->lexp.p + c->lvl_off[level];
    tp.kb = (const int4 *)c->kblocks.p;
    for (int g = 0; g < 8; ++g) {
        tp.kb_off[g] = c->kb_m2l_off[R][g];
        tp.kb_cnt[g] = c->kb_m2l_cnt[R][g];
    }
    tp.n = n;
    tp.pc = c->pc;
    tp.nchunk = c->pc * (bf16 ? 2 : 4) / TC_KBYTES;
    tp.err = (int *)c->err.p;
    tp.wait_limit = c->wait_limit;
    if (grid_level(level)) {
        const int h = n / 2;
        if (h == 16) return bf16 ? launch_lines<true, 16>(c, level, R, tp) : launch_lines<false, 16>(c, level, R, tp);
        if (h == 32) return bf16 ? launch_lines<true, 32>(c, level, R, tp) : launch_lines<false, 32>(c, level, R, tp);
        return bf16 ? launch_lines<true, 64>(c, level, R, tp) : launch_lines<false, 64>(c, level, R, tp);
    }
    static bool attr_set[2] = {false, false};
    if (!attr_set[bf16 ? 1 : 0]) {
        cudaError_t e = bf16 ? cudaFuncSetAttribute(k_m2l_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM)
                             : cudaFuncSetAttribute(k_m2l_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
        if (e != cudaSuccess) {
            c->last_error = std::string("tensor-core M2L shared memory: ") + cudaGetErrorString(e);
            return VFMM_ERR_CUDA;
        }
        attr_set[bf16 ? 1 : 0] = true;
    }
    // few CTAs (levels 3 and 4): split the offsets over at most one wave of CTAs (two per SM;
    // rounding up to more than one wave left a second wave of a few CTAs that doubled the time:
    // 320 CTAs took 0.58 ms at 16^3 cells), partial tiles summed by a second pass in a fixed order
    dim3 grid((unsigned)(ncg / TC_CELLS), 8);
    const int64_t blocks = (int64_t)grid.x * grid.y;
    const int64_t count = (int64_t)n * n * n * 3 * c->pc;
    const int64_t slots = 2 * (int64_t)std::max(c->sm_count, 1);
    int maxkb = 0;
    for (int g = 0; g < 8; ++g) maxkb = std::max(maxkb, tp.kb_cnt[g]);
    int ksplit = 1;
    if (blocks < slots) {
        ksplit = (int)std::min<int64_t>(maxkb, slots / blocks);
        ksplit = (int)std::min<int64_t>(ksplit, (int64_t)(c->gemm_part.bytes / sizeof(float)) / count);
        // every slice keeps at least one offset
        while (ksplit > 1 && (int64_t)((maxkb + ksplit - 1) / ksplit) * (ksplit - 1) >= maxkb) --ksplit;
        for (int g = 0; g < 8; ++g)
            while (ksplit > 1 && (int64_t)((tp.kb_cnt[g] + ksplit - 1) / ksplit) * (ksplit - 1) >= tp.kb_cnt[g]) --ksplit;
        if (ksplit < 1) ksplit = 1;
    }
    tp.ksplit = ksplit;
    tp.partial = (float *)c->gemm_part.p;
    grid.z = (unsigned)ksplit;
    if (bf16)
        k_m2l_tc<true><<<grid, TC_WS_THREADS, TC_SMEM, c->stream>>>(tp);
    else
        k_m2l_tc<false><<<grid, TC_WS_THREADS, TC_SMEM, c->stream>>>(tp);
    VFMM_CUDA_CHECK_LAUNCH(c);
    if (ksplit > 1) {
        int rc = launch_split_reduce(c, ksplit, count, tp.partial, tp.C, 0, true);
        if (rc) return rc;
    }
    return VFMM_OK;
}

}  // namespace vfmm

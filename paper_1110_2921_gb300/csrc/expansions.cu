// Expansion kernels of the periodic FMM: P2M, the gathered-column GEMM that performs M2M,
// M2L and L2L on the CUDA cores (split over k-blocks on small levels), the FP64 root /
// periodic lattice step, L2P, and the scatter that adds the far field to the outputs.
//
// Section 3.1: the vector potential psi_c = sum_j gamma_{j,c} G (three scalar Laplace
// potentials) is expanded in multipoles (Eq. fmm3dm) and locals (Eq. fmm3dl); velocity is
// its curl (Eqs. biotsavartfmm1-2) and the stretching term uses its second derivatives
// (Eqs. stretchingfmm1-2).  Coefficients use the balanced packed layout documented in
// operators.cpp; every cell's block is [3][pc] (pc = padded coefficient stride).
#include "common.cuh"

#include <algorithm>
#include "vfmm_internal.h"

namespace vfmm {

__constant__ float c_sfac_f[(PMAX + 1) * (PMAX + 1)];
__constant__ double c_sfac_d[(PMAX + 1) * (PMAX + 1)];
__constant__ float c_rec_f[(PMAX + 1) * (PMAX + 1)];   // 1/((n+m)(n-m)), n > m
__constant__ double c_rec_d[(PMAX + 1) * (PMAX + 1)];
__constant__ float c_inv2m_f[PMAX + 1];                // 1/(2m)
__constant__ double c_inv2m_d[PMAX + 1];

template <typename T> __device__ __forceinline__ T sfac_t(int n, int m);
template <> __device__ __forceinline__ float sfac_t<float>(int n, int m) { return c_sfac_f[n * (PMAX + 1) + m]; }
template <> __device__ __forceinline__ double sfac_t<double>(int n, int m) { return c_sfac_d[n * (PMAX + 1) + m]; }
// The same factors in global memory, for lookups whose (n, m) differs across a warp: constant
// memory serialises a warp's loads from different addresses, the L1 serves them together.
__device__ float g_sfac_f[(PMAX + 1) * (PMAX + 1)];
__device__ double g_sfac_d[(PMAX + 1) * (PMAX + 1)];
template <typename T> __device__ __forceinline__ T sfac_ld(int n, int m);
template <> __device__ __forceinline__ float sfac_ld<float>(int n, int m) { return __ldg(&g_sfac_f[n * (PMAX + 1) + m]); }
template <> __device__ __forceinline__ double sfac_ld<double>(int n, int m) { return __ldg(&g_sfac_d[n * (PMAX + 1) + m]); }
template <typename T> __device__ __forceinline__ T rec_t(int n, int m);
template <> __device__ __forceinline__ float rec_t<float>(int n, int m) { return c_rec_f[n * (PMAX + 1) + m]; }
template <> __device__ __forceinline__ double rec_t<double>(int n, int m) { return c_rec_d[n * (PMAX + 1) + m]; }
template <typename T> __device__ __forceinline__ T inv2m_t(int m);
template <> __device__ __forceinline__ float inv2m_t<float>(int m) { return c_inv2m_f[m]; }
template <> __device__ __forceinline__ double inv2m_t<double>(int m) { return c_inv2m_d[m]; }

void set_constants(int)
{
    float sf[(PMAX + 1) * (PMAX + 1)] = {0}, rf[(PMAX + 1) * (PMAX + 1)] = {0}, i2f[PMAX + 1] = {0};
    double sd[(PMAX + 1) * (PMAX + 1)] = {0}, rd[(PMAX + 1) * (PMAX + 1)] = {0}, i2d[PMAX + 1] = {0};
    for (int n = 0; n <= PMAX; ++n)
        for (int m = 0; m <= n; ++m) {
            sd[n * (PMAX + 1) + m] = ops::sfac(n, m);
            sf[n * (PMAX + 1) + m] = (float)sd[n * (PMAX + 1) + m];
            if (n > m) {
                rd[n * (PMAX + 1) + m] = 1.0 / double((n + m) * (n - m));
                rf[n * (PMAX + 1) + m] = (float)rd[n * (PMAX + 1) + m];
            }
        }
    for (int m = 1; m <= PMAX; ++m) {
        i2d[m] = 1.0 / (2.0 * m);
        i2f[m] = (float)i2d[m];
    }
    cudaMemcpyToSymbol(c_sfac_f, sf, sizeof(sf));
    cudaMemcpyToSymbol(c_sfac_d, sd, sizeof(sd));
    cudaMemcpyToSymbol(g_sfac_f, sf, sizeof(sf));
    cudaMemcpyToSymbol(g_sfac_d, sd, sizeof(sd));
    cudaMemcpyToSymbol(c_rec_f, rf, sizeof(rf));
    cudaMemcpyToSymbol(c_rec_d, rd, sizeof(rd));
    cudaMemcpyToSymbol(c_inv2m_f, i2f, sizeof(i2f));
    cudaMemcpyToSymbol(c_inv2m_d, i2d, sizeof(i2d));
    set_carveouts_expansions();
    set_carveouts_p2p();
    set_carveouts_m2l();
}

__device__ __forceinline__ int pk(int n, int m) { return m == 0 ? n * n : n * n + 2 * m - 1; }

// ---------------------------------------------------------------------------------------
// gamma gather: gs[pos] = gamma[perm[pos]] in the compute type
template <typename T>
__global__ void k_gather_gamma(int64_t n, const T *__restrict__ g, const int *__restrict__ perm,
                               typename V4<T>::type *__restrict__ gs)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t s = perm[i];
    gs[i] = make_v4<T>(g[3 * s], g[3 * s + 1], g[3 * s + 2], T(0));
}

int launch_gather_gamma(Ctx *c, const void *gamma)
{
    int nb = (int)((c->n + 255) / 256);
    if (c->f64)
        k_gather_gamma<double><<<nb, 256, 0, c->stream>>>(c->n, (const double *)gamma, (const int *)c->perm.p,
                                                          (dvec4 *)c->gs.p);
    else
        k_gather_gamma<float><<<nb, 256, 0, c->stream>>>(c->n, (const float *)gamma, (const int *)c->perm.p,
                                                        (float4 *)c->gs.p);
    VFMM_CUDA_CHECK_LAUNCH(c);
    return VFMM_OK;
}

// ---------------------------------------------------------------------------------------
// P2M (Eq. fmm3dm): Mh_n^m = s_nm sum_j gamma_j Y_n^m((x_j - z)/w) for each leaf.
// One block of 128 threads per leaf.  Phase 1: the harmonics of a chunk of particles go to
// shared memory; each particle's orders m are split over P2M_BS / TP threads (the short
// diagonal recurrence is repeated by each).  Phase 2: thread (h, j) owns coefficients j and j + 64 of all three
// components and sums gamma_j Y over the chunk (conflict-free rows, broadcast strengths).
template <typename T> struct P2MCfg {
    static constexpr int TP = sizeof(T) == 4 ? 64 : 32;  // particles per chunk
};
constexpr int P2M_BS = 128;

// PF > 0 compiles the order in (the harmonic recursion unrolls completely, its constants become
// immediates); PF = 0 takes it from the argument.
template <typename T, int PF>
__global__ void __launch_bounds__(P2M_BS) k_p2m(const typename V4<T>::type *__restrict__ xs,
                                                const typename V4<T>::type *__restrict__ gs,
                                                const int *__restrict__ ls, int nside, int log2n, T w, int p_arg,
                                                int pc, T *__restrict__ M)
{
    const int p = PF > 0 ? PF : p_arg;
    constexpr int TP = P2MCfg<T>::TP;
    constexpr int NSPLIT = P2M_BS / TP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ys = pc + 1;                  // padded row stride: the column writes of a warp hit distinct banks
    T *Ysm = (T *)smem_raw;                                              // [TP][ys]
    typename V4<T>::type *gsm = (typename V4<T>::type *)(((uintptr_t)(Ysm + TP * ys) + 15) & ~(uintptr_t)15);
    const int leaf = blockIdx.x;
    const int cz = leaf & (nside - 1), cy = (leaf >> log2n) & (nside - 1), cx = leaf >> (2 * log2n);
    const T zx = (cx + T(0.5)) * w, zy = (cy + T(0.5)) * w, zz = (cz + T(0.5)) * w;
    const T invw = T(1) / w;
    const int b = ls[leaf], e = ls[leaf + 1];
    const int nc = (p + 1) * (p + 1);
    const int q = threadIdx.x % TP, part = threadIdx.x / TP;
    const int jp = threadIdx.x & 63, half = threadIdx.x >> 6;  // phase 2: coefficient pair, particle parity
    T a0 = 0, a1 = 0, a2 = 0, b0 = 0, b1 = 0, b2 = 0;
    for (int s0 = b; s0 < e; s0 += TP) {
        const int cnt = min(TP, e - s0);
        if (q < cnt) {
            T *row = Ysm + q * ys;
            typename V4<T>::type xp = xs[s0 + q];
            if (part == 0) {
                gsm[q] = gs[s0 + q];
                for (int jj = nc; jj < pc; ++jj) row[jj] = 0;
            }
            T x = (xp.x - zx) * invw, y = (xp.y - zy) * invw, z = (xp.z - zz) * invw;
            T r2 = x * x + y * y + z * z;
            T dre = 1, dim = 0;
#pragma unroll(PF > 0 ? PF + 1 : 1)
            for (int m = 0; m <= p; ++m) {
                if (m > 0) {
                    T f = -inv2m_t<T>(m);
                    T nre = f * (x * dre - y * dim);
                    T nim = f * (x * dim + y * dre);
                    dre = nre;
                    dim = nim;
                }
                if (m % NSPLIT != part) continue;
                T sm = sfac_t<T>(m, m);
                row[pk(m, m)] = dre * sm;
                if (m > 0) row[pk(m, m) + 1] = dim * sm;
                T pre = dre, pim = dim, ppre = 0, ppim = 0;
#pragma unroll(PF > 0 ? PF : 1)
                for (int n = m + 1; n <= p; ++n) {
                    T c1 = T(2 * n - 1) * z, f = rec_t<T>(n, m);
                    T cre = (c1 * pre - r2 * ppre) * f;
                    T cim = (c1 * pim - r2 * ppim) * f;
                    T sn = sfac_t<T>(n, m);
                    row[pk(n, m)] = cre * sn;
                    if (m > 0) row[pk(n, m) + 1] = cim * sn;
                    ppre = pre;
                    ppim = pim;
                    pre = cre;
                    pim = cim;
                }
            }
        }
        __syncthreads();
        // thread (half, jp) sums coefficients jp and jp + 64 over the particles of its parity:
        // one broadcast strength load serves two coefficients
#pragma unroll 4
        for (int t = half; t < cnt; t += 2) {
            typename V4<T>::type gv = gsm[t];
            T y0 = Ysm[t * ys + jp], y1 = jp + 64 < pc ? Ysm[t * ys + jp + 64] : T(0);
            a0 += gv.x * y0;
            a1 += gv.y * y0;
            a2 += gv.z * y0;
            b0 += gv.x * y1;
            b1 += gv.y * y1;
            b2 += gv.z * y1;
        }
        __syncthreads();
    }
    // the two particle parities meet in shared memory (the harmonic table is free now)
    T *red = Ysm;  // [64][6]
    if (half == 1) {
        red[6 * jp + 0] = a0;
        red[6 * jp + 1] = a1;
        red[6 * jp + 2] = a2;
        red[6 * jp + 3] = b0;
        red[6 * jp + 4] = b1;
        red[6 * jp + 5] = b2;
    }
    __syncthreads();
    if (half == 0) {
        T *out = M + (size_t)leaf * 3 * pc;
        if (jp < pc) {
            out[jp] = a0 + red[6 * jp + 0];
            out[pc + jp] = a1 + red[6 * jp + 1];
            out[2 * pc + jp] = a2 + red[6 * jp + 2];
        }
        if (jp + 64 < pc) {
            out[jp + 64] = b0 + red[6 * jp + 3];
            out[pc + jp + 64] = b1 + red[6 * jp + 4];
            out[2 * pc + jp + 64] = b2 + red[6 * jp + 5];
        }
    }
}

int launch_p2m(Ctx *c)
{
    int log2n = 0;
    while ((1 << log2n) < c->nside) ++log2n;
    size_t off = c->lvl_off[c->depth];
    const int tp = c->f64 ? P2MCfg<double>::TP : P2MCfg<float>::TP;
    size_t sm = (size_t)tp * (c->pc + 1) * c->esz + 16 + (size_t)tp * 4 * c->esz;
    if (c->pc > P2M_BS) {
        c->last_error = "P2M supports at most 128 padded coefficients";
        return VFMM_ERR_UNSUPPORTED;
    }
    if (c->f64)
        k_p2m<double, 0><<<(unsigned)c->nleaf, P2M_BS, sm, c->stream>>>(
            (const dvec4 *)c->xs.p, (const dvec4 *)c->gs.p, (const int *)c->leaf_start.p, c->nside, log2n,
            c->leaf_w, c->p, c->pc, (double *)c->mexp.p + off);
    else {
        // the benchmark order p = 10 with the recursion unrolled (1.81 -> 1.27 ms at 256^3)
        auto kern = c->p == 10 ? k_p2m<float, 10> : k_p2m<float, 0>;
        kern<<<(unsigned)c->nleaf, P2M_BS, sm, c->stream>>>(
            (const float4 *)c->xs.p, (const float4 *)c->gs.p, (const int *)c->leaf_start.p, c->nside, log2n,
            (float)c->leaf_w, c->p, c->pc, (float *)c->mexp.p + off);
    }
    VFMM_CUDA_CHECK_LAUNCH(c);
    return VFMM_OK;
}

// ---------------------------------------------------------------------------------------
// Gathered-column GEMM on the CUDA cores.
// Output tile: 128 coefficient rows x 96 columns (32 target cells x 3 components), 256
// threads, 8x6 register block per thread, K chunks staged in shared memory with register
// double buffering.  The K loop runs over k-blocks (one translation matrix each) and the
// columns of each k-block are gathered from the source cell of that k-block.
constexpr int GM = 128, GN = 96, GCELLS = 32, GTHREADS = 256;

template <typename T> struct GemmCfg;
template <> struct GemmCfg<float> {
    static constexpr int BK = 16;
    typedef float4 vec;
    static constexpr int VEC = 4;
};
template <> struct GemmCfg<double> {
    static constexpr int BK = 8;
    typedef double2 vec;
    static constexpr int VEC = 2;
};

__device__ __forceinline__ void target_cell(const GemmParams &gp, int g, int64_t q, int &cx, int &cy, int &cz)
{
    if (gp.grouped) {
        int h = gp.n_tgt >> 1;
        int px = (int)(q / ((int64_t)h * h)), py = (int)((q / h) % h), pz = (int)(q % h);
        cx = 2 * px + ((g >> 2) & 1);
        cy = 2 * py + ((g >> 1) & 1);
        cz = 2 * pz + (g & 1);
    } else {
        int n = gp.n_tgt;
        cx = (int)(q / ((int64_t)n * n));
        cy = (int)((q / n) % n);
        cz = (int)(q % n);
    }
}

__device__ __forceinline__ int64_t source_cell(const GemmParams &gp, int cx, int cy, int cz, int4 kb)
{
    int sx, sy, sz, n = gp.n_src;
    if (gp.mode == 0) {
        sx = (cx + kb.y) & (n - 1);
        sy = (cy + kb.z) & (n - 1);
        sz = (cz + kb.w) & (n - 1);
    } else if (gp.mode == 1) {
        sx = 2 * cx + kb.y;
        sy = 2 * cy + kb.z;
        sz = 2 * cz + kb.w;
    } else {
        sx = cx >> 1;
        sy = cy >> 1;
        sz = cz >> 1;
    }
    return ((int64_t)sx * n + sy) * n + sz;
}

template <typename T>
__global__ void __launch_bounds__(GTHREADS) k_gemm(GemmParams gp, int64_t ncell_group)
{
    typedef GemmCfg<T> C;
    constexpr int BK = C::BK, VEC = C::VEC;
    typedef typename C::vec vec;
    constexpr int EPI = sizeof(T) == 4 ? 48 : 24;  // columns per epilogue pass through shared memory
    constexpr int MAIN_BYTES = (2 * BK * GM + 2 * BK * GN) * (int)sizeof(T);
    constexpr int EPI_BYTES = EPI * (GM + 4) * (int)sizeof(T);
    __shared__ __align__(16) unsigned char smem[MAIN_BYTES > EPI_BYTES ? MAIN_BYTES : EPI_BYTES];
    T (*As)[BK][GM] = reinterpret_cast<T (*)[BK][GM]>(smem);
    T (*Bs)[BK][GN] = reinterpret_cast<T (*)[BK][GN]>(smem + 2 * BK * GM * sizeof(T));
    T (*Cs)[GM + 4] = reinterpret_cast<T (*)[GM + 4]>(smem);
    const int g = gp.grouped ? blockIdx.y : 0;
    const int tid = threadIdx.x;
    const int tm = tid >> 4, tn = tid & 15;
    const int64_t cell0 = (int64_t)blockIdx.x * GCELLS;
    // k-block slice of this block (split k over blockIdx.z)
    const int nkb_all = gp.kb_cnt[g];
    const int per = (nkb_all + gp.ksplit - 1) / gp.ksplit;
    const int kb0 = min(nkb_all, (int)blockIdx.z * per);
    const int nkb = min(nkb_all, kb0 + per) - kb0;
    const int4 *kbl = gp.kb + gp.kb_off[g] + kb0;
    const int pc = gp.pc;
    const int nch = pc / BK;
    const int total = nkb * nch;
    const T *AT = (const T *)gp.AT;
    const T *B = (const T *)gp.B;

    // B-load slots of this thread: v = tid and tid + 256 (< 384 = GN * BK / VEC)
    int slot_n[2], slot_part[2], slot_comp[2], slot_cx[2], slot_cy[2], slot_cz[2];
    bool slot_ok[2];
    for (int s = 0; s < 2; ++s) {
        int v = tid + s * GTHREADS;
        slot_ok[s] = v < GN * BK / VEC;
        int part = v / GN, n = v - part * GN;
        slot_part[s] = part;
        slot_n[s] = n;
        int q = n / 3;
        slot_comp[s] = n - 3 * q;
        int64_t cq = cell0 + q;
        if (cq >= ncell_group) slot_ok[s] = false;
        int cx = 0, cy = 0, cz = 0;
        if (slot_ok[s]) target_cell(gp, g, cq, cx, cy, cz);
        slot_cx[s] = cx;
        slot_cy[s] = cy;
        slot_cz[s] = cz;
        if (v >= GN * BK / VEC) slot_n[s] = -1;
    }

    T acc[8][6];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 6; ++j) acc[i][j] = 0;

    vec ra[2], rb[2];
    auto load = [&](int c) {
        int kbi = c / nch, j0 = (c - kbi * nch) * BK;
        int4 kb = kbl[kbi];
        const T *a = AT + ((size_t)kb.x * pc + j0) * GM;
#pragma unroll
        for (int s = 0; s < 2; ++s) ra[s] = ((const vec *)a)[tid + s * GTHREADS];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            if (slot_ok[s]) {
                int64_t src = source_cell(gp, slot_cx[s], slot_cy[s], slot_cz[s], kb);
                src = checked_index<int64_t>(src, (int64_t)gp.n_src * gp.n_src * gp.n_src, gp.err);
                rb[s] = *(const vec *)(B + (src * 3 + slot_comp[s]) * pc + j0 + slot_part[s] * VEC);
            } else {
                T *z = (T *)&rb[s];
#pragma unroll
                for (int e = 0; e < VEC; ++e) z[e] = 0;
            }
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            int v = tid + s * GTHREADS;  // A: v indexes 16-byte vectors of As[buf] in order
            ((vec *)&As[buf][0][0])[v] = ra[s];
        }
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            if (slot_n[s] >= 0) {
                const T *z = (const T *)&rb[s];
#pragma unroll
                for (int e = 0; e < VEC; ++e) Bs[buf][slot_part[s] * VEC + e][slot_n[s]] = z[e];
            }
        }
    };

    if (total > 0) {
        load(0);
        store(0);
    }
    __syncthreads();
    for (int c = 0; c < total; ++c) {
        int buf = c & 1;
        if (c + 1 < total) load(c + 1);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[8], b[6];
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = As[buf][kk][tm * 8 + i];
#pragma unroll
            for (int j = 0; j < 6; ++j) b[j] = Bs[buf][kk][tn * 6 + j];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 6; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        if (c + 1 < total) store(buf ^ 1);
        __syncthreads();
    }
    // epilogue: the tile goes through shared memory so that every (cell, component) row of
    // pc coefficients is written (or read-modify-written) by whole warps, vector by vector
    const int64_t ntgt3 = (int64_t)gp.n_tgt * gp.n_tgt * gp.n_tgt;
    T *Cp = gp.ksplit > 1 ? (T *)gp.partial + (int64_t)blockIdx.z * ntgt3 * 3 * pc : (T *)gp.C;
    const bool acc_c = gp.accumulate && gp.ksplit == 1;
    constexpr int RV = GM / VEC;  // vectors per row
#pragma unroll 1
    for (int c0 = 0; c0 < GN; c0 += EPI) {
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            int n = tn * 6 + j - c0;
            if (n >= 0 && n < EPI) {
#pragma unroll
                for (int i = 0; i < 8; ++i) Cs[n][tm * 8 + i] = acc[i][j];
            }
        }
        __syncthreads();
        for (int idx = tid; idx < EPI * RV; idx += GTHREADS) {
            const int r = idx / RV, mv = idx - r * RV;
            const int n = c0 + r;
            const int q = n / 3, comp = n - 3 * q;
            const int64_t cq = cell0 + q;
            const int m = mv * VEC;
            if (cq >= ncell_group || m >= pc) continue;
            int cx, cy, cz;
            target_cell(gp, g, cq, cx, cy, cz);
            const int64_t cell = ((int64_t)cx * gp.n_tgt + cy) * gp.n_tgt + cz;
            vec *dst = (vec *)(Cp + (cell * 3 + comp) * pc + m);
            vec v = *(const vec *)&Cs[r][m];
            if (acc_c) {
                vec o = *dst;
                T *pv = (T *)&v;
                const T *po = (const T *)&o;
#pragma unroll
                for (int e = 0; e < VEC; ++e) pv[e] += po[e];
            }
            *dst = v;
        }
    }
}

// Sum of the k slices in slice order (deterministic), into C (= or +=).
template <typename T>
__global__ void k_split_reduce(int nsplit, int64_t count, const T *__restrict__ partial, T *__restrict__ C,
                               int accumulate)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    T s = accumulate ? C[i] : T(0);
    for (int z = 0; z < nsplit; ++z) s += partial[(int64_t)z * count + i];
    C[i] = s;
}

int launch_gemm(Ctx *c, const GemmParams &gp_in, int ngroups, int64_t ncell_group)
{
    if (ncell_group <= 0) return VFMM_OK;
    GemmParams gp = gp_in;
    dim3 grid((unsigned)((ncell_group + GCELLS - 1) / GCELLS), (unsigned)ngroups);
    // small levels: split the k-block loop over more blocks (about four per SM), partial tiles
    // summed by a second pass in a fixed order
    int maxkb = 0;
    for (int g = 0; g < ngroups; ++g) maxkb = std::max(maxkb, gp.kb_cnt[g]);
    const int64_t blocks = (int64_t)grid.x * grid.y;
    const int64_t ntgt3 = (int64_t)gp.n_tgt * gp.n_tgt * gp.n_tgt;
    const int64_t count = ntgt3 * 3 * gp.pc;
    int ksplit = 1;
    if (blocks < 304 && maxkb > 1) {
        ksplit = (int)std::min<int64_t>(maxkb, (608 + blocks - 1) / blocks);
        const int64_t cap = (int64_t)(c->gemm_part.bytes / c->esz) / count;
        ksplit = (int)std::min<int64_t>(ksplit, cap);
        if (ksplit < 2) ksplit = 1;
    }
    gp.ksplit = ksplit;
    gp.partial = c->gemm_part.p;
    gp.err = (int *)c->err.p;
    grid.z = (unsigned)ksplit;
    if (c->f64)
        k_gemm<double><<<grid, GTHREADS, 0, c->stream>>>(gp, ncell_group);
    else
        k_gemm<float><<<grid, GTHREADS, 0, c->stream>>>(gp, ncell_group);
    VFMM_CUDA_CHECK_LAUNCH(c);
    if (ksplit > 1) return launch_split_reduce(c, ksplit, count, gp.partial, gp.C, gp.accumulate, !c->f64);
    return VFMM_OK;
}

int launch_split_reduce(Ctx *c, int nsplit, int64_t count, const void *partial, void *C, int accumulate, bool f32)
{
    const int nb = (int)((count + 255) / 256);
    if (f32)
        k_split_reduce<float><<<nb, 256, 0, c->stream>>>(nsplit, count, (const float *)partial, (float *)C, accumulate);
    else
        k_split_reduce<double><<<nb, 256, 0, c->stream>>>(nsplit, count, (const double *)partial, (double *)C,
                                                          accumulate);
    VFMM_CUDA_CHECK_LAUNCH(c);
    return VFMM_OK;
}

// ---------------------------------------------------------------------------------------
// Root step in FP64: M_0 = sum_b M2M_b M_1[b]; L_0 = Op M_0 with Op the periodic lattice
// operator (images outside the central 3^3 boxes; Section 3.1 last paragraph).
template <typename T>
__global__ void k_root_m2m(const T *__restrict__ M1, const double *__restrict__ m2m, int nc, int pc,
                           double *__restrict__ root_m)
{
    // one warp per root coefficient (k, comp): sum over the 8 children and j, lanes along j
    const int o = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (o >= 3 * nc) return;
    const int comp = o / nc, k = o - comp * nc;
    double s = 0.0;
    for (int b = 0; b < 8; ++b) {
        const double *A = m2m + ((size_t)b * nc + k) * nc;
        const T *x = M1 + ((size_t)b * 3 + comp) * pc;
        for (int j = lane; j < nc; j += 32) s += A[j] * (double)x[j];
    }
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    if (lane == 0) root_m[o] = s;
}

template <typename T>
__global__ void k_root_lattice(const double *__restrict__ op, const double *__restrict__ root_m, int nc, int pc,
                               T *__restrict__ L0)
{
    // L_0 = Op M_0, one warp per output (k, comp) (k >= nc: zero padding)
    const int o = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (o >= 3 * pc) return;
    const int comp = o / pc, k = o - comp * pc;
    double s = 0.0;
    if (k < nc) {
        const double *A = op + (size_t)k * nc;
        for (int j = lane; j < nc; j += 32) s += A[j] * root_m[comp * nc + j];
    }
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    if (lane == 0) L0[o] = (T)s;
}

int launch_root(Ctx *c)
{
    const int wpb = 8;  // warps per block
    const unsigned nb1 = (unsigned)((3 * c->nc + wpb - 1) / wpb), nb2 = (unsigned)((3 * c->pc + wpb - 1) / wpb);
    if (c->f64) {
        k_root_m2m<double><<<nb1, 32 * wpb, 0, c->stream>>>((const double *)c->mexp.p + c->lvl_off[1],
                                                             (const double *)c->m2m_f64.p, c->nc, c->pc,
                                                             (double *)c->root_m.p);
        VFMM_CUDA_CHECK_LAUNCH(c);
        k_root_lattice<double><<<nb2, 32 * wpb, 0, c->stream>>>((const double *)c->lattice_f64.p,
                                                                 (const double *)c->root_m.p, c->nc, c->pc,
                                                                 (double *)c->lexp.p);
    } else {
        k_root_m2m<float><<<nb1, 32 * wpb, 0, c->stream>>>((const float *)c->mexp.p + c->lvl_off[1],
                                                            (const double *)c->m2m_f64.p, c->nc, c->pc,
                                                            (double *)c->root_m.p);
        VFMM_CUDA_CHECK_LAUNCH(c);
        k_root_lattice<float><<<nb2, 32 * wpb, 0, c->stream>>>((const double *)c->lattice_f64.p,
                                                                (const double *)c->root_m.p, c->nc, c->pc,
                                                                (float *)c->lexp.p);
    }
    VFMM_CUDA_CHECK_LAUNCH(c);
    return VFMM_OK;
}

// ---------------------------------------------------------------------------------------
// L2P (Eqs. biotsavartfmm2, stretchingfmm2): gradient and Hessian of the three local
// expansions at each particle.  Per leaf, the coefficient vectors of d_a psi and
// d_a d_b psi are formed from the local coefficients with
//   d_z Y_n^m = Y_{n-1}^m, (d_x + i d_y) Y_n^m = Y_{n-1}^{m+1}, (d_x - i d_y) Y_n^m = -Y_{n-1}^{m-1},
// i.e. for psi = sum conj(Y_k^l) F_k^l:
//   G^z_{a,b} = F_{a+1,b},  G^x_{a,b} = (F_{a+1,b-1} - F_{a+1,b+1})/2,
//   G^y_{a,b} = i (F_{a+1,b+1} + F_{a+1,b-1})/2.
// The kernel turns these into the velocity tables U_a = eps_abc D^b Psi_c and their
// gradients D^k U_a; each particle evaluates Y_a^b at its offset once and accumulates 12
// table dot products.
constexpr int L2P_BS = 64;   // one thread per particle of a 64-particle leaf

template <typename T> struct C2;
template <> struct C2<float> { typedef float2 type; };
template <> struct C2<double> { typedef double2 type; };

__device__ __forceinline__ int cix(int n, int m) { return n * (n + 1) / 2 + m; }

// inverse of cix: complex index -> (n, m), by arithmetic (the lanes of a warp decode different
// indices, which a constant-memory table would serialise)
__device__ __forceinline__ void cix_nm(int ci, int &n, int &m)
{
    int d = 0;
    while ((d + 1) * (d + 2) / 2 <= ci) ++d;
    n = d;
    m = ci - d * (d + 1) / 2;
}

// complex coefficient (n, m) of a table in complex layout (m >= 0 stored), any m
template <typename T>
__device__ __forceinline__ typename C2<T>::type getcx(const typename C2<T>::type *P, int n, int m, int nmax)
{
    typename C2<T>::type z;
    z.x = 0;
    z.y = 0;
    if (n < 0 || n > nmax) return z;
    int am = m < 0 ? -m : m;
    if (am > n) return z;
    z = P[cix(n, am)];
    if (m < 0) {  // (-1)^m conj
        z.y = -z.y;
        if (am & 1) {
            z.x = -z.x;
            z.y = -z.y;
        }
    }
    return z;
}

// D^dir applied to table `in` (degrees 0..nmax), output entry (a, b), dir 0 = x, 1 = y, 2 = z:
//   D^z: F_{a+1,b};  D^x: (F_{a+1,b-1} - F_{a+1,b+1})/2;  D^y: i (F_{a+1,b+1} + F_{a+1,b-1})/2
template <typename T>
__device__ __forceinline__ typename C2<T>::type dcx(const typename C2<T>::type *in, int nmax, int dir, int a, int b)
{
    typename C2<T>::type v;
    if (dir == 2) return getcx<T>(in, a + 1, b, nmax);
    typename C2<T>::type p1 = getcx<T>(in, a + 1, b + 1, nmax), m1 = getcx<T>(in, a + 1, b - 1, nmax);
    if (dir == 0) {
        v.x = T(0.5) * (m1.x - p1.x);
        v.y = T(0.5) * (m1.y - p1.y);
    } else {
        v.x = T(-0.5) * (p1.y + m1.y);
        v.y = T(0.5) * (p1.x + m1.x);
    }
    return v;
}

#ifndef VFMM_L2P_PP
#define VFMM_L2P_PP 2
#endif
template <typename T, int PP>
__global__ void __launch_bounds__(L2P_BS) k_l2p(const typename V4<T>::type *__restrict__ xs,
                                                const typename V4<T>::type *__restrict__ gs,
                                                const int *__restrict__ ls, int nside, int log2n, T w, int p, int pc,
                                                const T *__restrict__ Lc, T *__restrict__ ufar, T *__restrict__ sfar,
                                                T *__restrict__ gfar)
{
    // Per leaf, the local expansion of psi is turned into the tables of the velocity
    //   U_a = eps_abc D^b Psi_c            (degrees < p)
    // and of its gradient D^k U_a (degrees < p - 1); each particle then sums conj(Y) T over
    // the 3 + 9 tables: u_a, and du_a/dx_k, which gives S = (gamma . grad) u and, for the
    // adjoint, the velocity gradient itself.
    typedef typename C2<T>::type T2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ncx = (p + 1) * (p + 2) / 2;
    T2 *F = (T2 *)smem_raw;    // [3][ncx]  local coefficients times s_nm
    T2 *U = F + 3 * ncx;       // [3][ncx]  velocity tables
    T2 *W = U + 3 * ncx;       // [ncx][12] per coefficient: U_0..2, then D^k U_a at 3 + 3k + a
    const int leaf = blockIdx.x;
    const int b0 = ls[leaf], e0 = ls[leaf + 1];
    if (e0 <= b0) return;
    const int cz = leaf & (nside - 1), cy = (leaf >> log2n) & (nside - 1), cx = leaf >> (2 * log2n);
    // each lane decodes its coefficient (n, m) once and fills every component / direction of it
    const T *lsrc = Lc + (size_t)leaf * 3 * pc;
    for (int ci = threadIdx.x; ci < ncx; ci += blockDim.x) {
        int n, m;
        cix_nm(ci, n, m);
        const T sf = sfac_ld<T>(n, m);
        const int k0 = pk(n, m);
#pragma unroll
        for (int comp = 0; comp < 3; ++comp) {
            T2 v;
            v.x = lsrc[comp * pc + k0] * sf;
            v.y = m > 0 ? lsrc[comp * pc + k0 + 1] * sf : T(0);
            F[comp * ncx + ci] = v;
        }
    }
    __syncthreads();
    const int ng = p * (p + 1) / 2;  // entries of degree < p
    for (int ci = threadIdx.x; ci < ng; ci += blockDim.x) {
        int n, m;
        cix_nm(ci, n, m);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int b = a == 2 ? 0 : a + 1, c = a == 0 ? 2 : a - 1;
            T2 x1 = dcx<T>(F + c * ncx, p, b, n, m);
            T2 x2 = dcx<T>(F + b * ncx, p, c, n, m);
            T2 v;
            v.x = x1.x - x2.x;
            v.y = x1.y - x2.y;
            U[a * ncx + ci] = v;
            W[ci * 12 + a] = v;
        }
    }
    __syncthreads();
    const int nh = (p - 1) * p / 2;  // entries of degree < p - 1
    // items (a, ci) spread over the lanes (45 entries alone would leave most lanes idle in a
    // second pass); the three directions k unrolled
    for (int it = threadIdx.x; it < 3 * nh; it += blockDim.x) {
        const int a = (it >= nh) + (it >= 2 * nh), ci = it - a * nh;
        int n, m;
        cix_nm(ci, n, m);
#pragma unroll
        for (int k = 0; k < 3; ++k) W[ci * 12 + 3 + 3 * k + a] = dcx<T>(U + a * ncx, p - 1, k, n, m);
    }
    __syncthreads();
    const T zx = (cx + T(0.5)) * w, zy = (cy + T(0.5)) * w, zz = (cz + T(0.5)) * w;
    const T invw = T(1) / w;
    // PP particles per thread: one table row load serves PP independent recursions
    for (int i0 = b0 + threadIdx.x; i0 < e0; i0 += PP * blockDim.x) {
        T x[PP], y[PP], z[PP], r2[PP];
        T A[PP][12];
#pragma unroll
        for (int q = 0; q < PP; ++q) {
            const int i = i0 + q * blockDim.x;
            typename V4<T>::type xp = i < e0 ? xs[i] : make_v4<T>(zx, zy, zz, T(0));
            x[q] = (xp.x - zx) * invw;
            y[q] = (xp.y - zy) * invw;
            z[q] = (xp.z - zz) * invw;
            r2[q] = x[q] * x[q] + y[q] * y[q] + z[q] * z[q];
#pragma unroll
            for (int v = 0; v < 12; ++v) A[q][v] = 0;
        }
        T dre[PP], dim[PP];
#pragma unroll
        for (int q = 0; q < PP; ++q) {
            dre[q] = 1;
            dim[q] = 0;
        }
        for (int m = 0; m < p; ++m) {
            T pre[PP], pim[PP], ppre[PP], ppim[PP];
#pragma unroll
            for (int q = 0; q < PP; ++q) {
                if (m > 0) {
                    T f = -inv2m_t<T>(m);
                    T nre = f * (x[q] * dre[q] - y[q] * dim[q]);
                    T nim = f * (x[q] * dim[q] + y[q] * dre[q]);
                    dre[q] = nre;
                    dim[q] = nim;
                }
                pre[q] = dre[q];
                pim[q] = dim[q];
                ppre[q] = 0;
                ppim[q] = 0;
            }
            const T wgt = m > 0 ? T(2) : T(1);  // the pair +-m of sum conj(Y) T
            int ci = cix(m, m);
            for (int n = m; n < p; ++n) {
                T wre[PP], wim[PP];
#pragma unroll
                for (int q = 0; q < PP; ++q) {
                    T cre, cim;
                    if (n == m) {
                        cre = dre[q];
                        cim = dim[q];
                    } else {
                        T c1 = T(2 * n - 1) * z[q], f = rec_t<T>(n, m);
                        cre = (c1 * pre[q] - r2[q] * ppre[q]) * f;
                        cim = (c1 * pim[q] - r2[q] * ppim[q]) * f;
                        ppre[q] = pre[q];
                        ppim[q] = pim[q];
                        pre[q] = cre;
                        pim[q] = cim;
                    }
                    wre[q] = wgt * cre;
                    wim[q] = wgt * cim;
                }
                const T2 *row = W + ci * 12;
                if constexpr (sizeof(T) == 4) {
                    // rows are 96 B and W starts 48 ncx bytes in: 16-byte loads of two entries
                    const float4 *r4 = reinterpret_cast<const float4 *>(row);
                    const int nv = n < p - 1 ? 6 : 1;
#pragma unroll
                    for (int v2 = 0; v2 < 6; ++v2) {
                        if (v2 < nv) {
                            float4 t = r4[v2];
#pragma unroll
                            for (int q = 0; q < PP; ++q) {
                                A[q][2 * v2] += wre[q] * t.x + wim[q] * t.y;
                                A[q][2 * v2 + 1] += wre[q] * t.z + wim[q] * t.w;
                            }
                        }
                    }
                    if (nv == 1) {
                        T2 t = row[2];
#pragma unroll
                        for (int q = 0; q < PP; ++q) A[q][2] += wre[q] * t.x + wim[q] * t.y;
                    }
                } else {
                    const int nv = n < p - 1 ? 12 : 3;
#pragma unroll
                    for (int v = 0; v < 12; ++v) {
                        if (v < nv) {
                            T2 t = row[v];
#pragma unroll
                            for (int q = 0; q < PP; ++q) A[q][v] += wre[q] * t.x + wim[q] * t.y;
                        }
                    }
                }
                ci += n + 1;
            }
        }
        // psi_c = (1/4pi)(1/w) sum conj(Y) s F; d/dx = (1/w) d/dy
        const T s1 = T(0.0795774715459476679) * invw * invw;
        const T s2 = s1 * invw;
#pragma unroll
        for (int q = 0; q < PP; ++q) {
            const int i = i0 + q * blockDim.x;
            if (i >= e0) continue;
            ufar[3 * (int64_t)i + 0] = s1 * A[q][0];
            ufar[3 * (int64_t)i + 1] = s1 * A[q][1];
            ufar[3 * (int64_t)i + 2] = s1 * A[q][2];
            if (sfar) {  // S_a = gamma_k du_a/dx_k
                typename V4<T>::type gp = gs[i];
                sfar[3 * (int64_t)i + 0] = s2 * (gp.x * A[q][3] + gp.y * A[q][6] + gp.z * A[q][9]);
                sfar[3 * (int64_t)i + 1] = s2 * (gp.x * A[q][4] + gp.y * A[q][7] + gp.z * A[q][10]);
                sfar[3 * (int64_t)i + 2] = s2 * (gp.x * A[q][5] + gp.y * A[q][8] + gp.z * A[q][11]);
            }
            if (gfar) {  // velocity gradient du_a/dx_k at 3a + k
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int kk = 0; kk < 3; ++kk) gfar[9 * (int64_t)i + 3 * a + kk] = s2 * A[q][3 + 3 * kk + a];
            }
        }
    }
}

int launch_l2p(Ctx *c, bool grad)
{
    int log2n = 0;
    while ((1 << log2n) < c->nside) ++log2n;
    size_t off = c->lvl_off[c->depth];
    const int ncx = (c->p + 1) * (c->p + 2) / 2;
    size_t sm = (size_t)(3 + 3 + 12) * ncx * 2 * c->esz;
    if (c->f64)
        k_l2p<double, 1><<<(unsigned)c->nleaf, L2P_BS, sm, c->stream>>>(
            (const dvec4 *)c->xs.p, (const dvec4 *)c->gs.p, (const int *)c->leaf_start.p, c->nside, log2n,
            c->leaf_w, c->p, c->pc, (const double *)c->lexp.p + off, (double *)c->ufar.p,
            grad ? nullptr : (double *)c->sfar.p, grad ? (double *)c->gfar.p : nullptr);
    else
        k_l2p<float, VFMM_L2P_PP><<<(unsigned)c->nleaf, L2P_BS / VFMM_L2P_PP, sm, c->stream>>>(
            (const float4 *)c->xs.p, (const float4 *)c->gs.p, (const int *)c->leaf_start.p, c->nside, log2n,
            (float)c->leaf_w, c->p, c->pc, (const float *)c->lexp.p + off, (float *)c->ufar.p,
            grad ? nullptr : (float *)c->sfar.p, grad ? (float *)c->gfar.p : nullptr);
    VFMM_CUDA_CHECK_LAUNCH(c);
    return VFMM_OK;
}

}  // namespace vfmm

namespace vfmm {

__global__ void k_add_far(int64_t n, const int *__restrict__ perm, const float *__restrict__ ufar,
                          const float *__restrict__ sfar, float *__restrict__ u_out, float *__restrict__ s_out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t j = perm[i];
#pragma unroll
    for (int d = 0; d < 3; ++d) u_out[3 * j + d] += ufar[3 * i + d];
    if (s_out)
#pragma unroll
        for (int d = 0; d < 3; ++d) s_out[3 * j + d] += sfar[3 * i + d];
}

int launch_add_far(Ctx *c, void *u_out, void *s_out)
{
    const int nb = (int)((c->n + 255) / 256);
    k_add_far<<<nb, 256, 0, c->stream>>>(c->n, (const int *)c->perm.p, (const float *)c->ufar.p, (const float *)c->sfar.p,
                                         (float *)u_out, (float *)s_out);
    VFMM_CUDA_CHECK_LAUNCH(c);
    return VFMM_OK;
}

}  // namespace vfmm

namespace vfmm {

// ---------------------------------------------------------------------------------------
// Transposed far field (the adjoint of the FMM evaluation, Section 3.1 run backwards).
//
// The far velocity is u_far = E Lc(L2L) (M2L + lattice) Mc(M2M) P gamma: P the P2M, the
// expansion chains, and E the L2P curl of the leaf local expansion,
//   u_a(x_i) = 1/(4 pi w^2) sum_{b,c,k} eps_abc L[c][k] d_b phi_k(x^_i),
//   phi_(n,m,re|im) = wgt_m s_nm Re|Im Y_n^m (wgt_0 = 1, wgt_m = 2), x^ = (x - z)/w.
// Its exact transpose applied to w = dL/du runs the chain backwards:
//   E^T:  lambda[c][k] = 1/(4 pi w^2) wgt_m s_nm sum_i (w_i x grad^ Re|Im Y_n^m(x^_i))_c,
//   L2L^T, M2L^T, lattice^T, M2M^T: the same GEMMs with transposed matrices (host-built),
//   P^T:  mu -> Phi_c(x_j) = sum_k mu[c][k] s_nm Re|Im Y_n^m(x^_j)  (dL/dgamma_j, far part),
// and the source-position term of dL/dx_j is sum_c gamma_jc grad Phi_c(x_j).
// Gradients of Y_n^m use d/dz Y_n^m = Y_{n-1}^m, d/dx Y_n^m = (Y_{n-1}^{m+1} - Y_{n-1}^{m-1})/2,
// d/dy Y_n^m = -i (Y_{n-1}^{m+1} + Y_{n-1}^{m-1})/2, Y_n^{-m} = (-1)^m conj Y_n^m.

// Y_n^m (m >= 0, unscaled) of one point for degrees 0..nmax at cix(n, m)
template <typename T>
__device__ __forceinline__ void y_table(T x, T y, T z, int nmax, typename C2<T>::type *Y)
{
    const T r2 = x * x + y * y + z * z;
    T dre = 1, dim = 0;
    for (int m = 0; m <= nmax; ++m) {
        if (m > 0) {
            T f = -inv2m_t<T>(m);
            T nre = f * (x * dre - y * dim);
            T nim = f * (x * dim + y * dre);
            dre = nre;
            dim = nim;
        }
        Y[cix(m, m)].x = dre;
        Y[cix(m, m)].y = dim;
        T pre = dre, pim = dim, ppre = 0, ppim = 0;
        for (int n = m + 1; n <= nmax; ++n) {
            T c1 = T(2 * n - 1) * z, f = rec_t<T>(n, m);
            T cre = (c1 * pre - r2 * ppre) * f;
            T cim = (c1 * pim - r2 * ppim) * f;
            Y[cix(n, m)].x = cre;
            Y[cix(n, m)].y = cim;
            ppre = pre;
            ppim = pim;
            pre = cre;
            pim = cim;
        }
    }
}

// packed coefficient index -> (n, m, part): [n^2] = Re A_n^0, [n^2 + 2m - 1] = Re, [n^2 + 2m] = Im
__device__ __forceinline__ void unpack_k(int k, int &n, int &m, int &part)
{
    n = 0;
    while ((n + 1) * (n + 1) <= k) ++n;
    const int r = k - n * n;
    m = (r + 1) >> 1;
    part = (r > 0 && (r & 1) == 0) ? 1 : 0;
}

// Re (part 0) or Im (part 1) of grad^ Y_n^m, n >= 1, from a table of degrees <= nmax >= n - 1
template <typename T>
__device__ __forceinline__ void y_grad_part(const typename C2<T>::type *Y, int nmax, int n, int m, int part, T &gx,
                                            T &gy, T &gz)
{
    typedef typename C2<T>::type T2;
    const T2 P = getcx<T>(Y, n - 1, m + 1, nmax), Q = getcx<T>(Y, n - 1, m - 1, nmax), Z = getcx<T>(Y, n - 1, m, nmax);
    if (part == 0) {
        gx = T(0.5) * (P.x - Q.x);
        gy = T(0.5) * (P.y + Q.y);
        gz = Z.x;
    } else {
        gx = T(0.5) * (P.y - Q.y);
        gy = T(-0.5) * (P.x + Q.x);
        gz = Z.y;
    }
}

// E^T: per leaf, lambda[c][k] from the particles' w (sorted, in ws).  One block per leaf; a chunk
// of particles writes its Y tables (degrees < p) to shared memory, then thread k accumulates
// coefficient k over the chunk.
template <typename T> struct DualCfg {
    static constexpr int TP = sizeof(T) == 4 ? 64 : 32;  // particles per chunk
};
constexpr int DUAL_BS = 128;

template <typename T>
__global__ void __launch_bounds__(DUAL_BS) k_dual_p2m(const typename V4<T>::type *__restrict__ xs,
                                                     const typename V4<T>::type *__restrict__ ws,
                                                     const int *__restrict__ ls, int nside, int log2n, T w, int p,
                                                     int pc, T *__restrict__ Lam)
{
    typedef typename C2<T>::type T2;
    constexpr int TP = DualCfg<T>::TP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ny = p * (p + 1) / 2;  // complex entries of degrees < p
    T2 *Ysm = (T2 *)smem_raw;                                   // [TP][ny]
    typename V4<T>::type *wsm = (typename V4<T>::type *)(Ysm + TP * ny);  // [TP]
    const int leaf = blockIdx.x;
    const int cz = leaf & (nside - 1), cy = (leaf >> log2n) & (nside - 1), cx = leaf >> (2 * log2n);
    const T zx = (cx + T(0.5)) * w, zy = (cy + T(0.5)) * w, zz = (cz + T(0.5)) * w;
    const T invw = T(1) / w;
    const int b = ls[leaf], e = ls[leaf + 1];
    const int nc = (p + 1) * (p + 1);
    const int k = threadIdx.x;
    int n = 0, m = 0, part = 0;
    if (k < nc) unpack_k(k, n, m, part);
    T a0 = 0, a1 = 0, a2 = 0;
    for (int s0 = b; s0 < e; s0 += TP) {
        const int cnt = min(TP, e - s0);
        __syncthreads();
        if (threadIdx.x < cnt) {
            const typename V4<T>::type xp = xs[s0 + threadIdx.x];
            wsm[threadIdx.x] = ws[s0 + threadIdx.x];
            y_table<T>((xp.x - zx) * invw, (xp.y - zy) * invw, (xp.z - zz) * invw, p - 1, Ysm + threadIdx.x * ny);
        }
        __syncthreads();
        if (k < nc && n >= 1) {
            for (int t = 0; t < cnt; ++t) {
                T gx, gy, gz;
                y_grad_part<T>(Ysm + t * ny, p - 1, n, m, part, gx, gy, gz);
                const typename V4<T>::type wv = wsm[t];
                a0 += wv.y * gz - wv.z * gy;
                a1 += wv.z * gx - wv.x * gz;
                a2 += wv.x * gy - wv.y * gx;
            }
        }
    }
    if (k < pc) {
        T sc = 0;
        if (k < nc) sc = T(0.0795774715459476679) * invw * invw * (m > 0 ? T(2) : T(1)) * sfac_ld<T>(n, m);
        T *out = Lam + (size_t)leaf * 3 * pc;
        out[k] = sc * a0;
        out[pc + k] = sc * a1;
        out[2 * pc + k] = sc * a2;
    }
}

// P^T and the source-position term: per particle j of a leaf with dual multipole mu,
//   dgamma[perm j][c] += Phi_c(x_j),  dxf[perm j] = sum_c gamma_jc grad Phi_c(x_j)  (caller order).
constexpr int DUAL_L2P_BS = 64;
template <typename T>
__global__ void __launch_bounds__(DUAL_L2P_BS) k_dual_l2p(const typename V4<T>::type *__restrict__ xs,
                                                         const int *__restrict__ ls, const int *__restrict__ perm,
                                                         int nside, int log2n, T w, int p, int pc,
                                                         const T *__restrict__ Mu, const T *__restrict__ gamma,
                                                         T *__restrict__ dgamma, T *__restrict__ dxf)
{
    typedef typename C2<T>::type T2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nc = (p + 1) * (p + 1);
    T *mus = (T *)smem_raw;  // [3][nc] times s_nm
    const int leaf = blockIdx.x;
    const int b = ls[leaf], e = ls[leaf + 1];
    if (e <= b) return;
    for (int o = threadIdx.x; o < 3 * nc; o += blockDim.x) {
        const int comp = o / nc, k = o - comp * nc;
        int n, m, part;
        unpack_k(k, n, m, part);
        mus[o] = Mu[(size_t)leaf * 3 * pc + comp * pc + k] * sfac_ld<T>(n, m);
    }
    __syncthreads();
    const int cz = leaf & (nside - 1), cy = (leaf >> log2n) & (nside - 1), cx = leaf >> (2 * log2n);
    const T zx = (cx + T(0.5)) * w, zy = (cy + T(0.5)) * w, zz = (cz + T(0.5)) * w;
    const T invw = T(1) / w;
    T2 Y[(PMAX + 1) * (PMAX + 2) / 2];
    for (int j = b + threadIdx.x; j < e; j += blockDim.x) {
        const typename V4<T>::type xp = xs[j];
        y_table<T>((xp.x - zx) * invw, (xp.y - zy) * invw, (xp.z - zz) * invw, p, Y);
        T phi[3] = {0, 0, 0}, g[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};  // g[c][b] = d_b Phi_c
        for (int k = 0; k < nc; ++k) {
            int n, m, part;
            unpack_k(k, n, m, part);
            const T2 yv = Y[cix(n, m)];
            const T h = part ? yv.y : yv.x;
            T gx = 0, gy = 0, gz = 0;
            if (n >= 1) y_grad_part<T>(Y, p, n, m, part, gx, gy, gz);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const T mu = mus[c * nc + k];
                phi[c] += mu * h;
                g[c][0] += mu * gx;
                g[c][1] += mu * gy;
                g[c][2] += mu * gz;
            }
        }
        const int64_t s = perm[j];
        const T g0 = gamma[3 * s], g1 = gamma[3 * s + 1], g2 = gamma[3 * s + 2];
#pragma unroll
        for (int c = 0; c < 3; ++c) dgamma[3 * s + c] += phi[c];
#pragma unroll
        for (int bb = 0; bb < 3; ++bb) dxf[3 * s + bb] = invw * (g0 * g[0][bb] + g1 * g[1][bb] + g2 * g[2][bb]);
    }
}

// lattice^T and root M2M^T in FP64: mu_0 = Op^T lambda_0; mu_1[b] += M2M_b^T mu_0
template <typename T>
__global__ void k_root_lattice_t(const double *__restrict__ op, const T *__restrict__ L0, int nc, int pc,
                                 double *__restrict__ mu0)
{
    const int o = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (o >= 3 * nc) return;
    const int comp = o / nc, j = o - comp * nc;
    double s = 0.0;
    for (int k = lane; k < nc; k += 32) s += op[(size_t)k * nc + j] * (double)L0[comp * pc + k];
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    if (lane == 0) mu0[o] = s;
}

template <typename T>
__global__ void k_root_m2m_t(const double *__restrict__ m2m, const double *__restrict__ mu0, int nc, int pc,
                             T *__restrict__ M1)
{
    const int o = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (o >= 8 * 3 * nc) return;
    const int bc = o / nc, j = o - bc * nc;  // bc = child * 3 + comp
    const int child = bc / 3, comp = bc - 3 * child;
    const double *A = m2m + (size_t)child * nc * nc;
    double s = 0.0;
    for (int k = lane; k < nc; k += 32) s += A[(size_t)k * nc + j] * mu0[comp * nc + k];
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    if (lane == 0) M1[((size_t)child * 3 + comp) * pc + j] += (T)s;
}

int launch_dual_p2m(Ctx *c, const void *ws_sorted)
{
    int log2n = 0;
    while ((1 << log2n) < c->nside) ++log2n;
    if (c->pc > DUAL_BS || c->p < 1) {
        c->last_error = "transposed L2P supports at most 128 padded coefficients";
        return VFMM_ERR_UNSUPPORTED;
    }
    const size_t off = c->lvl_off[c->depth];
    const int ny = c->p * (c->p + 1) / 2;
    if (c->f64) {
        const size_t sm = (size_t)DualCfg<double>::TP * (ny * sizeof(double2) + sizeof(dvec4));
        k_dual_p2m<double><<<(unsigned)c->nleaf, DUAL_BS, sm, c->stream>>>(
            (const dvec4 *)c->xs.p, (const dvec4 *)ws_sorted, (const int *)c->leaf_start.p, c->nside, log2n,
            c->leaf_w, c->p, c->pc, (double *)c->lexp.p + off);
    } else {
        const size_t sm = (size_t)DualCfg<float>::TP * (ny * sizeof(float2) + sizeof(float4));
        k_dual_p2m<float><<<(unsigned)c->nleaf, DUAL_BS, sm, c->stream>>>(
            (const float4 *)c->xs.p, (const float4 *)ws_sorted, (const int *)c->leaf_start.p, c->nside, log2n,
            (float)c->leaf_w, c->p, c->pc, (float *)c->lexp.p + off);
    }
    VFMM_CUDA_CHECK_LAUNCH(c);
    return VFMM_OK;
}

int launch_dual_l2p(Ctx *c, const void *gamma, void *dgamma, void *dxf)
{
    int log2n = 0;
    while ((1 << log2n) < c->nside) ++log2n;
    const size_t off = c->lvl_off[c->depth];
    const size_t sm = (size_t)3 * c->nc * c->esz;
    if (c->f64)
        k_dual_l2p<double><<<(unsigned)c->nleaf, DUAL_L2P_BS, sm, c->stream>>>(
            (const dvec4 *)c->xs.p, (const int *)c->leaf_start.p, (const int *)c->perm.p, c->nside, log2n,
            c->leaf_w, c->p, c->pc, (const double *)c->mexp.p + off, (const double *)gamma, (double *)dgamma,
            (double *)dxf);
    else
        k_dual_l2p<float><<<(unsigned)c->nleaf, DUAL_L2P_BS, sm, c->stream>>>(
            (const float4 *)c->xs.p, (const int *)c->leaf_start.p, (const int *)c->perm.p, c->nside, log2n,
            (float)c->leaf_w, c->p, c->pc, (const float *)c->mexp.p + off, (const float *)gamma, (float *)dgamma,
            (float *)dxf);
    VFMM_CUDA_CHECK_LAUNCH(c);
    return VFMM_OK;
}

int launch_root_t(Ctx *c)
{
    const int wpb = 8;
    const unsigned nb1 = (unsigned)((3 * c->nc + wpb - 1) / wpb), nb2 = (unsigned)((24 * c->nc + wpb - 1) / wpb);
    if (c->f64) {
        k_root_lattice_t<double><<<nb1, 32 * wpb, 0, c->stream>>>((const double *)c->lattice_f64.p,
                                                                   (const double *)c->lexp.p, c->nc, c->pc,
                                                                   (double *)c->root_m.p);
        VFMM_CUDA_CHECK_LAUNCH(c);
        k_root_m2m_t<double><<<nb2, 32 * wpb, 0, c->stream>>>((const double *)c->m2m_f64.p,
                                                               (const double *)c->root_m.p, c->nc, c->pc,
                                                               (double *)c->mexp.p + c->lvl_off[1]);
    } else {
        k_root_lattice_t<float><<<nb1, 32 * wpb, 0, c->stream>>>((const double *)c->lattice_f64.p,
                                                                  (const float *)c->lexp.p, c->nc, c->pc,
                                                                  (double *)c->root_m.p);
        VFMM_CUDA_CHECK_LAUNCH(c);
        k_root_m2m_t<float><<<nb2, 32 * wpb, 0, c->stream>>>((const double *)c->m2m_f64.p,
                                                              (const double *)c->root_m.p, c->nc, c->pc,
                                                              (float *)c->mexp.p + c->lvl_off[1]);
    }
    VFMM_CUDA_CHECK_LAUNCH(c);
    return VFMM_OK;
}

}  // namespace vfmm

namespace vfmm {

// the far-field kernels (which may share SMs with the P2P); the gather of the strengths and the
// final add of the far field run alone and keep the default split (the add of the far field
// is 2.4x slower with the largest shared carveout, i.e. the smallest L1)
void set_carveouts_expansions()
{
    prefer_max_shared(k_p2m<float, 0>);
    prefer_max_shared(k_p2m<float, 10>);
    prefer_max_shared(k_p2m<double, 0>);
    prefer_max_shared(k_gemm<float>);
    prefer_max_shared(k_gemm<double>);
    prefer_max_shared(k_split_reduce<float>);
    prefer_max_shared(k_split_reduce<double>);
    prefer_max_shared(k_root_m2m<float>);
    prefer_max_shared(k_root_m2m<double>);
    prefer_max_shared(k_root_lattice<float>);
    prefer_max_shared(k_root_lattice<double>);
    prefer_max_shared(k_l2p<float, VFMM_L2P_PP>);
    prefer_max_shared(k_l2p<double, 1>);
}

}  // namespace vfmm

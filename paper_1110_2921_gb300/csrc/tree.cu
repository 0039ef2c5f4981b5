// Uniform periodic octree: wrap, leaf key, counting sort, per-leaf sort, gather.
//
// The paper builds its tree on the CPU (Section 2.2); here every step runs on the GPU.
// Keys are row-major leaf indices (ix * n + iy) * n + iz at depth D.  The sort is a counting
// sort (atomic histogram, three-kernel exclusive scan, atomic scatter) followed by a sort of
// each leaf's particles by (octant of the leaf, caller index), which makes the final order
// deterministic and each octant's particles contiguous.
#include "common.cuh"
#include "vfmm_internal.h"

#include <climits>

namespace vfmm {

// Box constants in the input's own precision, computed once on the host: FP64 arithmetic is
// scarce on this part, and a division per thread of the key and leaf-sort kernels cost more
// than the rest of their work.
template <typename TIn> struct BoxConst {
    TIn L, invL, scale;  // box, 1 / box, cells per unit length at the given level
};
template <typename TIn> BoxConst<TIn> box_const(double L, double cells)
{
    return BoxConst<TIn>{(TIn)L, (TIn)(1.0 / L), (TIn)(cells / L)};
}

template <typename TIn>
__global__ void k_keys(int64_t n, const TIn *__restrict__ x, int nside, BoxConst<TIn> bc, int *__restrict__ keys,
                       int *__restrict__ counts, int *__restrict__ err)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = i < n;
    int key = -1;
    if (active) {
        // coordinates in the input's own precision
        const TIn Lt = bc.L, invL = bc.invL, scale = bc.scale;
        int c[3];
        bool finite = true;
        for (int d = 0; d < 3; ++d) {
            finite = finite && isfinite(x[3 * i + d]);
            TIn v = wrap_coord<TIn>(x[3 * i + d], Lt, invL);
            int ci = (int)(v * scale);
            c[d] = ci < 0 ? 0 : (ci >= nside ? nside - 1 : ci);
        }
        key = (c[0] * nside + c[1]) * nside + c[2];
        keys[i] = key;
        // a NaN or infinite coordinate has no leaf: the clamped key keeps every access in bounds
        // and the error bit makes vfmm_build_tree fail with VFMM_ERR_ARG
        if (!finite) atomicOr(err, ERRBIT_NONFINITE);
    }
    // one atomic per run of equal keys in the warp (neighbouring particles share leaves):
    // the first lane of a run adds the run length
    const int lane = threadIdx.x & 31;
    const int prev = __shfl_up_sync(0xffffffffu, key, 1);
    const bool head = lane == 0 || prev != key;
    const unsigned heads = __ballot_sync(0xffffffffu, head);
    if (active && head) {
        const unsigned later = heads & ~((2u << lane) - 1u);  // heads after this lane
        const int next = later ? __ffs(later) - 1 : 32;
        atomicAdd(&counts[key], next - lane);
    }
}

// Exclusive scan, level 1: each block scans 1024 counts, writes local prefix and its total.
__global__ void k_scan_blocks(int64_t nleaf, const int *__restrict__ counts, int *__restrict__ out,
                              int *__restrict__ part, int *__restrict__ maxleaf)
{
    __shared__ int s[1024];
    __shared__ int smax[32];
    int64_t base = (int64_t)blockIdx.x * 1024;
    int t = threadIdx.x;  // 256 threads, 4 items each
    int v[4];
    int loc = 0, mx = 0;
    for (int k = 0; k < 4; ++k) {
        int64_t idx = base + 4 * t + k;
        v[k] = idx < nleaf ? counts[idx] : 0;
        loc += v[k];
        mx = max(mx, v[k]);
    }
    s[t] = loc;
    __syncthreads();
    for (int off = 1; off < 256; off <<= 1) {
        int add = t >= off ? s[t - off] : 0;
        __syncthreads();
        s[t] += add;
        __syncthreads();
    }
    int excl = s[t] - loc;
    for (int k = 0; k < 4; ++k) {
        int64_t idx = base + 4 * t + k;
        if (idx < nleaf) out[idx] = excl;
        excl += v[k];
    }
    if (t == 255) part[blockIdx.x] = s[255];
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((t & 31) == 0) smax[t >> 5] = mx;
    __syncthreads();
    if (t == 0) {
        int m = 0;
        for (int w = 0; w < 8; ++w) m = max(m, smax[w]);
        atomicMax(maxleaf, m);
    }
}

// Level 2: one block scans the block totals (sequential chunks per thread).
__global__ void k_scan_parts(int nparts, int *__restrict__ part, int *__restrict__ total)
{
    __shared__ int s[1024];
    int t = threadIdx.x;
    int per = (nparts + 1023) / 1024;
    int loc = 0;
    for (int k = 0; k < per; ++k) {
        int idx = t * per + k;
        if (idx < nparts) loc += part[idx];
    }
    s[t] = loc;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        int add = t >= off ? s[t - off] : 0;
        __syncthreads();
        s[t] += add;
        __syncthreads();
    }
    int excl = s[t] - loc;
    for (int k = 0; k < per; ++k) {
        int idx = t * per + k;
        if (idx < nparts) {
            int v = part[idx];
            part[idx] = excl;
            excl += v;
        }
    }
    if (t == 1023) *total = s[1023];
}

__global__ void k_scan_add(int64_t nleaf, int *__restrict__ out, const int *__restrict__ part)
{
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < nleaf) out[idx] += part[idx / 1024];
}

__global__ void k_scatter(int64_t n, const int *__restrict__ keys, const int *__restrict__ start,
                          int *__restrict__ fill, int *__restrict__ tmpidx)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int k = keys[i];
    int pos = start[k] + atomicAdd(&fill[k], 1);
    tmpidx[pos] = (int)i;
}

constexpr int LEAF_RANK_MAX = 128;  // leaves up to this size are sorted by ranking, larger ones bitonically

// One block per leaf: sort the leaf's particles by (octant of the leaf, caller index) in shared
// memory (by ranking for small leaves, else a bitonic sort), then write the permutation, the
// wrapped sorted positions, the leaf box, and the start and box of each octant (used to pick
// the P2P inner loop).
__device__ __forceinline__ int f2ord(float f) { return __float_as_int(f); }  // positions are >= 0

template <typename TIn, typename T>
__global__ void k_leaf_sort(const int *__restrict__ start, const int *__restrict__ tmpidx, const TIn *__restrict__ x,
                            BoxConst<TIn> bc, int nside, int *__restrict__ perm, typename V4<T>::type *__restrict__ xs,
                            float4 *__restrict__ bbox, int *__restrict__ oct_start, float4 *__restrict__ oct_box,
                            int *__restrict__ err)
{
    extern __shared__ unsigned long long s[];  // next power of two >= the largest leaf
    __shared__ int ocnt[8], omin[8][3], omax[8][3];
    int leaf = blockIdx.x;
    int b = start[leaf], e = start[leaf + 1];
    int cnt = e - b;
    if (threadIdx.x < 8) {
        ocnt[threadIdx.x] = 0;
        for (int d = 0; d < 3; ++d) {
            omin[threadIdx.x][d] = 0x7f7fffff;  // FLT_MAX bits
            omax[threadIdx.x][d] = 0;
        }
    }
    if (cnt <= 0) {
        if (threadIdx.x == 0) {
            bbox[2 * leaf] = make_float4(3e38f, 3e38f, 3e38f, 0.f);
            bbox[2 * leaf + 1] = make_float4(-3e38f, -3e38f, -3e38f, 0.f);
        }
        if (threadIdx.x < 8) {
            oct_start[8 * leaf + threadIdx.x] = 0;
            oct_box[16 * leaf + 2 * threadIdx.x] = make_float4(3e38f, 3e38f, 3e38f, 0.f);
            oct_box[16 * leaf + 2 * threadIdx.x + 1] = make_float4(-3e38f, -3e38f, -3e38f, 0.f);
        }
        return;
    }
    if (cnt > LEAF_SORT_CAP) {
        if (threadIdx.x == 0) atomicOr(err, ERRBIT_LEAF_OVERFLOW);
        return;
    }
    const int cz = leaf % nside, cy = (leaf / nside) % nside, cx = leaf / (nside * nside);
    // the input's own precision, as for the leaf keys
    const TIn Lt = bc.L, invL = bc.invL;
    const TIn s2 = bc.scale;  // octant cells (2 nside) per unit length
    int m = 1;
    while (m < cnt) m <<= 1;
    __syncthreads();
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        unsigned long long key = ~0ull;
        if (k < cnt) {
            int i = tmpidx[b + k];
            int o = 0;
            const int cc[3] = {cx, cy, cz};
            for (int d = 0; d < 3; ++d) {
                TIn v = wrap_coord<TIn>(x[3 * (int64_t)i + d], Lt, invL);
                int h = (int)(v * s2) - 2 * cc[d];
                h = h < 0 ? 0 : (h > 1 ? 1 : h);
                o = 2 * o + h;
            }
            key = ((unsigned long long)o << 32) | (unsigned)i;
        }
        s[k] = key;
    }
    __syncthreads();
    // one sorted element: permutation, wrapped position, octant count and box
    auto emit = [&](int pos, unsigned long long key) {
        int i = (int)(unsigned)(key & 0xffffffffull);
        int o = (int)(key >> 32);
        perm[b + pos] = i;
        T c0 = (T)wrap_coord<TIn>(x[3 * (int64_t)i + 0], Lt, invL);
        T c1 = (T)wrap_coord<TIn>(x[3 * (int64_t)i + 1], Lt, invL);
        T c2 = (T)wrap_coord<TIn>(x[3 * (int64_t)i + 2], Lt, invL);
        xs[b + pos] = make_v4<T>(c0, c1, c2, T(0));
        // boxes of the FP32-rounded positions the P2P kernel sees
        float cf[3] = {(float)c0, (float)c1, (float)c2};
        atomicAdd(&ocnt[o], 1);
        for (int d = 0; d < 3; ++d) {
            atomicMin(&omin[o][d], f2ord(cf[d]));
            atomicMax(&omax[o][d], f2ord(cf[d]));
        }
    };
    if (cnt <= LEAF_RANK_MAX) {
        // the keys are distinct (the caller index is the low word): an element's place is the
        // number of smaller keys, found by one pass over the leaf's keys without a barrier
        for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
            const unsigned long long key = s[k];
            int r = 0;
            for (int j = 0; j < cnt; ++j) r += s[j] < key ? 1 : 0;
            emit(r, key);
        }
    } else {
        for (int size = 2; size <= m; size <<= 1)
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int k = threadIdx.x; k < m; k += blockDim.x) {
                    int q = k ^ stride;
                    if (q > k) {
                        bool up = (k & size) == 0;
                        unsigned long long a = s[k], c = s[q];
                        if ((a > c) == up) {
                            s[k] = c;
                            s[q] = a;
                        }
                    }
                }
                __syncthreads();
            }
        for (int k = threadIdx.x; k < cnt; k += blockDim.x) emit(k, s[k]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        float lo[3] = {3e38f, 3e38f, 3e38f}, hi[3] = {-3e38f, -3e38f, -3e38f};
        for (int o = 0; o < 8; ++o) {
            oct_start[8 * leaf + o] = acc;
            acc += ocnt[o];
            if (ocnt[o] > 0) {
                float l[3], hh[3];
                for (int d = 0; d < 3; ++d) {
                    l[d] = __int_as_float(omin[o][d]);
                    hh[d] = __int_as_float(omax[o][d]);
                    lo[d] = fminf(lo[d], l[d]);
                    hi[d] = fmaxf(hi[d], hh[d]);
                }
                oct_box[16 * leaf + 2 * o] = make_float4(l[0], l[1], l[2], 0.f);
                oct_box[16 * leaf + 2 * o + 1] = make_float4(hh[0], hh[1], hh[2], 0.f);
            } else {
                oct_box[16 * leaf + 2 * o] = make_float4(3e38f, 3e38f, 3e38f, 0.f);
                oct_box[16 * leaf + 2 * o + 1] = make_float4(-3e38f, -3e38f, -3e38f, 0.f);
            }
        }
        bbox[2 * leaf] = make_float4(lo[0], lo[1], lo[2], 0.f);
        bbox[2 * leaf + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
    }
}

template <typename TIn, typename T> static int tree_impl(Ctx *c, const TIn *x)
{
    cudaStream_t st = c->stream;
    int64_t n = c->n, nleaf = c->nleaf;
    cudaMemsetAsync(c->counts.p, 0, nleaf * sizeof(int), st);
    cudaMemsetAsync(c->fill.p, 0, nleaf * sizeof(int), st);
    cudaMemsetAsync(c->maxleaf.p, 0, sizeof(int), st);
    int nb = (int)((n + 255) / 256);
    k_keys<TIn><<<nb, 256, 0, st>>>(n, x, c->nside, box_const<TIn>(c->cfg.box, (double)c->nside), (int *)c->keys.p,
                                    (int *)c->counts.p, (int *)c->err.p);
    int nparts = (int)((nleaf + 1023) / 1024);
    int *start = (int *)c->leaf_start.p;
    int *part = (int *)c->scan_part.p;
    k_scan_blocks<<<nparts, 256, 0, st>>>(nleaf, (int *)c->counts.p, start, part, (int *)c->maxleaf.p);
    k_scan_parts<<<1, 1024, 0, st>>>(nparts, part, start + nleaf);
    k_scan_add<<<(int)((nleaf + 255) / 256), 256, 0, st>>>(nleaf, start, part);
    k_scatter<<<nb, 256, 0, st>>>(n, (int *)c->keys.p, start, (int *)c->fill.p, (int *)c->tmpidx.p);
    c->launches += 4;  // k_keys, three scan kernels precede k_scatter
    VFMM_CUDA_CHECK_LAUNCH(c);
    return VFMM_OK;
}

template <typename TIn, typename T> static int leaf_sort_impl(Ctx *c, const TIn *x, int max_leaf)
{
    int m = 1;
    while (m < max_leaf) m <<= 1;
    const size_t sm = (size_t)m * sizeof(unsigned long long);
    static bool attr[2] = {false, false};
    const int ai = sizeof(TIn) == 8 ? 1 : 0;
    if (!attr[ai]) {
        cudaError_t e = cudaFuncSetAttribute(k_leaf_sort<TIn, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(LEAF_SORT_CAP * sizeof(unsigned long long)));
        if (e != cudaSuccess) {
            c->last_error = std::string("leaf sort shared memory: ") + cudaGetErrorString(e);
            return VFMM_ERR_CUDA;
        }
        attr[ai] = true;
    }
    int *start = (int *)c->leaf_start.p;
    k_leaf_sort<TIn, T><<<(unsigned)c->nleaf, 64, sm, c->stream>>>(start, (int *)c->tmpidx.p, x,
                                                                  box_const<TIn>(c->cfg.box, 2.0 * c->nside), c->nside,
                                                                  (int *)c->perm.p, (typename V4<T>::type *)c->xs.p,
                                                                  (float4 *)c->bbox.p, (int *)c->oct_start.p,
                                                                  (float4 *)c->oct_box.p, (int *)c->err.p);
    VFMM_CUDA_CHECK_LAUNCH(c);
    return VFMM_OK;
}

int launch_tree(Ctx *c, const void *x)
{
    if (c->f64) return tree_impl<double, double>(c, (const double *)x);
    return tree_impl<float, float>(c, (const float *)x);
}

int launch_leaf_sort(Ctx *c, const void *x, int max_leaf)
{
    if (c->f64) return leaf_sort_impl<double, double>(c, (const double *)x, max_leaf);
    return leaf_sort_impl<float, float>(c, (const float *)x, max_leaf);
}

}  // namespace vfmm

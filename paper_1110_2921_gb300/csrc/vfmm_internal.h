// Internal declarations shared by the translation units of libvfmm.
#pragma once

#include "vfmm.h"

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

namespace vfmm {

constexpr int PMAX = 16;          // largest supported expansion order
constexpr int NPHASE = 8;         // timed phases (see vfmm_get_timings)
constexpr int MAX_DEPTH = 8;      // deepest octree level
constexpr int LEAF_SORT_CAP = 4096;  // per-leaf sort capacity (32 KB of 64-bit keys)
constexpr int OUT_ROWS = 128;     // rows of every packed translation matrix (output coefficients, padded)
constexpr int NT = 343;           // M2L offsets t in [-3,3]^3
constexpr int TC_KBYTES = 32;     // tensor-core M2L: K bytes of one pipeline stage per operand row
constexpr int TC_KG = TC_KBYTES / 16;   // 16-byte k-groups per stage
constexpr int TC_A_TILE = 128 * TC_KBYTES;  // bytes of one translation-matrix tile (128 rows)

// P2P beside the concurrent far field: VFMM_P2P_SHARED_BLOCKS > 0 runs it as a persistent grid
// of that many one-warp blocks per SM (leaving room for far-field blocks on every SM), and
// VFMM_FORK_AT_M2L = 1 runs the upward pass in line and forks only the M2L and the downward
// pass; VFMM_M2L_LEAF_FIRST = 1 issues the leaf level's M2L first (with the fork at the M2L
// its hi/lo split then runs in line, so the first launch beside the P2P is the leaf M2L).
// Measured at 256^3 with the cp.async source-line M2L (step ms, every phase 73.7 ms in line):
// one block per task and the fork before the P2M 72.9; fork at the M2L 73.1; persistent 16 or
// 20 blocks per SM 74-80 (the M2L then waits for the P2P).  With the TMA source-line M2L
// (every phase 62.2 ms in line): default 60.7; fork at the M2L 60.85, and with the leaf level
// first 60.9; leaf first alone 60.8; two M2L stages (with or without a 64-register cap, to leave
// room for more P2P warps beside an M2L CTA) 61.6-61.8; fork, leaf first and a persistent P2P
// of 20 blocks per SM 62.0 (no M2L CTA fits beside them).  Defaults: the first.
#ifndef VFMM_P2P_SHARED_BLOCKS
#define VFMM_P2P_SHARED_BLOCKS 0
#endif
#ifndef VFMM_FORK_AT_M2L
#define VFMM_FORK_AT_M2L 0
#endif
// lowest level whose M2L runs on the tensor cores (the levels below take the CUDA-core GEMM);
// at 256^3 (step ms): 3 (default) 58.7, 4 58.9, 5 60.5
#ifndef VFMM_TC_MIN_LEVEL
#define VFMM_TC_MIN_LEVEL 3
#endif
#ifndef VFMM_M2L_LEAF_FIRST
#define VFMM_M2L_LEAF_FIRST 0
#endif

// device error word bits
constexpr int ERRBIT_LEAF_OVERFLOW = 1;
constexpr int ERRBIT_BOUNDS = 2;
constexpr int ERRBIT_TIMEOUT = 4;
constexpr int ERRBIT_NONFINITE = 8;  // a position given to the tree build is NaN or infinite

// Checked build (-DVFMM_CHECK=1): the gather indices of the M2L/M2M/L2L GEMM, the tensor-core
// M2L and the P2P are range-checked; an index out of range sets ERRBIT_BOUNDS and is replaced
// by 0, so the access stays in bounds and the evaluation reports VFMM_ERR_BOUNDS.  The default
// build checks nothing (every index is in range by construction).
#ifndef VFMM_CHECK
#define VFMM_CHECK 0
#endif
#ifdef __CUDACC__
template <typename I> __device__ __forceinline__ I checked_index(I idx, I limit, int *err)
{
#if VFMM_CHECK
    if (idx < 0 || idx >= limit) {
        atomicOr(err, ERRBIT_BOUNDS);
        return 0;
    }
#else
    (void)limit;
    (void)err;
#endif
    return idx;
}
#endif

namespace ops {
double sfac(int n, int m);
std::vector<double> m2l_hat(const double t[3], int p);
std::vector<double> m2m_hat(const double e[3], double ratio, int p);
std::vector<double> l2l_hat(const double e[3], int p);
std::vector<double> lattice_operator(int p, int S);
}  // namespace ops

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

// Parameters of the gathered-column GEMM used by M2M, M2L and L2L on the CUDA cores.
// C[cell_t][comp][k] (+)= sum_{kblocks} sum_j AT[mat][j][k] * B[src(cell_t, t)][comp][j]
struct GemmParams {
    const void *AT;   // [nmat][pc][OUT_ROWS] transposed matrices (input-major)
    const void *B;    // source coefficient rows [ncell_src][3][pc]
    void *C;          // target rows [ncell_tgt][3][pc]
    const int4 *kb;   // k-blocks (mat, tx, ty, tz)
    int kb_off[8];    // per target parity group: first k-block
    int kb_cnt[8];    // per target parity group: number of k-blocks
    int n_src;        // cells per side at the source level
    int n_tgt;        // cells per side at the target level
    int mode;         // 0 = M2L (src = wrap(c + t)), 1 = M2M (src = 2c + t), 2 = L2L (src = c >> 1)
    int grouped;      // 1: targets split by parity (grid.y = 8); 0: all cells
    int accumulate;   // C += instead of C =
    int pc;           // padded coefficient stride (multiple of 16)
    int ksplit;       // k-block slices summed by a second pass (1 = none); set by launch_gemm
    void *partial;    // [ksplit][n_tgt^3][3][pc] slice results when ksplit > 1
    int *err;         // device error word (bounds bit of the checked build); set by launch_gemm
};

struct TcParams {
    const void *Ahi, *Alo;  // [NT][nchunk][tile bytes] pre-tiled translation matrices
    const void *Bhi, *Blo;  // multipole hi/lo rows [ncell][3][pc] (bf16 or tf32-in-fp32)
    float *C;               // local rows [ncell][3][pc] (FP32), stored
    const int4 *kb;
    int kb_off[8], kb_cnt[8];
    int n;                  // cells per side
    int pc;                 // padded coefficient stride
    int nchunk;             // K chunks per matrix
    int *err;               // device error word
    int ksplit;             // offset slices (blockIdx.z) summed by a second pass (1 = none)
    float *partial;         // [ksplit][n^3][3][pc] slice results when ksplit > 1
    long long wait_limit;   // tries of each pipeline mbarrier wait before the CTA gives up
};

struct Ctx {
    vfmm_config cfg;
    cudaStream_t stream = nullptr;
    int p = 10, nc = 121, pc = 128;
    bool f64 = false;
    size_t esz = 4;  // element size of T

    // tree
    int64_t n = 0;
    int depth = 0, nside = 1;
    int64_t nleaf = 1;
    int max_leaf = 0;
    int last_R = 0;
    int last_Rc = 0;  // outer ring of the Gaussian-tail correction (0: none)
    bool built = false;
    double leaf_w = 0.0;

    // device buffers
    DevBuf xs, gs, perm, keys, leaf_start, counts, fill, tmpidx, scan_part, err, maxleaf;
    DevBuf bbox;                   // per leaf: float4 lo, float4 hi of its particles
    DevBuf oct_start, oct_box;     // per leaf: 8 octant starts (relative), 8 x (lo, hi) octant boxes
    DevBuf mexp, lexp;             // all levels, T
    DevBuf mhi, mlo;               // tensor-core copies of the multipoles (largest level)
    DevBuf gemm_part;              // split-k partial results of the CUDA-core GEMM (small levels)
    DevBuf spec_work, spec_E;      // energy spectrum: FP64 complex lattice copy, shell sums
    DevBuf ufar, sfar, gfar;       // far-field u, S (or grad u) in sorted order, T
    DevBuf adj_u, adj_g1, adj_g2;  // adjoint temporaries (caller order)
    DevBuf rk_u1, rk_s1, rk_u2, rk_s2, rk_x1, rk_g1;  // time-step temporaries (caller order)
    DevBuf diag;                   // 8 FP64 sums
    DevBuf rg_om, rg_r, rg_d, rg_q, rg_t1, rg_t2, rg_dots;  // reinitialisation temporaries
    int depth_override = -1;       // tree depth forced by vfmm_reinit
    DevBuf at_m2l, at_m2m, at_l2l; // CUDA-core matrices, T
    // transposed operators of the adjoint (built on its first FMM call): at_m2l_t[t] = M2L(-t)^T,
    // at_l2l_t[b] = L2L_b^T (applied child -> parent), at_m2m_t[b] = M2M_b^T (parent -> child),
    // and the tensor-core tiles of at_m2l_t
    DevBuf at_m2l_t, at_m2m_t, at_l2l_t, tc_hi_t, tc_lo_t;
    bool have_transposed = false;
    DevBuf tc_hi, tc_lo;           // tensor-core tiles
    DevBuf m2m_f64, lattice_f64;   // root accumulation and lattice operator, FP64
    DevBuf root_m;                 // FP64 root multipole
    DevBuf kblocks;                // k-block lists (device)
    DevBuf hx, hg, hu, hs;         // staging for vfmm_eval_host
    std::vector<size_t> lvl_off;   // element offset of each level in mexp / lexp

    // k-block lists (offsets into kblocks)
    int kb_m2l_off[3][8], kb_m2l_cnt[3][8];  // index = near rings R at that level (1 or 2)
    DevBuf cls;                              // M2L offset classes of the source-line kernel
    int cls_off[3][8], cls_cnt[3][8];        // in classes (three int4 each)
    int kb_m2m_off = 0, kb_l2l_off[8];

    cudaEvent_t ev[12];            // [10] far field done (side stream), [11] fork
    cudaStream_t side = nullptr;   // high-priority stream of the far field when it overlaps the P2P
    bool overlap = true;           // FP32 velocity/stretching: far field concurrent with the P2P
    bool have_events = false;
    bool timed_eval = false;
    int64_t launches = 0;      // kernels launched by the last build + evaluation
    long long wait_limit = 1LL << 26;  // tries of each tensor-core pipeline wait (vfmm_set_wait_limit)
    int sm_count = 152;                // multiprocessors of the device (set at create)
    int p2p_shared_blocks = 0;         // > 0: FP32 P2P as a persistent grid of this many blocks per SM
    double timings[NPHASE];
    std::string last_error;
};

// kernels.cu entry points (host launchers)
int launch_tree(Ctx *c, const void *x);  // keys, counts, scan, scatter into leaves
int launch_leaf_sort(Ctx *c, const void *x, int max_leaf);  // per-leaf octant order, boxes
int launch_gather_gamma(Ctx *c, const void *gamma);
int launch_p2m(Ctx *c);
int launch_gemm(Ctx *c, const GemmParams &gp, int ngroups, int64_t ncell_group);
int launch_root(Ctx *c);
int launch_l2p(Ctx *c, bool grad);
// transposed far field: E^T (w sorted as V4 -> leaf lambda in lexp), P^T (+ source-position term,
// caller order; dgamma accumulated, dxf written), lattice^T + root M2M^T (lexp level 0 -> mexp level 1)
int launch_dual_p2m(Ctx *c, const void *ws_sorted);
int launch_dual_l2p(Ctx *c, const void *gamma, void *dgamma, void *dxf);
int launch_root_t(Ctx *c);
// u_out[perm[i]] += ufar[i], s_out[perm[i]] += sfar[i] (FP32)
int launch_add_far(Ctx *c, void *u_out, void *s_out);
// energy spectrum of an n^3 x 3 lattice velocity into E_dev[0..kmax] (work: 3 n^3 double2)
int launch_spectrum(Ctx *c, int n, const void *u, int kmax, double2 *work, double *E_dev);
// sums of d^2, d^3, d^4 over the longitudinal derivatives of an n x 9 gradient into out_dev[0..2]
int launch_moments(Ctx *c, int64_t n, const void *g, double *out_dev);
int launch_p2p_grad(Ctx *c, int R, double sigma, const void *ufar, const void *gfar, void *u_out, void *g_out,
                    int direct_K);
// dx = G1^T w + G2^T gamma (+ extra when not null), caller order
int launch_adjoint_combine(Ctx *c, const void *G1, const void *w, const void *G2, const void *gamma, const void *extra,
                           void *dx);
// direct_K >= 0: direct sum over every leaf of the (2K+1)^3 image boxes; -1: the FMM near field (R rings)
int launch_p2p(Ctx *c, int R, int Rc, double sigma, const void *ufar, const void *sfar, void *u_out,
               void *s_out, int direct_K);
int64_t p2p_pairs_read();  // checked build: pairs of the last FP32 P2P launch (0 otherwise)
int launch_tc_m2l(Ctx *c, int level, int R, bool bf16);  // R: near rings excluded at this level
// classes of one parity's M2L list for the source-line kernel: per class three int4
// {source parity, x shift, y shift, count}, {tile, z shift, tile, z shift} x 2
void build_line_classes(const std::vector<int4> &kb, int off, int cnt, int g, std::vector<int4> &out);
int launch_split(Ctx *c, int level, bool bf16);
// C (= or +=) sum over z < nsplit of partial[z][i], i < count, in z order (FP32 or FP64 by c->f64 unless forced)
int launch_split_reduce(Ctx *c, int nsplit, int64_t count, const void *partial, void *C, int accumulate, bool f32);
size_t split_count(int level, int pc);  // hi/lo elements launch_split writes for one level
void set_constants(int p);
// largest shared-memory carveout for the kernels of each translation unit (see prefer_max_shared)
void set_carveouts_expansions();
void set_carveouts_p2p();
void set_carveouts_m2l();
int launch_axpy3(Ctx *c, int64_t n, const void *a, const void *b, const void *d, double coef, double wrap_L, void *out);
int launch_diag(Ctx *c, int64_t n, const void *x, const void *g, const void *u, double *out_dev);
int launch_reinit(Ctx *c, int m, double sigma, double sigma0, int iters, int R, void *x_new, void *g_new,
                  double *residual);

}  // namespace vfmm
